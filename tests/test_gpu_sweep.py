"""The multi-shift slot engine and the two-sided sketch, through the C ABI.

* transec_shifted_columns: every column at every energy of a window from one Krylov
  run per column (A(E, k) = A(E0, k) + (E - E0) 1, Sec. II.A), against the oracle's
  dense LU at k and at -k (the shadow system, A(E, k)^T = A(E, -k), Sec. II.B), and
  against the plain engine's separate solves; runs that retire and refill give the
  same numbers as runs that all fit at once.
* transec_transmission_sketch: the full trace T(E, k) = 4 Tr[Gamma_L G^dagger Gamma_R G]
  from random left and right right-hand sides, against the dense-LU full trace over
  every left-CAP column, at k and -k, within |dT| <= 1e-6 (the metric's bar); also
  with P-symmetric COCG runs on inversion-symmetric cells (Sec. II.C).

Both arithmetics of the engine are covered: FP64 (precision 0) and double-float
(precision 2: vectors and the stencil, vector and per-shift updates in pairs of floats).
"""

import numpy as np
import pytest

from tests.gpu_util import context, library, need_gpu
import dataclasses

from workloads import inversion_symmetrize, small_instance
from oracle.transmission import left_support, transmission_dense

pytestmark = pytest.mark.gpu

TOL_T = 1e-6


def _inst(kf, seed=5, nx=6, ny=5, nz=40, order=8, ncap=8):
    return small_instance(nx, ny, nz, 0.45, order, ncap, v_amp=0.7, kfrac=(kf, (-kf[0], -kf[1])),
                          energies=(0.3,), seed=seed)


def _dense_cols(inst, e, kf, cols):
    g = inst.grid
    return transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, kf, cols)[1]


PRECISIONS = [0, 2]


@pytest.mark.parametrize("precision", PRECISIONS)
def test_shifted_columns_match_dense_lu_at_both_k(precision):
    need_gpu()
    kf = (0.21, -0.34)
    inst = _inst(kf)
    g = inst.grid
    energies = np.linspace(0.12, 0.78, 9)
    sup = left_support(g, inst.gamma_l)
    cols = np.array([0, 17, 101, 239], np.int64)
    with context(inst, precision=precision) as tr:
        r = tr.shifted_columns(energies, np.zeros(cols.size, np.int32), cols)
    assert np.all(r["status"] == 0), r["status"]
    for s, e in enumerate(energies):
        ref_p = _dense_cols(inst, e, kf, sup[cols])
        ref_m = _dense_cols(inst, e, (-kf[0], -kf[1]), sup[cols])
        assert np.abs(r["t"][:, s] - ref_p).max() <= TOL_T * 1e-3, (e, r["t"][:, s], ref_p)
        assert np.abs(r["t_minus"][:, s] - ref_m).max() <= TOL_T * 1e-3, (e, r["t_minus"][:, s], ref_m)
    # the run length is set by the slowest energy; every energy reports its own stop
    assert np.all(r["iters"] > 0) and np.all(r["iters"].max(axis=1) >= r["iters"].min(axis=1))


@pytest.mark.parametrize("precision", PRECISIONS)
def test_shifted_columns_agree_with_separate_solves_and_refill(precision):
    need_gpu()
    kf = (0.4375, 0.1875)
    inst = _inst(kf, seed=9, nx=5, ny=6, nz=36, order=12, ncap=7)
    energies = np.array([0.2, 0.35, 0.5, 0.65])
    cols = np.array([3, 44, 90, 131, 170], np.int64)
    ik = np.zeros(cols.size, np.int32)
    with context(inst, tol=1e-11, precision=precision) as tr:
        all_in = tr.shifted_columns(energies, ik, cols)
        tr.set_solver(slots=2)  # five runs through two slots: retire and refill on the GPU
        refill = tr.shifted_columns(energies, ik, cols)
        tr.set_solver(slots=0, precision=0)
        sep = [tr.column_contributions(np.full(cols.size, e), ik, cols) for e in energies]
    assert np.all(all_in["status"] == 0) and np.all(refill["status"] == 0)
    np.testing.assert_array_equal(all_in["t"], refill["t"])
    np.testing.assert_array_equal(all_in["t_minus"], refill["t_minus"])
    for s in range(energies.size):
        assert np.abs(all_in["t"][:, s] - sep[s]["t"]).max() <= 1e-9
        assert np.abs(all_in["t_minus"][:, s] - sep[s]["t_minus"]).max() <= 1e-9


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("kf,order", [((0.23, -0.37), 8), ((0.0, 0.0), 4), ((0.4375, 0.3125), 12)])
def test_sketch_full_trace_matches_dense_lu(kf, order, precision):
    need_gpu()
    inst = _inst(kf, seed=13, nx=6, ny=6, nz=44, order=order, ncap=9)
    g = inst.grid
    energies = np.linspace(0.1, 0.9, 7)
    with context(inst, precision=precision) as tr:
        r = tr.transmission_sketch(energies, [0], s_left=8, s_right=16, seed=3)
    assert np.all(r["status"] == 0), r["status"]
    for s, e in enumerate(energies):
        tp, _ = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, kf)
        tm, _ = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, (-kf[0], -kf[1]))
        assert abs(r["T"][0, s] - tp) <= TOL_T, (e, r["T"][0, s], tp)
        assert abs(r["T_minus"][0, s] - tm) <= TOL_T, (e, r["T_minus"][0, s], tm)
        assert 1 <= r["rank"][0, s] <= 8


def test_sketch_two_k_groups_and_seeds():
    """Two k-points in one call (independent run groups), and a second random draw:
    both estimates agree with dense LU."""
    need_gpu()
    kf1, kf2 = (0.3125, -0.1875), (-0.0625, 0.4375)
    inst = small_instance(5, 5, 40, 0.45, 8, 8, v_amp=0.7, kfrac=(kf1, kf2), energies=(0.3,), seed=21)
    g = inst.grid
    energies = np.array([0.25, 0.55])
    with context(inst) as tr:
        a = tr.transmission_sketch(energies, [0, 1], s_left=6, s_right=12, seed=1)
        b = tr.transmission_sketch(energies, [1, 0], s_left=6, s_right=12, seed=2)
    for r, order in ((a, (kf1, kf2)), (b, (kf2, kf1))):
        assert np.all(r["status"] == 0)
        for q, kf in enumerate(order):
            for s, e in enumerate(energies):
                tp, _ = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, kf)
                assert abs(r["T"][q, s] - tp) <= TOL_T


def test_sweep_argument_checks():
    need_gpu()
    pkg = library()
    inst = _inst((0.1, 0.2))
    with context(inst) as tr:
        for bad in (dict(s_left=0, s_right=4), dict(s_left=8, s_right=4), dict(s_left=33, s_right=40),
                    dict(s_left=4, s_right=65)):
            with pytest.raises(pkg.TransecError) as ei:
                tr.transmission_sketch([0.3], [0], **bad)
            assert ei.value.status == pkg.EINVAL
        with pytest.raises(pkg.TransecError):
            tr.transmission_sketch([0.3], [5])
        with pytest.raises(pkg.TransecError):
            tr.shifted_columns([0.3], [0], [10 ** 6])
        with pytest.raises(pkg.TransecError):
            tr.shifted_columns([float("nan")], [0], [1])


@pytest.mark.parametrize("precision", PRECISIONS)
def test_sketch_unequal_spacings(precision):
    """hx, hy, hz all different: the stencil takes each axis's own coefficients."""
    need_gpu()
    kf = (0.3125, -0.4375)
    inst = small_instance(6, 5, 40, 0.45, 8, 8, v_amp=0.7, kfrac=(kf,), energies=(0.3,), seed=23,
                          hy=0.5, hz=0.4)
    g = inst.grid
    energies = np.array([0.2, 0.45, 0.7])
    with context(inst, precision=precision) as tr:
        r = tr.transmission_sketch(energies, [0], s_left=8, s_right=16, seed=4)
    assert np.all(r["status"] == 0)
    for s, e in enumerate(energies):
        tp, _ = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, kf)
        assert abs(r["T"][0, s] - tp) <= TOL_T


def test_double_float_results_that_stall_are_solved_again_in_fp64():
    """A stall limit far too short makes every double-float run stop early: every
    result then comes from the FP64 re-solve inside the same call, bit-identical to an
    FP64 call for the unit columns, and counted in the stats."""
    need_gpu()
    kf = (0.21, -0.34)
    inst = _inst(kf)
    energies = np.linspace(0.2, 0.6, 5)
    cols = np.array([5, 60, 200], np.int64)
    ik = np.zeros(cols.size, np.int32)
    with context(inst, precision=0) as tr:
        ref = tr.shifted_columns(energies, ik, cols)
        sk_ref = tr.transmission_sketch(energies, [0], s_left=8, s_right=16, seed=3)
        tr.set_solver(precision=2, df_stall_its=5)
        tr.stats_reset()
        got = tr.shifted_columns(energies, ik, cols)
        redone_cols = tr.sweep_stats()["fp64_redone"]
        sk = tr.transmission_sketch(energies, [0], s_left=8, s_right=16, seed=3)
        redone_all = tr.sweep_stats()["fp64_redone"]
    assert np.all(ref["status"] == 0) and np.all(got["status"] == 0)
    assert redone_cols == cols.size * energies.size
    np.testing.assert_array_equal(got["t"], ref["t"])
    np.testing.assert_array_equal(got["t_minus"], ref["t_minus"])
    assert redone_all - redone_cols == energies.size
    assert np.all(sk["status"] == 0)
    assert np.abs(sk["T"] - sk_ref["T"]).max() <= TOL_T


def _sym_inst(kf, nx, ny, nz, order, seed):
    inst = small_instance(nx, ny, nz, 0.45, order, 9, v_amp=0.7, kfrac=(kf, (-kf[0], -kf[1])),
                          energies=(0.3,), seed=seed)
    return dataclasses.replace(inst, v=inversion_symmetrize(inst.v))


@pytest.mark.parametrize("kf,order,shape", [((0.23, -0.37), 8, (6, 6, 44)), ((0.4375, 0.3125), 12, (5, 4, 40)),
                                            ((0.0, 0.0), 4, (7, 6, 40))])
def test_psym_sketch_matches_dense_lu(kf, order, shape):
    """P-symmetric COCG runs (one operator application per iteration) on cells whose V
    is invariant under the in-plane inversion: T(E, k) and T(E, -k) against the dense-LU
    full trace; the -k estimate is the mirrored data, equal to T to rounding; the runs
    update one half (half the per-shift points of transpose BiCG)."""
    need_gpu()
    inst = _sym_inst(kf, *shape, order, seed=17)
    g = inst.grid
    energies = np.linspace(0.1, 0.9, 7)
    with context(inst, precision=2, psym=1) as tr:
        tr.stats_reset()
        r = tr.transmission_sketch(energies, [0], s_left=8, s_right=16, seed=3)
        ps = tr.sweep_stats()
        tr.set_solver(psym=0)
        tr.stats_reset()
        b = tr.transmission_sketch(energies, [0], s_left=8, s_right=16, seed=3)
        bs = tr.sweep_stats()
    assert np.all(r["status"] == 0) and np.all(b["status"] == 0), (r["status"], b["status"])
    assert ps["fp64_redone"] == 0
    for s, e in enumerate(energies):
        tp, _ = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, kf)
        tm, _ = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, (-kf[0], -kf[1]))
        assert abs(r["T"][0, s] - tp) <= TOL_T, (e, r["T"][0, s], tp)
        assert abs(r["T_minus"][0, s] - tm) <= TOL_T, (e, r["T_minus"][0, s], tm)
        assert abs(r["T"][0, s] - b["T"][0, s]) <= TOL_T
        assert 1 <= r["rank"][0, s] <= 8
    assert np.abs(r["T"] - r["T_minus"]).max() <= 1e-9
    # per-shift work: one half per iteration against two
    per_it_p = ps["shift_points"] / max(1, ps["iters"])
    per_it_b = bs["shift_points"] / max(1, bs["iters"])
    assert per_it_p < 0.75 * per_it_b, (per_it_p, per_it_b)


def test_psym_argument_checks():
    need_gpu()
    pkg = library()
    kf = (0.23, -0.37)
    sym = _sym_inst(kf, 6, 6, 40, 8, seed=17)
    asym = _inst(kf)
    wide = _sym_inst(kf, 30, 30, 30, 4, seed=2)  # 900 points: the plane does not fit one tile
    for inst, prec in ((sym, 0), (asym, 2), (wide, 2)):
        with context(inst, precision=prec, psym=1) as tr:
            with pytest.raises(pkg.TransecError) as ei:
                tr.transmission_sketch([0.3], [0], s_left=4, s_right=8)
            assert ei.value.status == pkg.EINVAL


def test_sketch_guard_redoes_disagreeing_results():
    """The a-posteriori checks acting: with the guard below rounding, every result is
    computed again with doubled sketches (counted in the stats) and still matches dense
    LU, as do the results under the default guard (1e-7); the missed-energy estimate
    is reported for every result and is at most T."""
    need_gpu()
    kf = (0.23, -0.37)
    inst = _inst(kf, seed=13, nx=6, ny=6, nz=44, order=8, ncap=9)
    g = inst.grid
    energies = np.linspace(0.2, 0.8, 4)
    with context(inst, precision=2) as tr:
        tr.stats_reset()
        a = tr.transmission_sketch(energies, [0], s_left=8, s_right=16, seed=3)
        ga = tr.sweep_stats()["guard_redone"]
        tr.set_solver(sketch_guard=1e-300)
        tr.stats_reset()
        b = tr.transmission_sketch(energies, [0], s_left=8, s_right=16, seed=3)
        gb = tr.sweep_stats()["guard_redone"]
    assert gb >= energies.size and gb >= ga
    assert np.all(b["iters"] >= a["iters"])
    assert np.all(np.isfinite(a["miss"])) and np.all(a["miss"] >= 0)
    assert np.all(a["miss"] <= 4 * np.maximum(a["T"], 1e-30) + 1e-12)
    for r in (a, b):
        assert np.all(r["status"] == 0)
        for s, e in enumerate(energies):
            tp, _ = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, kf)
            assert abs(r["T"][0, s] - tp) <= TOL_T


def test_sketch_matches_oracle_sketch_with_the_same_draws():
    """The sketch's arithmetic, not only its limit: with fewer left vectors than the rank
    of M (a truncated sketch, off the exact T by up to 0.6 here), the GPU's T(E, k),
    T(E, -k) and missed-energy estimate equal the oracle's two-sided sketch computed
    with the same splitmix64 draws (FP64 runs, guard off)."""
    need_gpu()
    from oracle.sketch import sketch_transmission

    kf = (0.23, -0.37)
    inst = small_instance(8, 8, 36, 0.4, 4, 8, v_amp=0.2, kfrac=(kf, (-kf[0], -kf[1])), energies=(0.3,), seed=13)
    g = inst.grid
    energies = np.array([1.2, 2.0, 3.0])
    with context(inst, precision=0, sketch_guard=-1.0) as tr:
        r = tr.transmission_sketch(energies, [0], s_left=3, s_right=6, seed=5)
    assert np.all(r["status"] == 0), r["status"]
    for s, e in enumerate(energies):
        tp, tm, miss = sketch_transmission(g, inst.v, inst.gamma_l, inst.gamma_r, e, kf, 3, 6, 5)
        assert abs(r["T"][0, s] - tp) <= 1e-6 * max(1.0, tp), (e, r["T"][0, s], tp)
        assert abs(r["T_minus"][0, s] - tm) <= 1e-6 * max(1.0, tm), (e, r["T_minus"][0, s], tm)
        assert abs(r["miss"][0, s] - miss) <= 1e-6 * max(1.0, miss), (e, r["miss"][0, s], miss)
