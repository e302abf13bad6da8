"""Solver parity: the GPU library against the CPU oracle, through the C ABI.

Tolerance: |dT| <= 1e-6 absolute per (E, k), the accuracy the method is required to
reach; per column the solver stops at ||A x - e_j|| <= 1e-10, so the column
contributions agree far below that bar on these well-conditioned small cases.
"""

import numpy as np
import pytest

from tests.gpu_util import context, need_gpu
from workloads import free_electron_slab, small_instance
from oracle.transmission import left_support, transmission_dense
from oracle.closed_form import separable_transmission

pytestmark = pytest.mark.gpu

TOL_T = 1e-6


def _dense_all(inst):
    g = inst.grid
    out = np.zeros((len(inst.energies), len(inst.kfrac)))
    cols = {}
    for i, e in enumerate(inst.energies):
        for k, kf in enumerate(inst.kfrac):
            out[i, k], cols[(i, k)] = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, kf)
    return out, cols


@pytest.mark.parametrize(
    "nx,ny,nz,order,kfrac",
    [
        (5, 4, 24, 2, ((0.0, 0.0),)),                        # COCG, real H
        (6, 5, 26, 8, ((0.5, 0.0), (0.0, 0.5))),              # COCG, real phases
        (6, 5, 26, 12, ((0.21, -0.34), (-0.21, 0.34))),       # BiCG with the mirror folded
        (7, 3, 22, 6, ((0.125, 0.375), (0.3, -0.1), (0.0, 0.0))),  # mixed groups
    ],
)
def test_transmission_matches_dense(nx, ny, nz, order, kfrac):
    need_gpu()
    inst = small_instance(nx, ny, nz, 0.45, order, 6, v_amp=0.7, kfrac=kfrac,
                          energies=(0.15, 0.55, 1.1), seed=nx + 10 * order)
    ref, _ = _dense_all(inst)
    with context(inst) as tr:
        out = tr.transmission(inst.energies, len(kfrac))
    assert np.all(out["status"] == 0), out["status"]
    assert np.abs(out["T"] - ref).max() <= TOL_T, (out["T"], ref)
    assert np.allclose(out["T_avg"], ref @ inst.kweights, atol=TOL_T, rtol=0)


def test_column_contributions_and_shadow_columns():
    need_gpu()
    kf = (0.27, -0.16)
    inst = small_instance(6, 5, 28, 0.45, 10, 6, v_amp=0.8, kfrac=(kf, (-kf[0], -kf[1])),
                          energies=(0.42,), seed=21)
    g = inst.grid
    _, tj_p = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, 0.42, kf)
    _, tj_m = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, 0.42, (-kf[0], -kf[1]))
    nrhs = len(left_support(g, inst.gamma_l))
    pos = np.arange(0, nrhs, 7, dtype=np.int64)
    with context(inst, method=2) as tr:
        assert tr.n_rhs == nrhs
        r = tr.column_contributions(np.full(len(pos), 0.42), np.zeros(len(pos), np.int32), pos)
    assert np.all(r["status"] == 0)
    assert np.abs(r["t"] - tj_p[pos]).max() <= 1e-9
    assert np.abs(r["t_minus"] - tj_m[pos]).max() <= 1e-9
    assert np.all(r["iters"] > 0)


def test_free_electron_slab_full_transmission():
    # configuration 1: every column of all 64 energies; checked against the separable
    # closed form (exact for V = 0)
    need_gpu()
    inst = free_electron_slab()
    g = inst.grid
    ref = np.array([separable_transmission(g, inst.gamma_l, inst.gamma_r, e, (0.0, 0.0))
                    for e in inst.energies])
    with context(inst) as tr:
        out = tr.transmission(inst.energies, 1)
    assert np.all(out["status"] == 0)
    assert np.abs(out["T"][:, 0] - ref).max() <= TOL_T


def test_device_arrays_match_host_arrays():
    need_gpu()
    import torch

    inst = small_instance(5, 5, 24, 0.45, 6, 5, kfrac=((0.3, 0.2),), energies=(0.5,), seed=4)
    pos = np.arange(0, 40, 3, dtype=np.int64)
    e = np.full(len(pos), 0.5)
    ik = np.zeros(len(pos), np.int32)
    with context(inst) as tr:
        h = tr.column_contributions(e, ik, pos)
        d = tr.column_contributions(torch.tensor(e, device="cuda"), torch.tensor(ik, device="cuda"),
                                    torch.tensor(pos, device="cuda"))
    assert np.array_equal(h["t"], d["t"].cpu().numpy())
    assert np.array_equal(h["iters"], d["iters"].cpu().numpy())


def test_failures_are_reported_not_raised():
    need_gpu()
    inst = small_instance(5, 4, 24, 0.45, 4, 5, kfrac=((0.2, 0.1),), energies=(0.5,), seed=8)
    with context(inst, maxit=3) as tr:
        r = tr.column_contributions(np.array([0.5, 0.5]), np.array([0, 0], np.int32),
                                    np.array([0, 10**9], np.int64))
    assert r["status"][0] == -4 and np.isnan(r["t"][0])      # maxit reached
    assert r["status"][1] == -1 and np.isnan(r["t"][1])      # column out of range


@pytest.mark.parametrize(
    "nx,ny,nz,order,kfrac",
    [
        (5, 4, 24, 2, ((0.0, 0.0),)),
        (6, 5, 26, 12, ((0.21, -0.34), (-0.21, 0.34))),
        (7, 3, 22, 6, ((0.125, 0.375), (0.0, 0.5))),
    ],
)
def test_mixed_precision_matches_dense_and_fp64(nx, ny, nz, order, kfrac):
    # the mixed form (complex FP32 iteration, FP64 scalars, FP64 residual replacement)
    # must meet the same |dT| <= 1e-6 against the oracle and against the plain FP64 form
    need_gpu()
    inst = small_instance(nx, ny, nz, 0.45, order, 6, v_amp=0.7, kfrac=kfrac,
                          energies=(0.15, 0.55, 1.1), seed=nx + 10 * order)
    ref, _ = _dense_all(inst)
    with context(inst) as tr:
        plain = tr.transmission(inst.energies, len(kfrac))
        tr.set_solver(precision=1)
        tr.stats_reset()
        mixed = tr.transmission(inst.energies, len(kfrac))
        fallbacks = tr.stats()["fallbacks"]
    assert np.all(mixed["status"] == 0), mixed["status"]
    assert fallbacks == 0
    assert np.abs(mixed["T"] - ref).max() <= TOL_T
    assert np.abs(mixed["T"] - plain["T"]).max() <= TOL_T


def test_mixed_precision_free_electron_slab():
    need_gpu()
    inst = free_electron_slab()
    g = inst.grid
    ref = np.array([separable_transmission(g, inst.gamma_l, inst.gamma_r, e, (0.0, 0.0))
                    for e in inst.energies])
    with context(inst, precision=1) as tr:
        out = tr.transmission(inst.energies, 1)
        fallbacks = tr.stats()["fallbacks"]
    assert np.all(out["status"] == 0), np.unique(out["status"], return_counts=True)
    assert np.abs(out["T"][:, 0] - ref).max() <= TOL_T
    assert fallbacks == 0, (fallbacks, out["iters"].max())


def test_device_loop_matches_host_loop():
    # one graph launch with a device-side WHILE loop must compute exactly what the
    # host-polled chunk graphs compute
    need_gpu()
    inst = small_instance(6, 5, 28, 0.45, 10, 6, v_amp=0.8, kfrac=((0.27, -0.16),),
                          energies=(0.42,), seed=21)
    pos = np.arange(0, 120, 7, dtype=np.int64)
    e = np.full(len(pos), 0.42)
    ik = np.zeros(len(pos), np.int32)
    with context(inst, slots=5, chunk=4) as tr:
        dev = tr.column_contributions(e, ik, pos)
        tr.set_solver(host_loop=1)
        host = tr.column_contributions(e, ik, pos)
    assert np.all(dev["status"] == 0)
    assert np.array_equal(dev["t"], host["t"])
    assert np.array_equal(dev["iters"], host["iters"])


def test_autotune_picks_a_valid_shape():
    need_gpu()
    inst = small_instance(20, 20, 64, 0.341, 12, 8, v_amp=0.7, kfrac=((0.3125, -0.4375),),
                          energies=(0.2,), seed=22)
    with context(inst) as tr:
        cfg = tr.autotune(0.2, 0)
        o = tr.solver()
        assert o["slab"] == cfg["slab"] and o["slots"] == cfg["slots"] and o["tile_y"] == cfg["tile_y"]
        assert cfg["slab"] in (16, 32, 64, 128) and cfg["slots"] >= 1
        r = tr.column_contributions(np.full(6, 0.2), np.zeros(6, np.int32), np.arange(6, dtype=np.int64) * 97)
    _, tj = transmission_dense(inst.grid, inst.v, inst.gamma_l, inst.gamma_r, 0.2, inst.kfrac[0])
    assert np.all(r["status"] == 0)
    assert np.abs(r["t"] - tj[np.arange(6) * 97]).max() <= 1e-9
