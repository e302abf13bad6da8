"""Pins for the oracle's transmission (oracle.transmission, oracle.closed_form).

What fixes the answer, independently of the oracle's own trace code:

* separable closed form for V = 0 (sum of 1D chain transmissions over lateral
  Bloch modes), which checks the 3D operator, phases and trace together;
* the long-CAP limit of the 1D chain: a long, smooth absorber reflects nothing, so
  T_1D -> 1 inside the band and -> 0 outside it (the mode counting of Sec. III:
  T equals the number of forward modes).  This fixes the factor 4 and the use of
  G^dagger; a missing 4 gives 1/4, a G^T gives a wrong value at k != 0;
* T_LR = T_RL and T(k) = T(-k) (Sec. II.B/II.C: H_{-k} = H_k^*, the CAPs are
  constant in xy); T(k + 1) = T(k); invariance under a lateral grid shift of V;
  the z mirror with Gamma_L <-> Gamma_R;
* the per-column Ward identity sum_i Gamma_i |x_ji|^2 = -Im x_jj, exact because
  G^-1 - G^-dagger = 2i Gamma;
* transmission eigenvalues (of 4 Gamma_L^1/2 G^dagger Gamma_R G Gamma_L^1/2) lie in
  [0, 1];
* the iterative and sparse-LU tiers agree with dense LU where sizes overlap.
"""

import numpy as np
import pytest
import scipy.linalg as sla

from workloads import Grid, free_electron_slab, quadratic_cap, small_instance
from oracle.hamiltonian import gamma_points, system_matrix
from oracle.transmission import (
    column_contributions,
    left_support,
    transmission_dense,
    transmission_iterative,
    transmission_splu,
    k_average,
)
from oracle.closed_form import (
    chain_transmission,
    lateral_energies,
    open_channels,
    separable_transmission,
)


def _green(g, v, gl, gr, e, kf):
    return sla.inv(system_matrix(g, v, gl, gr, e, kf).toarray())


@pytest.mark.parametrize(
    "g,kf,energies",
    [
        (Grid(5, 4, 30, 0.5, 0.45, 0.5, 2), (0.0, 0.0), (0.1, 0.6, 1.4)),
        (Grid(6, 5, 28, 0.5, 0.55, 0.45, 4), (0.3, -0.2), (0.3, 1.5)),
        (Grid(4, 4, 26, 0.45, 0.45, 0.4, 12), (0.41, 0.13), (0.25, 0.9, 2.0)),
        (Grid(3, 5, 24, 0.5, 0.5, 0.5, 8), (0.5, 0.5), (0.3, 1.5)),
    ],
)
def test_dense_matches_separable_closed_form(g, kf, energies):
    gl, gr = quadratic_cap(g.nz, 7, 0.5)
    v = np.zeros((g.nz, g.ny, g.nx))
    for e in energies:
        t, _ = transmission_dense(g, v, gl, gr, e, kf)
        tc = separable_transmission(g, gl, gr, e, kf)
        assert abs(t - tc) <= 1e-10 * max(1.0, tc), (e, t, tc)


def test_long_cap_limit_counts_one_mode_per_channel():
    hz, order = 0.5, 2
    w = 2.0 / hz**2  # top of the order-2 band
    errs = []
    for ncap in (40, 160, 640):
        nz = 2 * ncap + 60
        gl, gr = quadratic_cap(nz, ncap, 0.5)
        inside = [chain_transmission(nz, hz, order, gl, gr, e) for e in (0.2, 1.0, 3.0, 6.0)]
        outside = [chain_transmission(nz, hz, order, gl, gr, e) for e in (-0.3, w + 0.5)]
        errs.append(max(abs(1 - t) for t in inside))
        assert max(outside) < 1e-8
    assert errs[0] > errs[1] > errs[2] or errs[2] < 1e-12
    assert errs[-1] < 1e-6


def test_long_cap_limit_3d_mode_count():
    # 3D slab with a long absorber: T equals the integer number of open channels
    g = Grid(3, 3, 200, 0.6, 0.6, 0.5, 4)
    gl, gr = quadratic_cap(g.nz, 90, 0.5)
    for kf in ((0.0, 0.0), (0.3, -0.1)):
        for e in (0.2, 1.3, 3.1):
            tc = separable_transmission(g, gl, gr, e, kf)
            eps = e - lateral_energies(g, kf)
            # channels within 0.05 Ha of a band edge converge slowly; skip those energies
            wz = 2.0 * 0.5 / 0.25 * 2
            if np.any(np.abs(eps) < 0.05):
                continue
            assert abs(tc - open_channels(g, e, kf)) < 2e-3, (kf, e, tc)


def test_free_electron_slab_mode_count_within_cap_reflection():
    inst = free_electron_slab()
    g = inst.grid
    e00 = lateral_energies(g, (0.0, 0.0)).min()
    # reflection loss of the open channel, from the 1D chain alone
    refl = max(1 - chain_transmission(g.nz, g.hz, g.order, inst.gamma_l, inst.gamma_r, e - e00)
               for e in inst.energies)
    assert 0.25 < refl < 0.35  # a 16-plane ramp reflects about 30% at 0.05 Ha
    for e in inst.energies:
        tc = separable_transmission(g, inst.gamma_l, inst.gamma_r, e, (0.0, 0.0))
        assert open_channels(g, e, (0.0, 0.0)) == 1
        assert abs(tc - 1) <= refl + 1e-9
    for e in (0.05, 0.5):
        t, tj = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, (0.0, 0.0))
        tc = separable_transmission(g, inst.gamma_l, inst.gamma_r, e, (0.0, 0.0))
        assert abs(t - tc) < 1e-10
        assert np.all(tj >= 0)


def _general():
    return small_instance(5, 4, 26, 0.45, 6, 7, v_amp=0.8, n_blobs=5, seed=11)


def test_lr_equals_rl_and_ward_identity():
    inst = _general()
    g = inst.grid
    kf = (0.27, -0.16)
    gmat = _green(g, inst.v, inst.gamma_l, inst.gamma_r, 0.35, kf)
    glp = gamma_points(g, inst.gamma_l)
    grp = gamma_points(g, inst.gamma_r)
    t_lr = 4 * np.einsum("j,i,ij->", glp, grp, np.abs(gmat) ** 2)
    t_rl = 4 * np.einsum("j,i,ij->", grp, glp, np.abs(gmat) ** 2)
    assert abs(t_lr - t_rl) < 1e-12 * max(1, t_lr)
    gam = glp + grp
    ward = (gam[:, None] * np.abs(gmat) ** 2).sum(axis=0)
    assert np.allclose(ward, -np.diag(gmat).imag, rtol=1e-11, atol=1e-14)


def test_time_reversal_and_periodicity_in_k():
    inst = _general()
    g = inst.grid
    args = (g, inst.v, inst.gamma_l, inst.gamma_r, 0.42)
    t0, _ = transmission_dense(*args, (0.31, 0.07))
    t1, _ = transmission_dense(*args, (-0.31, -0.07))
    t2, _ = transmission_dense(*args, (1.31, -0.93))
    assert abs(t0 - t1) < 1e-11 * max(1, t0)
    assert abs(t0 - t2) < 1e-11 * max(1, t0)


def test_lateral_shift_and_z_mirror():
    inst = _general()
    g = inst.grid
    kf = (0.21, 0.39)
    t0, _ = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, 0.3, kf)
    vs = np.roll(np.roll(inst.v, 2, axis=2), 1, axis=1)
    t1, _ = transmission_dense(g, vs, inst.gamma_l, inst.gamma_r, 0.3, kf)
    vm = inst.v[::-1].copy()
    t2, _ = transmission_dense(g, vm, inst.gamma_r[::-1].copy(), inst.gamma_l[::-1].copy(), 0.3, kf)
    assert abs(t0 - t1) < 1e-11 * max(1, t0)
    assert abs(t0 - t2) < 1e-11 * max(1, t0)


def test_transmission_eigenvalues_in_unit_interval():
    inst = _general()
    g = inst.grid
    gmat = _green(g, inst.v, inst.gamma_l, inst.gamma_r, 0.5, (0.1, -0.3))
    sl = np.sqrt(gamma_points(g, inst.gamma_l))
    sr = np.sqrt(gamma_points(g, inst.gamma_r))
    tmat = 2 * sr[:, None] * gmat * sl[None, :]
    ev = np.linalg.eigvalsh(tmat.conj().T @ tmat)
    assert ev.min() > -1e-12 and ev.max() < 1 + 1e-10
    t, tj = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, 0.5, (0.1, -0.3))
    assert abs(ev.sum() - t) < 1e-10 * max(1, t)
    assert np.all(tj >= 0)


@pytest.mark.parametrize("kf", [(0.0, 0.0), (0.5, 0.0), (0.23, -0.37)])
def test_tiers_agree(kf):
    inst = small_instance(7, 6, 40, 0.45, 8, 10, v_amp=0.6, seed=5)
    g = inst.grid
    args = (g, inst.v, inst.gamma_l, inst.gamma_r, 0.4, kf)
    t, tj = transmission_dense(*args)
    cols = left_support(g, inst.gamma_l)[::17]
    _, ti, its = transmission_iterative(*args, cols)
    _, ts = transmission_splu(*args, cols)
    ref = tj[::17]
    assert np.all(its > 0)
    assert np.abs(ti - ref).max() < 1e-10
    assert np.abs(ts - ref).max() < 1e-12


def test_column_contributions_definition():
    # t_j on a hand-made solution: 4 * Gamma_L(j) * sum_i Gamma_R(i) |x_i|^2
    g = Grid(2, 1, 4, 1.0, 1.0, 1.0, 2)
    gl = np.array([0.5, 0, 0, 0])
    gr = np.array([0, 0, 0, 0.25])
    x = np.zeros((g.n, 1), complex)
    x[6, 0] = 1 + 1j  # plane 3
    x[7, 0] = 2.0
    t = column_contributions(g, gl, gr, [1], x)
    assert t[0] == pytest.approx(4 * 0.5 * 0.25 * (2 + 4))


def test_k_average():
    assert np.allclose(k_average([[1.0, 3.0], [2.0, 2.0]], [0.25, 0.75]), [2.5, 2.0])


@pytest.mark.parametrize(
    "dims,order,kf",
    [
        ((7, 6, 40, 0.45, 8, 10), 8, (0.23, -0.37)),
        ((3, 4, 30, 0.45, 12, 8), 12, (0.31, 0.12)),  # order 12 on a 3x4 cell: several wraps
    ],
)
def test_bicg_shadow_solution_is_the_minus_k_column(dims, order, kf):
    """The transpose BiCG's shadow iterate y solves A(E, k)^T y = e_j, and
    A(E, k)^T = A(E, -k) because H_{-k} = H_k^* with H_k Hermitian (Sec. II.B).  So y
    must be the dense-LU column of G(E, -k) and its trace t_j(-k); the full-size golden
    t_minus values rest on this."""
    from oracle.transmission import bicg_transpose, solve_dense

    nx, ny, nz, h, _, ncap = dims
    inst = small_instance(nx, ny, nz, h, order, ncap, v_amp=0.6, seed=17)
    g = inst.grid
    e = 0.45
    cols = left_support(g, inst.gamma_l)[::23][:6]
    a = system_matrix(g, inst.v, inst.gamma_l, inst.gamma_r, e, kf)
    b = np.zeros((g.n, cols.size), complex)
    b[cols, np.arange(cols.size)] = 1.0
    x, y, its = bicg_transpose(a, b, 1e-12, 20000)
    assert np.all(its > 0)
    mk = (-kf[0], -kf[1])
    xd = solve_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, kf, cols)
    yd = solve_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, mk, cols)
    scale = np.abs(yd).max()
    assert np.abs(x - xd).max() <= 1e-9 * scale
    assert np.abs(y - yd).max() <= 1e-9 * scale
    # y is not the +k column (the check has teeth at k != 0)
    assert np.abs(y - xd).max() > 1e-3 * scale
    ty = column_contributions(g, inst.gamma_l, inst.gamma_r, cols, y)
    _, tref = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, mk, cols)
    assert np.abs(ty - tref).max() <= 1e-10
