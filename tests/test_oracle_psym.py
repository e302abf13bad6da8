"""Pins of the P-symmetric form (paper Sec. II.C: with the C2 rotation R_{z,pi} about z a
symmetry of V, the -k states follow from the +k ones), on the CPU.

* oracle.hamiltonian.inversion: P_k is symmetric and P_{-k} P_k = 1; for an
  inversion-symmetric potential A(E, k)^T = P_k A(E, k) P_{-k} holds entry by entry,
  also for a stencil wider than the cell (several Bloch wraps); for a potential without
  the symmetry it fails (the identity is not true of every operator).
* oracle.transmission.cocg_psym: its solution agrees with sparse LU at k != 0, and
  P_k x solves the -k system for the mirrored right-hand side.
* workloads.inversion_symmetrize: exactly invariant; the ideal bulk Cu cell passes.
"""

import dataclasses

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.hamiltonian import inversion, system_matrix
from oracle.transmission import cocg_psym, transmission_dense
from workloads import inversion_symmetrize, small_instance

KF = (0.23, -0.37)


def _sym_inst(nx, ny, nz, order, seed=3):
    inst = small_instance(nx, ny, nz, 0.45, order, 6, v_amp=0.7, kfrac=(KF,), energies=(0.3,), seed=seed)
    return dataclasses.replace(inst, v=inversion_symmetrize(inst.v))


def _mirror(v):
    return np.roll(v[:, ::-1, ::-1], shift=(1, 1), axis=(1, 2))


@pytest.mark.parametrize("shape,order", [((6, 5, 14), 4), ((4, 3, 16), 12), ((7, 8, 12), 8)])
def test_inversion_identities(shape, order):
    nx, ny, nz = shape
    inst = _sym_inst(nx, ny, nz, order)
    g = inst.grid
    pk = inversion(g, KF).toarray()
    pm = inversion(g, (-KF[0], -KF[1])).toarray()
    assert np.array_equal(pk, pk.T)
    assert np.abs(pm @ pk - np.eye(g.n)).max() <= 1e-14
    assert np.allclose(np.abs(pk).sum(axis=1), 1.0)  # a phased permutation
    a = system_matrix(g, inst.v, inst.gamma_l, inst.gamma_r, 0.3, KF).toarray()
    scale = np.abs(a).max()
    assert np.abs(a.T - pk @ a @ pm).max() <= 1e-13 * scale
    # the -k operator is the mirrored +k one
    am = system_matrix(g, inst.v, inst.gamma_l, inst.gamma_r, 0.3, (-KF[0], -KF[1])).toarray()
    assert np.abs(am - pk @ a @ pm).max() <= 1e-13 * scale


def test_inversion_identity_fails_without_the_symmetry():
    inst = small_instance(6, 5, 14, 0.45, 4, 6, v_amp=0.7, kfrac=(KF,), energies=(0.3,), seed=3)
    g = inst.grid
    assert np.abs(inst.v - _mirror(inst.v)).max() > 1e-3
    pk = inversion(g, KF).toarray()
    pm = inversion(g, (-KF[0], -KF[1])).toarray()
    a = system_matrix(g, inst.v, inst.gamma_l, inst.gamma_r, 0.3, KF).toarray()
    assert np.abs(a.T - pk @ a @ pm).max() > 1e-3


def test_cocg_psym_solves_and_mirrors():
    inst = _sym_inst(6, 6, 30, 8, seed=9)
    g = inst.grid
    a = system_matrix(g, inst.v, inst.gamma_l, inst.gamma_r, 0.35, KF).tocsc()
    pk = inversion(g, KF).tocsr()
    rng = np.random.default_rng(4)
    b = np.zeros((g.n, 3), complex)
    b[: 6 * g.nxy] = np.exp(2j * np.pi * rng.random((6 * g.nxy, 3)))
    x, its = cocg_psym(a.tocsr(), pk, b, 1e-12, 5000)
    assert np.all(its > 0)
    ref = spla.splu(a).solve(b)
    assert np.abs(x - ref).max() <= 1e-9 * np.abs(ref).max()
    am = system_matrix(g, inst.v, inst.gamma_l, inst.gamma_r, 0.35, (-KF[0], -KF[1])).tocsr()
    res = am @ (pk @ x) - pk @ b
    assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(b)


def test_inversion_symmetric_transmission_is_even_in_k():
    """T(E, k) = T(E, -k) holds for every operator (time reversal); with the symmetry
    the -k columns are also the mirrored +k ones: t_j(-k) = t_{mirror j}(k)."""
    inst = _sym_inst(5, 4, 24, 4, seed=11)
    g = inst.grid
    tp, t_p = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, 0.4, KF)
    tm, t_m = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, 0.4, (-KF[0], -KF[1]))
    assert abs(tp - tm) <= 1e-12 * max(1.0, abs(tp))
    nl = t_p.size // g.nxy
    w = np.arange(g.nxy)
    x, y = w % g.nx, w // g.nx
    wm = np.where(x > 0, g.nx - x, 0) + g.nx * np.where(y > 0, g.ny - y, 0)
    mir = (np.arange(nl)[:, None] * g.nxy + wm[None, :]).reshape(-1)
    assert np.abs(t_m - t_p[mir]).max() <= 1e-12 * max(1.0, np.abs(t_p).max())


def test_symmetrizer_is_exact():
    rng = np.random.default_rng(0)
    for shape in ((3, 5, 4), (2, 6, 7), (1, 1, 1)):
        v = inversion_symmetrize(rng.normal(size=shape))
        assert np.array_equal(v, _mirror(v))


def test_ideal_bulk_cu_is_inversion_symmetric():
    from workloads import cu_bulk_ideal

    inst = cu_bulk_ideal()
    assert np.array_equal(inst.v, _mirror(inst.v))
