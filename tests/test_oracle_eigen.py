"""Pins of the oracle's eigen route (paper Sec. II.A Eqs. transmission-eigenbasis,
Gamma-tilde, G-diag; Sec. II.B), on the CPU.

* With every eigenpair the eigenbasis trace equals the dense-LU trace over every
  left-CAP column (an independent method) at k = 0 and k != 0.
* The left eigenvectors W of B(k) are right eigenvectors of B(-k) (B(k)^T = B(-k):
  the biorthogonal +-k pairing), and at k = 0 (real H_k) W is parallel to V (the
  complex-orthogonal basis of the complex symmetric case).
* Truncation to the eigenpairs nearest the energy converges to the full result.
"""

import numpy as np
import pytest

from oracle.eigen import eigenpairs, nearest, operator_b, transformed_caps, transmission_eigen
from oracle.transmission import transmission_dense
from workloads import small_instance

KS = [(0.0, 0.0), (0.23, -0.37)]


def _inst(kf, seed=4):
    return small_instance(4, 4, 24, 0.45, 4, 6, v_amp=0.7, kfrac=(kf,), energies=(0.3,), seed=seed)


@pytest.mark.parametrize("kf", KS)
def test_full_eigenbasis_trace_equals_dense_lu(kf):
    inst = _inst(kf)
    g = inst.grid
    lam, v, w = eigenpairs(g, inst.v, inst.gamma_l, inst.gamma_r, kf)
    rt, lt = transformed_caps(g, inst.gamma_l, inst.gamma_r, v, w)
    energies = np.array([0.15, 0.3, 0.55, 0.8])
    te = transmission_eigen(lam, rt, lt, energies)
    for e, t in zip(energies, te):
        td, _ = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, kf)
        assert abs(t - td) <= 1e-9 * max(1.0, abs(td)), (e, t, td)


def test_left_eigenvectors_are_minus_k_right_eigenvectors():
    kf = KS[1]
    inst = _inst(kf, seed=5)
    g = inst.grid
    lam, v, w = eigenpairs(g, inst.v, inst.gamma_l, inst.gamma_r, kf)
    bm = operator_b(g, inst.v, inst.gamma_l, inst.gamma_r, (-kf[0], -kf[1]))
    res = np.linalg.norm(bm @ w - w * lam[None, :], axis=0) / np.linalg.norm(w, axis=0)
    assert res.max() <= 1e-9 * np.abs(lam).max()
    assert np.abs(w.T @ v - np.eye(g.n)).max() <= 1e-8


def test_k0_left_and_right_eigenvectors_are_parallel():
    inst = _inst(KS[0], seed=6)
    g = inst.grid
    lam, v, w = eigenpairs(g, inst.v, inst.gamma_l, inst.gamma_r, KS[0])
    # |w_n . conj(v_n)|^2 = |w_n|^2 |v_n|^2 for parallel vectors
    cos = np.abs(np.einsum("in,in->n", w, v.conj())) / (np.linalg.norm(w, axis=0) * np.linalg.norm(v, axis=0))
    assert np.all(cos >= 1 - 1e-9)


def test_truncation_converges_to_the_full_trace():
    kf = KS[1]
    inst = _inst(kf, seed=7)
    g = inst.grid
    lam, v, w = eigenpairs(g, inst.v, inst.gamma_l, inst.gamma_r, kf)
    e = 0.4
    full = transmission_eigen(lam, *transformed_caps(g, inst.gamma_l, inst.gamma_r, v, w), [e])[0]
    errs = []
    for frac in (0.25, 0.5, 0.75, 1.0):
        sel = nearest(lam, e, int(round(frac * g.n)))
        rt, lt = transformed_caps(g, inst.gamma_l, inst.gamma_r, v[:, sel], w[:, sel])
        errs.append(abs(transmission_eigen(lam[sel], rt, lt, [e])[0] - full))
    assert errs[-1] <= 1e-12 * max(1.0, abs(full))
    assert errs[0] > errs[-1] and errs[1] <= errs[0] * 1.0001
