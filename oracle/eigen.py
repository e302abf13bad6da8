"""The paper's eigen route to T(E, k): the trace in the eigenbasis of H_k - i Gamma.

Test infrastructure only (see the package docstring).

Definitions followed (paper Sec. II.A, Eqs. transmission-eigenbasis, Gamma-tilde and
G-diag; Sec. II.B for the left eigenvectors at k != 0):

* B(k) = H_k - i Gamma, Gamma = Gamma_L + Gamma_R, so A(E, k) = E 1 - B(k) and
  G(E) = A^-1.  Right eigenvectors V (B V = V diag(lambda)), left eigenvectors W
  (W^T B = diag(lambda) W^T), normalised biorthogonally: W^T V = 1.  Since
  B(k)^T = B(-k) (H_{-k} = H_k^T), W holds the right eigenvectors of B(-k): the
  biorthogonal +-k pairing of Sec. II.B.  Where H_k is real (k = 0 or the zone
  boundary) B is complex symmetric and W = V, the paper's complex-orthogonal U.
* G(E) = V diag(g) W^T with g_n = 1/(E - lambda_n) (Eq. G-diag).
* With this library's reading of the trace, T = 4 Tr[Gamma_L G^dagger Gamma_R G]:
  T(E) = 4 sum_{m,n} conj(g_m) g_n Rt[m, n] Lt[n, m],
  Rt = V^H Gamma_R V, Lt = W^T Gamma_L conj(W)  (the transformed CAPs, Eq.
  Gamma-tilde, for the biorthogonal basis).
* Truncation (Sec. II.D: a fraction p of the eigenpairs near E_F): the sums run over a
  chosen subset of the eigenpairs; with all of them the result is exact.

Dense and small: for cells of a few thousand points.  Pinned in
tests/test_oracle_eigen.py against dense LU, the +-k relation and k = 0 symmetry.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .hamiltonian import gamma_points, hamiltonian


def operator_b(g, v, gamma_l, gamma_r, kfrac) -> np.ndarray:
    """B(k) = H_k - i (Gamma_L + Gamma_R) as a dense complex matrix."""
    gam = gamma_points(g, gamma_l) + gamma_points(g, gamma_r)
    return hamiltonian(g, v, kfrac).toarray() - 1j * np.diag(gam)


def eigenpairs(g, v, gamma_l, gamma_r, kfrac):
    """(lambda, V, W) of B(k), every eigenpair, with W^T V = 1.

    LAPACK's left eigenvectors y satisfy y^H B = lambda y^H, so W = conj(y); each pair
    is then scaled so that w_n^T v_n = 1.
    """
    b = operator_b(g, v, gamma_l, gamma_r, kfrac)
    lam, yl, vr = sla.eig(b, left=True, right=True)
    w = np.conj(yl)
    w = w / np.einsum("in,in->n", w, vr)[None, :]
    return lam, vr, w


def transformed_caps(g, gamma_l, gamma_r, v_right, w_left):
    """(Rt, Lt): Rt = V^H Gamma_R V, Lt = W^T Gamma_L conj(W) (Eq. Gamma-tilde)."""
    gr = gamma_points(g, gamma_r)
    gl = gamma_points(g, gamma_l)
    rt = v_right.conj().T @ (gr[:, None] * v_right)
    lt = w_left.T @ (gl[:, None] * w_left.conj())
    return rt, lt


def transmission_eigen(lam, rt, lt, energies) -> np.ndarray:
    """T(E) = 4 sum_{m,n} conj(g_m) g_n Rt[m, n] Lt[n, m] for each energy, g_n =
    1/(E - lambda_n), over the eigenpairs the inputs hold (Eq. transmission-eigenbasis
    with G-diag)."""
    out = []
    for e in np.atleast_1d(energies):
        gvec = 1.0 / (e - lam)
        t = 4.0 * np.einsum("m,n,mn,nm->", gvec.conj(), gvec, rt, lt)
        out.append(t.real)
    return np.array(out)


def nearest(lam, center: float, count: int) -> np.ndarray:
    """Indices of the `count` eigenvalues whose real part is nearest `center` (the
    paper's truncation to a fraction of the states near E_F)."""
    return np.argsort(np.abs(lam.real - center))[:count]
