"""The two-sided randomized sketch of T(E, k) = 4 ||M||_F^2, M = Gamma_R^1/2 G Gamma_L^1/2
(paper Sec. II.A for T; the estimator is the two-sided low-rank approximation of Tropp,
Yurtsever, Udell & Cevher, SIAM J. Matrix Anal. Appl. 38, 2017).

Test infrastructure only (see the package docstring).

Steps, with the library's conventions written out plainly:

* random draws: the i-th vector of kind 0 (left) or 1 (right) of run group `rep` holds
  unit-modulus phases exp(2 pi i theta) with theta = (h >> 11) 2^-53 and
  h = splitmix64(seed xor splitmix64(e)), e = ((rep 2 + kind) smax + i) np + u for the
  u-th point of the CAP support (support planes ascending, x fastest within a plane;
  np = the larger support).  splitmix64 is the published generator of Steele, Lea &
  Flood (OOPSLA 2014).
* M(k) on the CAP supports from a dense G(E, k); M(-k) = Gamma_R^1/2 G^T Gamma_L^1/2
  (G(E, -k) = G(E, k)^T, Sec. II.B).
* Y = M Omega, W = Psi^T M; Q an orthonormal basis of range(Y) (directions below
  1e-13 of the largest singular value dropped); T = 4 || (Psi^T Q)^+ W ||_F^2.
* missed-energy estimate: 4 ||(1 - P) y_last||^2 with P the projector on the span of
  the other columns of Y.

Dense and small: pinned in tests/test_oracle_sketch.py.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .hamiltonian import gamma_points, system_matrix

_MASK = (1 << 64) - 1


def splitmix64(z: int) -> int:
    """One output of SplitMix64 for state z (Python integers, arithmetic mod 2^64)."""
    z = (z + 0x9E3779B97F4A7C15) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def phases(seed: int, rep: int, kind: int, i: int, smax: int, npts: int, count: int) -> np.ndarray:
    """The first `count` draws of vector i of the given kind and run group."""
    base = ((rep * 2 + kind) * smax + i) * npts
    out = np.empty(count, complex)
    for u in range(count):
        h = splitmix64((seed & _MASK) ^ splitmix64(base + u))
        theta = (h >> 11) * 2.0**-53
        out[u] = np.exp(2j * np.pi * theta)
    return out


def cap_matrices(g, v, gamma_l, gamma_r, energy, kfrac):
    """(M(k), M(-k)) on the right-CAP rows x left-CAP columns, from a dense G(E, k)."""
    a = system_matrix(g, v, gamma_l, gamma_r, energy, kfrac).toarray()
    gmat = sla.inv(a)
    gl = gamma_points(g, gamma_l)
    gr = gamma_points(g, gamma_r)
    li = np.nonzero(gl > 0)[0]
    ri = np.nonzero(gr > 0)[0]
    sl = np.sqrt(gl[li])
    sr = np.sqrt(gr[ri])
    mp = sr[:, None] * gmat[np.ix_(ri, li)] * sl[None, :]
    mm = sr[:, None] * gmat.T[np.ix_(ri, li)] * sl[None, :]
    return mp, mm


def sketch_t(m, omega, psi, drop=1e-13):
    """(T, missed-energy estimate) of the two-sided sketch of M with test matrices
    Omega (left, columns) and Psi (right, columns)."""
    y = m @ omega
    w = psi.T @ m
    u, s, _ = np.linalg.svd(y, full_matrices=False)
    q = u[:, s > drop * s.max()] if s.max() > 0 else u[:, :0]
    x = np.linalg.pinv(psi.T @ q) @ w
    t = 4.0 * np.linalg.norm(x) ** 2
    prev = y[:, :-1]
    if prev.shape[1]:
        up, sp, _ = np.linalg.svd(prev, full_matrices=False)
        qp = up[:, sp > drop * sp.max()]
        rest = y[:, -1] - qp @ (qp.conj().T @ y[:, -1])
    else:
        rest = y[:, -1]
    return t, 4.0 * np.linalg.norm(rest) ** 2


def sketch_transmission(g, v, gamma_l, gamma_r, energy, kfrac, s_left, s_right, seed, rep=0):
    """(T(E, k), T(E, -k), missed-energy estimates) as the library's sketch computes them
    with the same random draws."""
    mp, mm = cap_matrices(g, v, gamma_l, gamma_r, energy, kfrac)
    nr, nl = mp.shape
    smax = max(s_left, s_right)
    npts = max(nr, nl)
    omega = np.stack([phases(seed, rep, 0, i, smax, npts, nl) for i in range(s_left)], axis=1)
    psi = np.stack([phases(seed, rep, 1, i, smax, npts, nr) for i in range(s_right)], axis=1)
    tp, mp_miss = sketch_t(mp, omega, psi)
    tm, mm_miss = sketch_t(mm, omega, psi)
    return tp, tm, max(mp_miss, mm_miss)
