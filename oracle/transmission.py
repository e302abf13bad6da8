"""Landauer transmission T(E, k) from the CAP-terminated Green's function.

Test infrastructure only (see the package docstring).

Definition followed (paper Sec. II.A, the transmission formula and the retarded
Green's function below Eq. CAP-Gaussian, with the k-averaging of Sec. II.A):

    G(E) = [E - H_k + i(Gamma_L + Gamma_R)]^-1
    T(E, k) = 4 Tr[Gamma_L G^dagger Gamma_R G]
            = sum_{j : Gamma_L(j) > 0} t_j,
    t_j = 4 Gamma_L(j) * sum_i Gamma_R(i) |G_ij|^2,   G e_j = x_j
    T(E) = sum_k w_k T(E, k).

The paper prints the trace without the factor 4 and with G* = G^dagger; the factor 4
goes with Gamma entering G as i*Gamma (not i*Gamma/2): a long smooth CAP then gives
T -> 1 per open channel, which the tests check.  For k != 0 G^dagger differs from G*,
and the conjugate transpose is the one used.

Three solver tiers compute the columns x_j = G e_j:

* ``transmission_dense``: dense LU of A (LAPACK), every column, exact to rounding;
* ``transmission_splu``: sparse LU (SuperLU) for chosen columns;
* ``transmission_iterative``: plain textbook Krylov in complex128 for chosen columns:
  COCG (van der Vorst & Melissen 1990) when H_k is real (A complex symmetric, the
  case the paper's Sec. II.A notes for k = 0), otherwise BiCG with the transposed
  shadow system, which is COCG on the paper's complex symmetric +-k operator
  (Eq. def-Gk) and also returns the -k columns.  (Plain BiCGStab stagnates on the
  bulk Cu workload at E_F, so it is not used.)

All tiers share ``column_contributions`` for the trace step and are checked against
one another where their sizes overlap.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .hamiltonian import gamma_points, system_matrix


def left_support(g, gamma_l) -> np.ndarray:
    """Grid indices j with Gamma_L(j) > 0, ascending."""
    return np.nonzero(gamma_points(g, gamma_l) > 0)[0].astype(np.int64)


def column_contributions(g, gamma_l, gamma_r, cols, x) -> np.ndarray:
    """t_j = 4 Gamma_L(j) sum_i Gamma_R(i) |x_ij|^2 for solution columns x[:, c]."""
    gl = gamma_points(g, gamma_l)
    gr = gamma_points(g, gamma_r)
    x = np.asarray(x).reshape(g.n, -1)
    return 4.0 * gl[np.asarray(cols)] * (gr[:, None] * np.abs(x) ** 2).sum(axis=0)


def _rhs(g, cols):
    b = np.zeros((g.n, len(cols)), dtype=np.complex128)
    b[np.asarray(cols), np.arange(len(cols))] = 1.0
    return b


def solve_dense(g, v, gamma_l, gamma_r, energy, kfrac, cols) -> np.ndarray:
    """x_j = A^-1 e_j for the given columns by dense LU (returns n x ncols)."""
    a = system_matrix(g, v, gamma_l, gamma_r, energy, kfrac).toarray()
    lu = sla.lu_factor(a, check_finite=False)
    return sla.lu_solve(lu, _rhs(g, cols), check_finite=False)


def transmission_dense(g, v, gamma_l, gamma_r, energy, kfrac, cols=None):
    """(T, t) with every left-CAP column (or the given subset) solved by dense LU."""
    if cols is None:
        cols = left_support(g, gamma_l)
    x = solve_dense(g, v, gamma_l, gamma_r, energy, kfrac, cols)
    t = column_contributions(g, gamma_l, gamma_r, cols, x)
    return float(t.sum()), t


def transmission_splu(g, v, gamma_l, gamma_r, energy, kfrac, cols):
    """(sum t, t) for the given columns by sparse LU."""
    a = system_matrix(g, v, gamma_l, gamma_r, energy, kfrac).tocsc()
    lu = spla.splu(a)
    x = lu.solve(_rhs(g, cols))
    t = column_contributions(g, gamma_l, gamma_r, cols, x)
    return float(t.sum()), t


def cocg(a, b, tol, maxit):
    """Conjugate orthogonal conjugate gradient for complex symmetric A.

    The CG recurrences with the bilinear form u^T v in place of u^H v.  Columns of
    ``b`` are solved independently; a column stops once ||r||_2 <= tol ||b||_2.
    Returns (x, iterations per column; negative where maxit was reached).
    """
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rho = np.einsum("ij,ij->j", r, r)
    nb = np.linalg.norm(b, axis=0)
    its = np.full(b.shape[1], -maxit)
    live = np.ones(b.shape[1], bool)
    for it in range(1, maxit + 1):
        q = a @ p[:, live]
        sigma = np.einsum("ij,ij->j", p[:, live], q)
        alpha = rho[live] / sigma
        x[:, live] += alpha * p[:, live]
        r[:, live] -= alpha * q
        rn = np.linalg.norm(r[:, live], axis=0)
        done = rn <= tol * nb[live]
        idx = np.nonzero(live)[0]
        its[idx[done]] = it
        live[idx[done]] = False
        if not live.any():
            break
        rho_new = np.einsum("ij,ij->j", r[:, live], r[:, live])
        beta = rho_new / rho[live]
        p[:, live] = r[:, live] + beta * p[:, live]
        rho[live] = rho_new
    return x, its


def bicg_transpose(a, b, tol, maxit, mark_tol=None):
    """BiCG whose shadow system is the transpose: A x = b and A^T y = b together.

    Since A(E, k)^T = A(E, -k) (H_{-k} = H_k^*, Sec. II.B), the shadow solution is
    G(E, -k) b: one run yields the columns of both +k and -k.  Stacking x and y gives
    the conjugate-orthogonal CG of the complex symmetric operator of Eq. def-Gk (the
    +-k pair), with the bilinear forms y^T x.  Textbook BiCG (Fletcher 1976) with
    r_hat_0 = r_0 = b, per column; a column stops once both residual norms are at
    most tol ||b||_2.  Returns (x, y, iterations; negative where maxit was reached).
    With ``mark_tol`` set, also returns the first iteration at which both residuals
    were at most mark_tol ||b||_2 (a looser tolerance reached on the way).
    """
    at = a.T.tocsr()
    x = np.zeros_like(b)
    y = np.zeros_like(b)
    r = b.copy()
    rs = b.copy()
    p = r.copy()
    ps = rs.copy()
    rho = np.einsum("ij,ij->j", rs, r)
    nb = np.linalg.norm(b, axis=0)
    its = np.full(b.shape[1], -maxit)
    marks = np.full(b.shape[1], -maxit)
    live = np.ones(b.shape[1], bool)
    for it in range(1, maxit + 1):
        L = live
        q = a @ p[:, L]
        qs = at @ ps[:, L]
        alpha = rho[L] / np.einsum("ij,ij->j", ps[:, L], q)
        x[:, L] += alpha * p[:, L]
        y[:, L] += alpha * ps[:, L]
        r[:, L] -= alpha * q
        rs[:, L] -= alpha * qs
        rn = np.maximum(np.linalg.norm(r[:, L], axis=0), np.linalg.norm(rs[:, L], axis=0))
        done = rn <= tol * nb[L]
        idx = np.nonzero(L)[0]
        if mark_tol is not None:
            hit = (rn <= mark_tol * nb[L]) & (marks[idx] < 0)
            marks[idx[hit]] = it
        its[idx[done]] = it
        live = L.copy()
        live[idx[done]] = False
        if not live.any():
            break
        rho_new = np.einsum("ij,ij->j", rs[:, live], r[:, live])
        beta = rho_new / rho[live]
        p[:, live] = r[:, live] + beta * p[:, live]
        ps[:, live] = rs[:, live] + beta * ps[:, live]
        rho[live] = rho_new
    if mark_tol is not None:
        return x, y, its, marks
    return x, y, its


def cocg_psym(a, pk, b, tol, maxit):
    """COCG for a P-symmetric A (paper Sec. II.C): A^T P = P A with P symmetric makes
    P A complex symmetric, so CG runs with the bilinear form [u, v] = u^T P v.

    This is BiCG whose shadow residual is P r (A^T P r = P A r keeps it so), with one
    product with A per iteration.  Columns of ``b`` are solved independently; a column
    stops once ||r||_2 <= tol ||b||_2 (||P r|| = ||r|| for the unitary P_k of
    ``oracle.hamiltonian.inversion``).  Returns (x, iterations; negative where maxit
    was reached).
    """
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rho = np.einsum("ij,ij->j", pk @ r, r)
    nb = np.linalg.norm(b, axis=0)
    its = np.full(b.shape[1], -maxit)
    live = np.ones(b.shape[1], bool)
    for it in range(1, maxit + 1):
        L = live
        q = a @ p[:, L]
        alpha = rho[L] / np.einsum("ij,ij->j", pk @ p[:, L], q)
        x[:, L] += alpha * p[:, L]
        r[:, L] -= alpha * q
        rn = np.linalg.norm(r[:, L], axis=0)
        done = rn <= tol * nb[L]
        idx = np.nonzero(L)[0]
        its[idx[done]] = it
        live = L.copy()
        live[idx[done]] = False
        if not live.any():
            break
        rho_new = np.einsum("ij,ij->j", pk @ r[:, live], r[:, live])
        beta = rho_new / rho[live]
        p[:, live] = r[:, live] + beta * p[:, live]
        rho[live] = rho_new
    return x, its


def is_real_phase(kfrac) -> bool:
    """True when exp(2 pi i kappa) is real on both axes (kappa in {0, 1/2} mod 1):
    then H_k is real symmetric and A is complex symmetric."""
    return all(abs((2 * float(kf)) - round(2 * float(kf))) < 1e-15 for kf in kfrac)


def solve_iterative(g, v, gamma_l, gamma_r, energy, kfrac, cols, tol=1e-12, maxit=200000):
    """x_j for the given columns by COCG (real H_k) or transpose BiCG (complex H_k)."""
    a = system_matrix(g, v, gamma_l, gamma_r, energy, kfrac)
    b = _rhs(g, cols)
    if is_real_phase(kfrac):
        return cocg(a, b, tol, maxit)
    x, _, its = bicg_transpose(a, b, tol, maxit)
    return x, its


def transmission_iterative(g, v, gamma_l, gamma_r, energy, kfrac, cols, tol=1e-12, maxit=200000):
    """(sum t, t, iterations) for the given columns by the plain iterative tier."""
    x, its = solve_iterative(g, v, gamma_l, gamma_r, energy, kfrac, cols, tol, maxit)
    t = column_contributions(g, gamma_l, gamma_r, cols, x)
    return float(t.sum()), t, its


def k_average(t_ek, weights) -> np.ndarray:
    """T(E) = sum_k w_k T(E, k) for an (n_E, n_k) array (Sec. II.A)."""
    return np.asarray(t_ek) @ np.asarray(weights)
