"""The k-resolved finite-difference Hamiltonian H_k and the system A(E, k).

Test infrastructure only (see the package docstring).

Definition followed (paper Sec. II.A, Eqs. Bloch and H_k; the boundary form with
Bloch phases on the lateral faces is the one the library implements):

* grid points r = (i hx, j hy, l hz), 0 <= i < nx, 0 <= j < ny, 0 <= l < nz, with
  index n = i + nx*(j + ny*l);
* kinetic term -1/2 * (D2_x + D2_y + D2_z), each D2 the order-2N central stencil of
  ``oracle.fd`` divided by h^2 on its axis;
* lateral neighbours wrap periodically; a neighbour i + m maps to (i + m) mod nx and
  picks up the Bloch factor exp(i k_a L_a w) with w = floor((i + m)/nx) (Eq. Bloch:
  phi(x + L_a) = exp(i k_a L_a) phi(x)); the same along y.  Several wraps are allowed
  when the stencil is wider than the cell;
* along z a neighbour outside [0, nz) is dropped (zero Dirichlet ends, the vacuum
  padding of Sec. IV.A);
* H_k = kinetic + diag(V_KS); A(E, k) = E*1 - H_k + i*diag(Gamma_L + Gamma_R), the
  inverse of the retarded Green's function G(E) of Sec. II.A.

k is given as kfrac = (k_a L_a, k_b L_b) / (2 pi).  The matrix is assembled as an
explicit coordinate list, one entry per (point, neighbour) pair, and summed into CSR.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fd import fd_coefficients


def _indices(g):
    n = np.arange(g.n, dtype=np.int64)
    i = n % g.nx
    j = (n // g.nx) % g.ny
    l = n // (g.nx * g.ny)
    return n, i, j, l


def hamiltonian(g, v, kfrac) -> sp.csr_matrix:
    """H_k as a complex128 CSR matrix of size g.n x g.n."""
    c = fd_coefficients(g.order)
    r = g.order // 2
    ka, kb = float(kfrac[0]), float(kfrac[1])
    n, i, j, l = _indices(g)
    rows, cols, vals = [], [], []
    for m in range(-r, r + 1):
        cm = c[abs(m)]
        # x axis, periodic with Bloch phase
        ii = i + m
        w = np.floor_divide(ii, g.nx)
        ii = ii - w * g.nx
        rows.append(n)
        cols.append(ii + g.nx * (j + g.ny * l))
        vals.append(-0.5 * cm / g.hx**2 * np.exp(2j * np.pi * ka * w))
        # y axis, periodic with Bloch phase
        jj = j + m
        w = np.floor_divide(jj, g.ny)
        jj = jj - w * g.ny
        rows.append(n)
        cols.append(i + g.nx * (jj + g.ny * l))
        vals.append(-0.5 * cm / g.hy**2 * np.exp(2j * np.pi * kb * w))
        # z axis, open ends
        ll = l + m
        ok = (ll >= 0) & (ll < g.nz)
        rows.append(n[ok])
        cols.append((i + g.nx * (j + g.ny * ll))[ok])
        vals.append(np.full(int(ok.sum()), -0.5 * cm / g.hz**2, dtype=np.complex128))
    rows.append(n)
    cols.append(n)
    vals.append(np.asarray(v, dtype=np.float64).reshape(-1).astype(np.complex128))
    h = sp.coo_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(g.n, g.n)
    )
    return h.tocsr()


def gamma_points(g, gamma_plane) -> np.ndarray:
    """Per-plane profile expanded to every grid point (CAPs are constant in xy)."""
    return np.repeat(np.asarray(gamma_plane, dtype=np.float64), g.nx * g.ny)


def system_matrix(g, v, gamma_l, gamma_r, energy, kfrac) -> sp.csr_matrix:
    """A(E, k) = E*1 - H_k + i*diag(Gamma_L + Gamma_R) in CSR form."""
    h = hamiltonian(g, v, kfrac)
    gam = gamma_points(g, gamma_l) + gamma_points(g, gamma_r)
    d = sp.diags(energy + 1j * gam)
    return (d - h).tocsr()


def inversion(g, kfrac) -> sp.csr_matrix:
    """P_k: the in-plane rotation R_{z,pi} (x, y, z) -> (-x, -y, z) about grid point
    (0, 0) acting on k-Bloch cell vectors (paper Sec. II.C, the C2 symmetry about z).

    (P_k u)(x, y, z) = u(-x, -y, z); a mirrored coordinate -i outside the cell is
    brought back by the Bloch condition u(i - nx) = exp(-i k_a L_a) u(i), so
    (P_k)_{n, m} = exp(-2 pi i (ka [i > 0] + kb [j > 0])) with m the point
    ((nx - i) mod nx, (ny - j) mod ny, l).  P_k is symmetric, and P_{-k} P_k = 1.
    When V(x, y, z) = V(-x, -y, z), A(E, k)^T = P_k A(E, k) P_{-k}.
    """
    ka, kb = float(kfrac[0]), float(kfrac[1])
    n, i, j, l = _indices(g)
    im = np.where(i > 0, g.nx - i, 0)
    jm = np.where(j > 0, g.ny - j, 0)
    m = im + g.nx * (jm + g.ny * l)
    ph = np.exp(-2j * np.pi * (ka * (i > 0) + kb * (j > 0)))
    return sp.csr_matrix((ph, (n, m)), shape=(g.n, g.n))
