"""Closed forms for a constant potential: separable transmission and mode counting.

Test infrastructure only (see the package docstring).

With V = 0 (any constant) and CAPs constant in xy (paper Sec. II.A: the CAPs are
constant in the xy-plane), A(E, k) separates into lateral plane waves times a 1D
chain along z.  With the Bloch-phase boundary, the lateral eigenvectors are
exp(i theta i)/sqrt(nx) with theta_m = (2 pi m + 2 pi kappa_a)/nx, and the order-2N
stencil gives the lateral band

    eps_a(theta) = -(1/(2 hx^2)) (c_0 + 2 sum_s c_s cos(s theta)),

so that T(E, k) = sum_{m,n} T_1D(E - eps_a(theta_m) - eps_b(theta_n)), where T_1D is
the same CAP trace for the nz-site chain (orthonormality of the lateral modes makes
the double sum over lateral positions collapse to one term per mode).

Mode counting (paper Sec. III, Eq. cond-ballist): in a ballistic conductor T equals
the number of forward-moving modes.  For the discrete free-electron slab a lateral
mode (m, n) carries one forward mode at energy E when E - eps_perp(m, n) lies inside
the open 1D band (0, W_z), W_z = eps_z(pi).  ``open_channels`` counts them.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .fd import fd_coefficients


def band(theta, h, order):
    """eps(theta) = -(1/(2h^2)) (c_0 + 2 sum_s c_s cos(s theta))."""
    c = fd_coefficients(order)
    theta = np.asarray(theta, dtype=np.float64)
    acc = np.full_like(theta, c[0])
    for s in range(1, len(c)):
        acc = acc + 2.0 * c[s] * np.cos(s * theta)
    return -acc / (2.0 * h * h)


def lateral_energies(g, kfrac) -> np.ndarray:
    """eps_perp(m, n) for every lateral mode, flattened."""
    tha = (2 * np.pi * np.arange(g.nx) + 2 * np.pi * kfrac[0]) / g.nx
    thb = (2 * np.pi * np.arange(g.ny) + 2 * np.pi * kfrac[1]) / g.ny
    ea = band(tha, g.hx, g.order)
    eb = band(thb, g.hy, g.order)
    return (ea[:, None] + eb[None, :]).reshape(-1)


def chain_matrix(nz, hz, order, gamma_l, gamma_r, eps):
    """Dense nz x nz matrix eps*1 - H_1D + i(Gamma_L + Gamma_R), H_1D = -D2_z/2 with
    zero Dirichlet ends."""
    c = fd_coefficients(order)
    h1 = np.zeros((nz, nz))
    for s in range(-(len(c) - 1), len(c)):
        h1 += np.diag(np.full(nz - abs(s), -0.5 * c[abs(s)] / hz**2), s)
    return eps * np.eye(nz) - h1 + 1j * np.diag(np.asarray(gamma_l) + np.asarray(gamma_r))


def chain_transmission(nz, hz, order, gamma_l, gamma_r, eps) -> float:
    """T_1D(eps) = 4 sum_{l, l'} Gamma_L(l) Gamma_R(l') |g_{l' l}|^2."""
    a = chain_matrix(nz, hz, order, gamma_l, gamma_r, eps)
    gmat = sla.inv(a)
    gl = np.asarray(gamma_l)
    gr = np.asarray(gamma_r)
    return float(4.0 * np.einsum("l,m,ml->", gl, gr, np.abs(gmat) ** 2))


def separable_transmission(g, gamma_l, gamma_r, energy, kfrac) -> float:
    """T(E, k) for V = 0 as a sum of 1D chain transmissions over lateral modes."""
    eps = energy - lateral_energies(g, kfrac)
    return float(
        sum(chain_transmission(g.nz, g.hz, g.order, gamma_l, gamma_r, e) for e in eps)
    )


def open_channels(g, energy, kfrac) -> int:
    """Number of lateral modes with 0 < E - eps_perp < W_z (one forward mode each)."""
    wz = float(band(np.pi, g.hz, g.order))
    e = energy - lateral_energies(g, kfrac)
    return int(np.count_nonzero((e > 0) & (e < wz)))
