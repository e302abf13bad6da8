"""Central finite-difference coefficients of the second derivative.

Test infrastructure only (see the package docstring).

The paper's Hamiltonian is the real-space finite-difference Kohn-Sham operator of
PARSEC/TRANSEC (Sec. I: a real-space grid and a very sparse Hamiltonian).  The
order-2N central stencil for d^2/dx^2 on a uniform grid has the closed form
(Fornberg 1988, the standard result for equispaced central differences)

    c_0 = -2 * sum_{m=1..N} 1/m^2
    c_m = 2 (-1)^(m+1) (N!)^2 / (m^2 (N-m)! (N+m)!),   m = 1..N,

so that f''(x) ~ h^-2 * sum_{m=-N..N} c_|m| f(x + m h).  The values are computed
with exact rational arithmetic and rounded once to float64.
"""

from __future__ import annotations

from fractions import Fraction
from math import factorial


def fd_coefficients_exact(order: int) -> list[Fraction]:
    """[c_0, c_1, ..., c_N] as exact fractions for an order-``order`` stencil."""
    if order < 2 or order % 2 or order > 24:
        raise ValueError(f"order must be even in [2, 24], got {order}")
    n = order // 2
    c0 = Fraction(-2) * sum(Fraction(1, m * m) for m in range(1, n + 1))
    out = [c0]
    fn2 = factorial(n) ** 2
    for m in range(1, n + 1):
        sign = 1 if (m + 1) % 2 == 0 else -1
        out.append(Fraction(2 * sign * fn2, m * m * factorial(n - m) * factorial(n + m)))
    return out


def fd_coefficients(order: int) -> list[float]:
    """[c_0, ..., c_N] rounded to float64."""
    return [float(c) for c in fd_coefficients_exact(order)]
