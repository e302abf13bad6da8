"""Pins for the oracle's finite-difference coefficients (oracle.fd).

The pins are the defining moment conditions of a central second-derivative stencil,
exact in rational arithmetic: sum_m c_|m| m^(2q) = 2 for q = 1 and 0 for q = 0 and
q = 2..N (the stencil is exact on polynomials up to degree 2N+1), plus the textbook
three-point stencil for order 2.  A wrong sign, factorial or power fails them.
"""

from fractions import Fraction
import numpy as np
import pytest

from oracle.fd import fd_coefficients, fd_coefficients_exact
from oracle.closed_form import band


@pytest.mark.parametrize("order", [2, 4, 6, 8, 10, 12])
def test_moment_conditions_exact(order):
    c = fd_coefficients_exact(order)
    n = order // 2
    for q in range(0, n + 1):
        s = c[0] * (1 if q == 0 else 0) + sum(2 * c[m] * Fraction(m) ** (2 * q) for m in range(1, n + 1))
        assert s == (2 if q == 1 else 0), (order, q, s)


def test_order2_is_textbook():
    assert fd_coefficients(2) == [-2.0, 1.0]


def test_order4_is_textbook():
    # f'' ~ (-f(x+2h) + 16 f(x+h) - 30 f(x) + 16 f(x-h) - f(x-2h)) / (12 h^2)
    assert fd_coefficients_exact(4) == [Fraction(-30, 12), Fraction(16, 12), Fraction(-1, 12)]


@pytest.mark.parametrize("order", [2, 4, 8, 12])
def test_dispersion_matches_continuum(order):
    # eps(theta) = theta^2/(2h^2) + O(theta^(order+2)): the stencil's Fourier symbol
    h = 0.37
    th = np.array([1e-2, 3e-2, 1e-1])
    err = band(th, h, order) - th**2 / (2 * h * h)
    # the truncation term is below theta^(order+2)/h^2 for these orders; rounding of
    # the symbol near theta = 0 adds about 1e-15 * c_0 / h^2
    bound = th ** (order + 2) / h**2 + 1e-12 / h**2
    assert np.all(np.abs(err) <= bound)


def test_band_is_monotone_on_zero_to_pi():
    # one forward mode per lateral channel inside (0, W): the 1D band is monotone
    for order in (2, 4, 6, 8, 10, 12):
        th = np.linspace(0, np.pi, 2001)
        e = band(th, 0.5, order)
        assert np.all(np.diff(e) > 0)
        assert abs(e[0]) < 1e-12
