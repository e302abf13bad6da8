"""Pins for the oracle's Hamiltonian H_k and system matrix (oracle.hamiltonian).

Fixed by the paper (Sec. II.A): H_k is Hermitian, H_{-k} = H_k^* in the real-space
basis, and H_k depends on k only through the Bloch factor exp(i k L) (so kappa and
kappa + 1 give the same matrix); at k = 0 (and any kappa in {0, 1/2}) H_k is real
symmetric.  Fixed by mathematics: the coordinate-list assembly must equal an
independent spectral construction of the same operator, in which each lateral
second derivative is built from its Bloch plane waves exp(i theta_m i)/sqrt(n),
theta_m = 2 pi (m + kappa)/n, and its Fourier symbol.  That construction shares no
index or phase arithmetic with the assembly, so a wrong wrap count, phase sign or
neighbour index fails it.
"""

import numpy as np
import pytest

from workloads import Grid, random_complex
from oracle.hamiltonian import hamiltonian, system_matrix
from oracle.closed_form import band
from oracle.fd import fd_coefficients


def _spectral_second_derivative(n, h, order, kappa):
    th = 2 * np.pi * (np.arange(n) + kappa) / n
    f = np.exp(1j * np.outer(np.arange(n), th)) / np.sqrt(n)
    lam = -2.0 * band(th, h, order)  # symbol of D2 is -2 * eps(theta)
    return f @ np.diag(lam) @ f.conj().T


def _dirichlet_second_derivative(n, h, order):
    c = fd_coefficients(order)
    d = np.zeros((n, n))
    for s in range(-(len(c) - 1), len(c)):
        d += np.diag(np.full(n - abs(s), c[abs(s)] / h**2), s)
    return d


def _spectral_hamiltonian(g, v, kfrac):
    dx = _spectral_second_derivative(g.nx, g.hx, g.order, kfrac[0])
    dy = _spectral_second_derivative(g.ny, g.hy, g.order, kfrac[1])
    dz = _dirichlet_second_derivative(g.nz, g.hz, g.order)
    ix, iy, iz = np.eye(g.nx), np.eye(g.ny), np.eye(g.nz)
    lap = np.kron(iz, np.kron(iy, dx)) + np.kron(iz, np.kron(dy, ix)) + np.kron(dz, np.kron(iy, ix))
    return -0.5 * lap + np.diag(np.asarray(v).reshape(-1))


CASES = [
    (Grid(5, 4, 9, 0.5, 0.45, 0.4, 2), (0.23, -0.41)),
    (Grid(6, 7, 14, 0.4, 0.4, 0.35, 8), (-0.37, 0.11)),
    (Grid(4, 3, 15, 0.5, 0.5, 0.5, 12), (0.3, 0.45)),  # stencil wider than the cell
    (Grid(9, 5, 13, 0.3, 0.33, 0.36, 6), (0.5, 0.0)),
]


@pytest.mark.parametrize("g,kf", CASES)
def test_assembly_matches_spectral_construction(g, kf):
    v = np.random.default_rng(1).uniform(-1, 0, (g.nz, g.ny, g.nx))
    h = hamiltonian(g, v, kf).toarray()
    ref = _spectral_hamiltonian(g, v, kf)
    assert np.abs(h - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("g,kf", CASES)
def test_hermitian_and_time_reversal(g, kf):
    v = np.random.default_rng(2).uniform(-1, 0, (g.nz, g.ny, g.nx))
    h = hamiltonian(g, v, kf).toarray()
    hm = hamiltonian(g, v, (-kf[0], -kf[1])).toarray()
    hp = hamiltonian(g, v, (kf[0] + 1.0, kf[1] - 2.0)).toarray()
    scale = np.abs(h).max()
    assert np.abs(h - h.conj().T).max() <= 1e-14 * scale
    assert np.abs(hm - h.conj()).max() <= 1e-14 * scale
    assert np.abs(hp - h).max() <= 1e-12 * scale


@pytest.mark.parametrize("kf", [(0.0, 0.0), (0.5, 0.0), (0.5, 0.5)])
def test_real_symmetric_at_real_phase(kf):
    g = Grid(6, 5, 10, 0.4, 0.4, 0.4, 10)
    v = np.random.default_rng(3).uniform(-1, 0, (g.nz, g.ny, g.nx))
    h = hamiltonian(g, v, kf).toarray()
    assert np.abs(h.imag).max() <= 1e-15
    assert np.abs(h - h.T).max() <= 1e-13


def test_system_matrix_definition():
    # A = E - H + i(Gamma_L + Gamma_R): check on random vectors, Gamma constant in xy
    g = Grid(4, 5, 12, 0.5, 0.5, 0.5, 4)
    v = np.random.default_rng(4).uniform(-1, 0, (g.nz, g.ny, g.nx))
    gl = np.linspace(0.5, 0, g.nz) * (np.arange(g.nz) < 4)
    gr = gl[::-1].copy()
    kf = (0.17, -0.29)
    a = system_matrix(g, v, gl, gr, 0.37, kf)
    h = hamiltonian(g, v, kf)
    x = random_complex(g.n, 5)
    gam = np.repeat(gl + gr, g.nx * g.ny)
    assert np.allclose(a @ x, 0.37 * x - h @ x + 1j * gam * x, rtol=0, atol=1e-12)
