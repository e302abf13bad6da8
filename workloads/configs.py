"""Synthetic workloads standing in for the paper's PARSEC Cu/Rh systems.

The paper's own inputs (Troullier-Martins pseudopotentials, self-consistent PARSEC
potentials, VASP bands) are not available, so every workload here is a seeded,
synthetic stand-in with the shapes and structure of the paper's systems:

* bulk fcc Cu and Rh along [001] with lateral periodic cells (paper Sec. IV.A, V.A),
* a periodic Rh point contact whose electrodes narrow to a neck (Sec. V.B),
* absorbing boundary ramps at both transport ends (Sec. II.A; the paper's Gaussian
  form, Eq. CAP-Gaussian, is also provided),
* Monkhorst-Pack lateral k-meshes (Sec. IV.A uses 11x11, Sec. V.B 3x3).

Units are Hartree and bohr.  Arrays use the grid's natural order: the potential has
shape (nz, ny, nx), so a C-order flatten gives the point index n = i + nx*(j + ny*l).
Seeds follow ``seed = 1000*config + instance``.
"""

from __future__ import annotations

from dataclasses import dataclass, field
import dataclasses
import math

import numpy as np


def config_seed(config: int, instance: int = 0) -> int:
    """Seed of one instance of a numbered workload family."""
    return 1000 * int(config) + int(instance)


@dataclass(frozen=True)
class Grid:
    """Uniform real-space grid, lateral (x, y) periodic, z open (transport axis)."""

    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float
    order: int  # finite-difference order of the Laplacian: 2, 4, ..., 12

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nxy(self) -> int:
        return self.nx * self.ny

    @property
    def lx(self) -> float:
        return self.nx * self.hx

    @property
    def ly(self) -> float:
        return self.ny * self.hy

    @property
    def lz(self) -> float:
        return self.nz * self.hz


@dataclass
class Instance:
    """One transport problem: grid, potential, CAPs, k-mesh and energies."""

    name: str
    grid: Grid
    v: np.ndarray  # (nz, ny, nx) float64, Hartree
    gamma_l: np.ndarray  # (nz,) float64, Hartree, left absorbing profile
    gamma_r: np.ndarray  # (nz,) float64, Hartree, right absorbing profile
    kfrac: np.ndarray  # (nk, 2) float64, (k_a L_a, k_b L_b) / 2 pi
    kweights: np.ndarray  # (nk,) float64, sums to 1
    energies: np.ndarray  # (ne,) float64, Hartree
    fermi: float
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def n_rhs(self) -> int:
        """Number of left-CAP grid points (one Krylov column each)."""
        return int(np.count_nonzero(self.gamma_l > 0)) * self.grid.nxy


# ----------------------------------------------------------------------------------
# building blocks
# ----------------------------------------------------------------------------------


def fcc_sites(a: float, ncx: int, ncy: int, lz: float) -> np.ndarray:
    """Sites of an fcc crystal with cubic cell ``a``, [001] along z.

    The lateral cell holds ncx x ncy conventional cells; sites fill 0 <= z < lz.
    The four-site basis (0,0,0), (1/2,1/2,0), (1/2,0,1/2), (0,1/2,1/2) is placed with
    its origin on grid point 0.  Returns an (n_atoms, 3) array, sorted by z.
    """
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    ncz = int(math.ceil(lz / a)) + 1
    cells = np.array(
        [[cx, cy, cz] for cz in range(ncz) for cy in range(ncy) for cx in range(ncx)],
        dtype=np.float64,
    )
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    sites = sites[(sites[:, 2] >= 0) & (sites[:, 2] < lz - 1e-9)]
    order = np.lexsort((sites[:, 0], sites[:, 1], sites[:, 2]))
    return sites[order]


def gaussian_potential(
    grid: Grid, sites: np.ndarray, v0: float, sigma: float, amps: np.ndarray | None = None
) -> np.ndarray:
    """V(r) = -sum_R v0*amp_R*exp(-|r-R|^2/(2 sigma^2)), lateral periodic images.

    Images are summed over the lateral lattice (Lx, Ly); z has no images (open ends).
    Each Gaussian factorises into x, y and z parts; the image sums are taken per axis.
    Returns (nz, ny, nx) float64.
    """
    g = grid
    if amps is None:
        amps = np.ones(len(sites))
    xs = np.arange(g.nx) * g.hx
    ys = np.arange(g.ny) * g.hy
    zs = np.arange(g.nz) * g.hz
    v = np.zeros((g.nz, g.ny, g.nx))
    s2 = 2.0 * sigma * sigma
    zcut = 8.0 * sigma

    def periodic_profile(coord, centre, length):
        reach = int(math.ceil((8.0 * sigma) / length)) + 1
        acc = np.zeros_like(coord)
        for p in range(-reach, reach + 1):
            d = coord - (centre + p * length)
            acc += np.exp(-(d * d) / s2)
        return acc

    for (x0, y0, z0), amp in zip(sites, amps):
        l0 = max(0, int(math.floor((z0 - zcut) / g.hz)))
        l1 = min(g.nz, int(math.ceil((z0 + zcut) / g.hz)) + 1)
        if l1 <= l0:
            continue
        dz = zs[l0:l1] - z0
        gz = np.exp(-(dz * dz) / s2)
        gx = periodic_profile(xs, x0, g.lx)
        gy = periodic_profile(ys, y0, g.ly)
        v[l0:l1] -= (v0 * amp) * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return v


def quadratic_cap(nz: int, ncap: int, peak: float) -> tuple[np.ndarray, np.ndarray]:
    """Quadratic absorbing ramps over the first and last ``ncap`` planes.

    Gamma_L(l) = peak*((ncap - l)/ncap)^2 for l < ncap, else 0: largest on the outer
    plane l = 0, reaching zero at l = ncap.  Gamma_R is its mirror image in z.
    """
    gl = np.zeros(nz)
    l = np.arange(min(ncap, nz))
    gl[: len(l)] = peak * ((ncap - l) / ncap) ** 2
    gr = gl[::-1].copy()
    return gl, gr


def gaussian_cap(
    nz: int, hz: float, gamma0: float, sigma: float, z_left: float, z_right: float, reach: float
) -> tuple[np.ndarray, np.ndarray]:
    """The paper's Gaussian CAPs (Eq. CAP-Gaussian), as per-plane arrays.

    Gamma_{L,R}(z) = gamma0*exp(-(z - z_{L,R})^2/(2 sigma^2)), kept on the outer side of
    each centre and inwards for ``reach`` bohr, zero beyond (a support of finite size
    keeps the set of left-CAP columns finite).
    """
    z = np.arange(nz) * hz
    gl = gamma0 * np.exp(-((z - z_left) ** 2) / (2 * sigma * sigma))
    gr = gamma0 * np.exp(-((z - z_right) ** 2) / (2 * sigma * sigma))
    gl[z > z_left + reach] = 0.0
    gr[z < z_right - reach] = 0.0
    return gl, gr


def monkhorst_pack(ma: int, mb: int) -> tuple[np.ndarray, np.ndarray]:
    """Monkhorst-Pack lateral mesh in units of the reciprocal cell.

    kappa_r = (2r - m - 1)/(2m), r = 1..m, per axis; uniform weights.  A mesh with an
    even m has no Gamma point and is symmetric under k -> -k.
    """
    ka = (2 * np.arange(1, ma + 1) - ma - 1) / (2.0 * ma)
    kb = (2 * np.arange(1, mb + 1) - mb - 1) / (2.0 * mb)
    kk = np.array([[a, b] for b in kb for a in ka], dtype=np.float64)
    w = np.full(len(kk), 1.0 / len(kk))
    return kk, w


def sommerfeld_fermi(v: np.ndarray, a: float, gamma_l: np.ndarray, gamma_r: np.ndarray) -> float:
    """Synthetic Fermi level: mean potential outside the CAP planes plus the
    free-electron Fermi energy of one conduction electron per fcc site,
    n = 4/a^3, E_kin = (3 pi^2 n)^(2/3)/2 (the Sommerfeld model of Sec. IV.A)."""
    inner = (gamma_l == 0) & (gamma_r == 0)
    vbar = float(v[inner].mean()) if inner.any() else float(v.mean())
    n = 4.0 / a**3
    return vbar + 0.5 * (3.0 * math.pi**2 * n) ** (2.0 / 3.0)


def left_cap_columns(grid: Grid, gamma_l: np.ndarray) -> np.ndarray:
    """Grid indices j with Gamma_L(j) > 0, ascending (the right-hand sides e_j)."""
    planes = np.nonzero(np.asarray(gamma_l) > 0)[0]
    base = planes[:, None] * grid.nxy + np.arange(grid.nxy)[None, :]
    return base.reshape(-1).astype(np.int64)


def sample_columns(n_rhs: int, count: int, seed: int) -> np.ndarray:
    """``count`` distinct positions in [0, n_rhs), seeded, ascending."""
    rng = np.random.default_rng(seed)
    count = min(count, n_rhs)
    return np.sort(rng.choice(n_rhs, size=count, replace=False)).astype(np.int64)


def random_complex(shape, seed: int) -> np.ndarray:
    """Seeded complex128 array with real and imaginary parts uniform in [-1, 1)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)


# ----------------------------------------------------------------------------------
# the workload families
# ----------------------------------------------------------------------------------


def free_electron_slab() -> Instance:
    """Free-electron slab: V = 0 on 8x8x64 at h = 0.5 bohr, order 2, 16-plane
    quadratic CAPs of peak 0.5 Ha, k = (0,0), 64 energies in [0.05, 1.0] Ha."""
    g = Grid(8, 8, 64, 0.5, 0.5, 0.5, 2)
    gl, gr = quadratic_cap(g.nz, 16, 0.5)
    return Instance(
        name="free-electron slab 8x8x64 h=0.5 order 2",
        grid=g,
        v=np.zeros((g.nz, g.ny, g.nx)),
        gamma_l=gl,
        gamma_r=gr,
        kfrac=np.zeros((1, 2)),
        kweights=np.ones(1),
        energies=np.linspace(0.05, 1.0, 64),
        fermi=float("nan"),
        seed=config_seed(1),
    )


def _crystal(
    name, a, ncx, ncy, nx, ny, nz, order, v0, sigma, jitter, ncap, peak, mk, ne, window,
    seed, neck_r0=None, vacancy=0.0,
):
    hx = ncx * a / nx
    hy = ncy * a / ny
    hz = hx
    g = Grid(nx, ny, nz, hx, hy, hz, order)
    rng = np.random.default_rng(seed)
    sites = fcc_sites(a, ncx, ncy, g.lz)
    gl, gr = quadratic_cap(nz, ncap, peak)
    meta = {"a": a, "cells": (ncx, ncy), "v0": v0, "sigma": sigma}
    if neck_r0 is not None:
        cx, cy, cz = g.lx / 2, g.ly / 2, g.lz / 2
        rho = np.hypot(sites[:, 0] - cx, sites[:, 1] - cy)
        rho_max = np.sqrt(neck_r0**2 + (sites[:, 2] - cz) ** 2)
        sites = sites[rho <= rho_max]
        meta["neck_r0"] = neck_r0
    if vacancy > 0:
        lplane = np.floor(sites[:, 2] / hz + 0.5).astype(int).clip(0, nz - 1)
        inner = (gl[lplane] == 0) & (gr[lplane] == 0)
        idx = np.nonzero(inner)[0]
        nvac = int(round(vacancy * len(idx)))
        drop = rng.choice(idx, size=nvac, replace=False) if nvac > 0 else np.array([], int)
        keep = np.ones(len(sites), bool)
        keep[drop] = False
        sites = sites[keep]
        meta["vacancies"] = nvac
    amps = 1.0 + rng.uniform(-jitter, jitter, len(sites)) if jitter > 0 else np.ones(len(sites))
    v = gaussian_potential(g, sites, v0, sigma, amps)
    ef = sommerfeld_fermi(v, a, gl, gr)
    kk, w = monkhorst_pack(*mk)
    meta["atoms"] = len(sites)
    return Instance(
        name=name,
        grid=g,
        v=v,
        gamma_l=gl,
        gamma_r=gr,
        kfrac=kk,
        kweights=w,
        energies=np.linspace(ef - window, ef + window, ne),
        fermi=ef,
        seed=seed,
        meta=meta,
    )


def cu_bulk(instance: int = 0) -> Instance:
    """Bulk fcc Cu along [001]: a = 6.82 bohr, 1x1 conventional lateral cell, 24 cells
    long, grid 20x20x480 (h = 0.341), order 12, Gaussian atoms V0 = 1.2 Ha, sigma =
    0.9 bohr with +-2% seeded amplitude jitter, 64-plane quadratic CAPs of peak 0.3 Ha,
    8x8 Monkhorst-Pack mesh, 256 energies in E_F +- 0.3 Ha."""
    return _crystal(
        "bulk fcc Cu [001] 20x20x480 order 12", 6.82, 1, 1, 20, 20, 480, 12, 1.2, 0.9,
        0.02, 64, 0.3, (8, 8), 256, 0.3, config_seed(2, instance),
    )


def inversion_symmetrize(v: np.ndarray) -> np.ndarray:
    """(V + V o R_{z,pi}) / 2 for an (nz, ny, nx) array, R_{z,pi} the in-plane inversion
    (x, y) -> (-x mod nx, -y mod ny) about grid point (0, 0): the result is invariant
    under it to the last bit (a + b = b + a)."""
    vm = np.roll(v[:, ::-1, ::-1], shift=(1, 1), axis=(1, 2))
    return 0.5 * (v + vm)


def cu_bulk_ideal(instance: int = 0) -> Instance:
    """The bulk Cu cell of ``cu_bulk`` without the amplitude jitter: the ideal fcc
    crystal, whose in-plane inversion about an atom (grid point (0, 0)) is a symmetry
    (the C2 rotation about z of Sec. II.C).  V is symmetrised so that the invariance
    holds to the last bit (the lattice sums leave rounding-level asymmetry)."""
    inst = _crystal(
        "ideal bulk fcc Cu [001] 20x20x480 order 12", 6.82, 1, 1, 20, 20, 480, 12, 1.2, 0.9,
        0.0, 64, 0.3, (8, 8), 256, 0.3, config_seed(2, instance),
    )
    return dataclasses.replace(inst, v=inversion_symmetrize(inst.v))


def rh_point_contact(instance: int = 0) -> Instance:
    """Periodic Rh point contact along [001]: a = 7.18 bohr, 3x3 conventional lateral
    cells, grid 60x60x512 (h = 0.359), order 12, V0 = 1.4 Ha, sigma = 0.95 bohr, atoms
    outside a hyperboloid neck of waist 4 bohr at mid-z removed, 1% seeded vacancies
    outside the CAP planes, 64-plane CAPs of peak 0.3 Ha, 4x4 mesh, 512 energies."""
    return _crystal(
        "Rh point contact [001] 60x60x512 order 12", 7.18, 3, 3, 60, 60, 512, 12, 1.4, 0.95,
        0.0, 64, 0.3, (4, 4), 512, 0.3, config_seed(3, instance), neck_r0=4.0, vacancy=0.01,
    )


def uneven_batch(count: int = 96, only=None) -> list[Instance]:
    """Seeded mix of Cu/Rh bulk and point-contact cells of uneven size: lateral cells
    1x1..4x4 conventional cells, 12-40 cells long, h in [0.30, 0.40] bohr, 1-16
    k-points and 64-512 energies per instance.  ``only`` builds just the listed
    instance indices (each instance depends only on its own seed)."""
    out = []
    for i in range(count):
        if only is not None and i not in only:
            continue
        seed = config_seed(4, i)
        rng = np.random.default_rng(seed)
        metal = "Cu" if rng.random() < 0.5 else "Rh"
        a, v0, sigma = (6.82, 1.2, 0.9) if metal == "Cu" else (7.18, 1.4, 0.95)
        contact = bool(rng.random() < 0.5)
        ncx, ncy = int(rng.integers(1, 5)), int(rng.integers(1, 5))
        ncz = int(rng.integers(12, 41))
        h = float(rng.uniform(0.30, 0.40))
        nx, ny = max(4, round(ncx * a / h)), max(4, round(ncy * a / h))
        nz = round(ncz * a / (ncx * a / nx))
        mk = (int(rng.integers(1, 5)), int(rng.integers(1, 5)))
        ne = int(rng.integers(64, 513))
        inst = _crystal(
            f"{metal} {'point contact' if contact else 'bulk'} {ncx}x{ncy}x{ncz} cells",
            a, ncx, ncy, nx, ny, nz, 12, v0, sigma, 0.02 if not contact else 0.0,
            64, 0.3, mk, ne, 0.3, seed,
            neck_r0=4.0 if contact else None, vacancy=0.01 if contact else 0.0,
        )
        out.append(inst)
    return out


def small_instance(
    nx: int, ny: int, nz: int, h: float, order: int, ncap: int, peak: float = 0.4,
    v_amp: float = 0.5, n_blobs: int = 4, kfrac=((0.0, 0.0),), energies=(0.3,), seed: int = 0,
    hy: float | None = None, hz: float | None = None,
) -> Instance:
    """Small seeded problem for parity tests: a few random Gaussian wells (no crystal
    symmetry), quadratic CAPs, the given k-points (uniform weights) and energies."""
    rng = np.random.default_rng(seed)
    g = Grid(nx, ny, nz, h, h if hy is None else hy, h if hz is None else hz, order)
    sites = np.column_stack(
        [rng.uniform(0, g.lx, n_blobs), rng.uniform(0, g.ly, n_blobs), rng.uniform(0, g.lz, n_blobs)]
    )
    amps = rng.uniform(0.5, 1.5, n_blobs)
    v = gaussian_potential(g, sites, v_amp, 0.8, amps) if v_amp != 0 else np.zeros((nz, ny, nx))
    gl, gr = quadratic_cap(nz, ncap, peak)
    kk = np.asarray(kfrac, dtype=np.float64).reshape(-1, 2)
    return Instance(
        name=f"small {nx}x{ny}x{nz} order {order}",
        grid=g,
        v=v,
        gamma_l=gl,
        gamma_r=gr,
        kfrac=kk,
        kweights=np.full(len(kk), 1.0 / len(kk)),
        energies=np.asarray(energies, dtype=np.float64),
        fermi=float("nan"),
        seed=seed,
    )
