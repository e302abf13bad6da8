"""The seeded synthetic inputs: the recipe the benchmarks and parity tests rely on.

Checks that each configuration has the sizes it is documented with, that its pieces
follow their definitions (fcc sites, Gaussian wells, quadratic CAPs, Monkhorst-Pack
mesh, energy window, Sommerfeld Fermi level), and that every draw is reproducible from
its seed."""

import math

import numpy as np

from workloads import cu_bulk, free_electron_slab, rh_point_contact, uneven_batch
from workloads.configs import fcc_sites, gaussian_potential, monkhorst_pack, quadratic_cap, Grid


def test_bulk_cu_recipe():
    inst = cu_bulk()
    g = inst.grid
    assert (g.nx, g.ny, g.nz, g.order) == (20, 20, 480, 12)
    assert math.isclose(g.hx, 0.341) and math.isclose(g.hz, g.hx)
    assert inst.meta["atoms"] == 96  # 4 sites x 24 conventional cells
    assert inst.n_rhs == 64 * 400 == 25600
    assert np.count_nonzero(inst.gamma_l) == 64 and np.count_nonzero(inst.gamma_r) == 64
    assert math.isclose(inst.gamma_l.max(), 0.3)
    # Fermi level: mean V outside the CAPs + (3 pi^2 n)^(2/3) / 2 with n = 4 / a^3
    inner = (inst.gamma_l == 0) & (inst.gamma_r == 0)
    ef = inst.v[inner].mean() + 0.5 * (3 * math.pi**2 * 4 / 6.82**3) ** (2 / 3)
    assert math.isclose(inst.fermi, ef, rel_tol=1e-12) and abs(inst.fermi - 0.0861) < 5e-4
    assert len(inst.energies) == 256
    assert math.isclose(inst.energies[0], ef - 0.3) and math.isclose(inst.energies[-1], ef + 0.3)
    assert inst.kfrac.shape == (64, 2) and math.isclose(inst.kweights.sum(), 1.0)
    # the potential is reproducible from the seed and lies in [-V0 * 1.02 * images, 0]
    assert np.array_equal(cu_bulk().v, inst.v)
    assert inst.v.max() <= 0.0 and inst.v.min() > -1.2 * 1.02 * 4


def test_rh_point_contact_recipe():
    inst = rh_point_contact()
    g = inst.grid
    assert (g.nx, g.ny, g.nz) == (60, 60, 512) and inst.n_rhs == 64 * 3600
    assert inst.kfrac.shape == (16, 2) and len(inst.energies) == 512
    # every remaining atom lies inside the neck, rho <= sqrt(r0^2 + (z - Lz/2)^2)
    sites = fcc_sites(7.18, 3, 3, g.lz)
    cx, cy, cz = g.lx / 2, g.ly / 2, g.lz / 2
    rho = np.hypot(sites[:, 0] - cx, sites[:, 1] - cy)
    inside = rho <= np.sqrt(16.0 + (sites[:, 2] - cz) ** 2)
    assert inst.meta["atoms"] == int(inside.sum()) - inst.meta["vacancies"]
    assert inst.meta["vacancies"] > 0


def test_pieces_follow_their_definitions():
    # quadratic CAP: peak on the outer plane, zero from plane ncap on, mirrored
    gl, gr = quadratic_cap(20, 5, 0.4)
    assert math.isclose(gl[0], 0.4) and gl[5] == 0.0 and np.all(np.diff(gl[:6]) < 0)
    assert np.array_equal(gr, gl[::-1])
    # Monkhorst-Pack: symmetric under k -> -k for even m, Gamma point for odd m
    kk, w = monkhorst_pack(4, 4)
    assert {tuple(k) for k in kk} == {tuple(-k) for k in kk} and not np.any(np.all(kk == 0, axis=1))
    kk3, _ = monkhorst_pack(3, 3)
    assert np.any(np.all(kk3 == 0, axis=1))
    # fcc sites: 4 per conventional cell, nearest-neighbour distance a / sqrt(2)
    s = fcc_sites(4.0, 1, 1, 8.0)
    assert len(s) == 8
    d = np.linalg.norm(s[:, None, :] - s[None, :, :], axis=2)
    assert math.isclose(d[d > 0].min(), 4.0 / math.sqrt(2))
    # Gaussian well: one atom at a grid point gives -V0 there, symmetric laterally
    g = Grid(8, 8, 16, 0.5, 0.5, 0.5, 2)
    v = gaussian_potential(g, np.array([[2.0, 2.0, 4.0]]), 1.0, 0.6)
    assert math.isclose(v[8, 4, 4], -1.0, rel_tol=1e-6)
    assert math.isclose(v[8, 4, 3], v[8, 4, 5]) and math.isclose(v[7, 4, 4], v[9, 4, 4])


def test_uneven_batch_is_reproducible_per_instance():
    full = uneven_batch(8)
    some = uneven_batch(8, only={3, 6})
    assert len(some) == 2
    assert np.array_equal(some[0].v, full[3].v) and np.array_equal(some[1].v, full[6].v)
    assert all(i.grid.order == 12 for i in full)
    assert len({i.grid.n for i in full}) > 1  # uneven sizes


def test_free_electron_slab():
    inst = free_electron_slab()
    assert not inst.v.any() and inst.grid.n == 8 * 8 * 64 and inst.n_rhs == 16 * 64
