"""Pins of the oracle's two-sided sketch (oracle/sketch.py), on the CPU.

* splitmix64 against its published first output for state 0;
* with at least rank(M) left vectors the sketch is exact: T = 4 ||M||_F^2, at k and,
  through M(-k) built from G^T (Sec. II.B), at -k;
* with fewer, the truncation shows and the missed-energy estimate flags it;
* the estimate is unbiased: the mean of ||(1 - P) M omega||^2 over unit-modulus omega
  equals ||(1 - P) M||_F^2.
"""

import numpy as np
import pytest

from oracle.sketch import cap_matrices, phases, sketch_transmission, splitmix64
from workloads import small_instance

KF = (0.23, -0.37)


@pytest.fixture(scope="module")
def cell():
    return small_instance(8, 8, 36, 0.4, 4, 8, v_amp=0.2, kfrac=(KF, (-KF[0], -KF[1])), energies=(0.3,), seed=13)


def test_splitmix64_published_value():
    assert splitmix64(0) == 0xE220A8397B1DCDAF
    p = phases(5, 0, 0, 0, 8, 64, 64)
    assert np.allclose(np.abs(p), 1.0) and len(set(np.round(p, 12))) == 64


def test_sketch_exact_at_full_rank(cell):
    g = cell.grid
    e = 1.2  # rank 2 at this energy
    mp, mm = cap_matrices(g, cell.v, cell.gamma_l, cell.gamma_r, e, KF)
    tp, tm, miss = sketch_transmission(g, cell.v, cell.gamma_l, cell.gamma_r, e, KF, 4, 8, 5)
    want = 4 * np.linalg.norm(mp) ** 2
    assert abs(tp - want) <= 1e-10 * want and abs(tm - want) <= 1e-10 * want
    assert abs(4 * np.linalg.norm(mm) ** 2 - want) <= 1e-10 * want  # T(-k) = T(k)
    assert miss <= 1e-9 * want


def test_sketch_truncated_and_flagged(cell):
    g = cell.grid
    e = 2.0  # rank 4 at this energy
    mp, _ = cap_matrices(g, cell.v, cell.gamma_l, cell.gamma_r, e, KF)
    want = 4 * np.linalg.norm(mp) ** 2
    tp, tm, miss = sketch_transmission(g, cell.v, cell.gamma_l, cell.gamma_r, e, KF, 3, 6, 5)
    assert max(abs(tp - want), abs(tm - want)) > 1e-3
    assert miss > 0.1
    tp6, tm6, miss6 = sketch_transmission(g, cell.v, cell.gamma_l, cell.gamma_r, e, KF, 6, 12, 5)
    assert abs(tp6 - want) <= 1e-9 * want and miss6 <= 1e-9 * want


def test_missed_energy_estimate_is_unbiased(cell):
    g = cell.grid
    mp, _ = cap_matrices(g, cell.v, cell.gamma_l, cell.gamma_r, 2.0, KF)
    rng = np.random.default_rng(3)
    nl = mp.shape[1]
    base = mp @ np.exp(2j * np.pi * rng.random((nl, 2)))
    q, _ = np.linalg.qr(base)
    resid = mp - q @ (q.conj().T @ mp)
    want = np.linalg.norm(resid) ** 2
    vals = [np.linalg.norm(resid @ np.exp(2j * np.pi * rng.random(nl))) ** 2 for _ in range(2000)]
    assert abs(np.mean(vals) - want) <= 0.05 * want
