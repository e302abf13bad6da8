"""Batched solves over operators of uneven size (one slot engine, one solve).

Items of several contexts -- cells of different lateral and transport sizes, stencil
wavelengths and k-meshes -- go through transec_batch_column_contributions together;
each item's t_j must match the same column solved on its own context and the CPU
oracle (dense LU), within the per-column bar the full-size tests use.
"""

import numpy as np
import pytest

from tests.gpu_util import library, need_gpu
from workloads import small_instance, uneven_batch
from oracle.transmission import transmission_dense

pytestmark = pytest.mark.gpu

TOL_COL = 1e-6 / 25600


def _contexts(pkg, insts, **solver):
    return [pkg.Transec.from_instance(i, device=0, **solver) for i in insts]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_individual_and_dense(precision):
    need_gpu()
    pkg = library()
    insts = [
        small_instance(6, 5, 26, 0.45, 12, 6, v_amp=0.7, kfrac=((0.21, -0.34), (-0.21, 0.34)),
                       energies=(0.4,), seed=41),
        small_instance(9, 4, 31, 0.4, 12, 7, v_amp=0.5, kfrac=((0.0, 0.0), (0.125, 0.375)),
                       energies=(0.7,), seed=42),
        small_instance(3, 7, 22, 0.5, 12, 5, v_amp=0.9, kfrac=((0.5, 0.0),), energies=(0.25,), seed=43),
    ]
    rng = np.random.default_rng(7)
    ictx, ks, cols, es = [], [], [], []
    for c, inst in enumerate(insts):
        for _ in range(5):
            ictx.append(c)
            ks.append(int(rng.integers(0, len(inst.kfrac))))
            cols.append(int(rng.integers(0, inst.n_rhs)))
            es.append(float(inst.energies[0]))
    ictx, ks, cols, es = map(np.asarray, (ictx, ks, cols, es))
    ctxs = _contexts(pkg, insts, precision=precision)
    try:
        b = pkg.batch_column_contributions(ctxs, ictx, es, ks.astype(np.int32), cols)
        assert np.all(b["status"] == 0), b["status"]
        for c, inst in enumerate(insts):
            sel = ictx == c
            r = ctxs[c].column_contributions(es[sel], ks[sel].astype(np.int32), cols[sel])
            assert np.abs(r["t"] - b["t"][sel]).max() <= TOL_COL
            for u in np.nonzero(sel)[0]:
                g = inst.grid
                _, tj = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, es[u],
                                           inst.kfrac[ks[u]])
                assert abs(tj[cols[u]] - b["t"][u]) <= TOL_COL
    finally:
        for c in ctxs:
            c.close()


def test_batch_rejects_mismatched_order():
    need_gpu()
    pkg = library()
    a = small_instance(4, 4, 20, 0.5, 12, 4, seed=1)
    b = small_instance(4, 4, 20, 0.5, 4, 4, seed=2)
    ctxs = _contexts(pkg, [a, b])
    try:
        with pytest.raises(pkg.TransecError) as ei:
            pkg.batch_column_contributions(ctxs, [0, 1], [0.3, 0.3], [0, 0], [0, 0])
        assert ei.value.status == pkg.EINVAL
    finally:
        for c in ctxs:
            c.close()


def test_uneven_cells_batch_matches_individual():
    # three of the smallest configuration-4 cells (full size), two columns each
    need_gpu()
    pkg = library()
    insts = uneven_batch(96, only={31, 94, 40})  # the three with the fewest grid points
    ictx = np.repeat(np.arange(3), 2)
    ks = np.zeros(6, np.int32)
    es = np.array([insts[c].fermi for c in ictx])
    cols = np.array([0, insts[0].n_rhs // 2, 5, insts[1].n_rhs - 1, 17, insts[2].n_rhs // 3], np.int64)
    ctxs = _contexts(pkg, insts, maxit=60000)
    try:
        b = pkg.batch_column_contributions(ctxs, ictx, es, ks, cols)
        assert np.all(b["status"] == 0), b["status"]
        for c in range(3):
            sel = ictx == c
            r = ctxs[c].column_contributions(es[sel], ks[sel], cols[sel])
            assert np.all(r["status"] == 0)
            assert np.abs(r["t"] - b["t"][sel]).max() <= TOL_COL
            assert np.abs(r["t_minus"] - b["t_minus"][sel]).max() <= TOL_COL
    finally:
        for c in ctxs:
            c.close()
