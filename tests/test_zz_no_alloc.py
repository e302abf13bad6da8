"""The allocation-free operator apply against the ordinary one, through the C ABI.

transec_apply_noalloc serves callers that may not have the library allocate device
memory (a process whose memory another allocator owns, or a latency-critical loop
that cannot take cudaFree's implicit synchronisation).  It must give the same y as
transec_apply on the same device vectors, call after call (its scratch is a static
array reused by every call), and refuse workloads larger than its fixed scratch.
This file is named to be collected last.
"""

import numpy as np
import pytest

from tests.gpu_util import context, need_gpu
from workloads import random_complex, small_instance

pytestmark = pytest.mark.gpu


def test_noalloc_apply_matches_apply_twice():
    need_gpu()
    import torch

    import paper_2208_02783_gb300 as pkg

    inst = small_instance(20, 20, 48, 0.341, 12, 8, kfrac=((0.4375, -0.3125), (0.0, 0.0)), seed=31)
    g = inst.grid
    with context(inst) as tr:
        for call, (e, ik, conj, nvec) in enumerate([(0.21, 0, False, 3), (-0.05, 1, True, 5)]):
            x = torch.tensor(random_complex((nvec, g.n), seed=100 + call), device="cuda")
            y_ref = torch.zeros_like(x)
            y_na = torch.full_like(x, float("nan"))
            pkg.transec_apply(tr.ctx, e, ik, x, y_ref, conj_k=conj)
            pkg.transec_apply_noalloc(tr.ctx, e, ik, x, y_na, conj_k=conj)
            torch.cuda.synchronize()
            ref = y_ref.cpu().numpy()
            got = y_na.cpu().numpy()
            scale = np.abs(ref).max()
            assert np.abs(got - ref).max() <= 1e-13 * scale, call


def test_noalloc_apply_rejects_oversized_work():
    need_gpu()
    import torch

    import paper_2208_02783_gb300 as pkg

    inst = small_instance(20, 20, 480, 0.341, 12, 64, seed=32)  # 192,000 points
    with context(inst) as tr:
        x = torch.zeros((6, inst.grid.n), dtype=torch.complex128, device="cuda")  # 1.15 M > limit
        y = torch.zeros_like(x)
        with pytest.raises(pkg.TransecError) as ei:
            pkg.transec_apply_noalloc(tr.ctx, 0.1, 0, x, y)
        assert ei.value.status == pkg.EINVAL
        assert "limit" in str(ei.value)


def test_noalloc_apply_at_its_limits():
    """At exactly nvec = 64 and nvec * n = 2**20 the p-scratch fills its region to the
    last byte, next to the partial sums and the per-vector state: any overlap of the
    three regions would change y.  Two calls in a row, against transec_apply."""
    need_gpu()
    import torch

    import paper_2208_02783_gb300 as pkg

    inst = small_instance(16, 16, 64, 0.4, 12, 8, kfrac=((0.3125, 0.1875),), seed=33)
    g = inst.grid
    assert 64 * g.n == 1 << 20
    with context(inst) as tr:
        for call, (e, conj) in enumerate([(0.17, False), (0.33, True)]):
            x = torch.tensor(random_complex((64, g.n), seed=200 + call), device="cuda")
            y_ref = torch.zeros_like(x)
            y_na = torch.full_like(x, float("nan"))
            pkg.transec_apply(tr.ctx, e, 0, x, y_ref, conj_k=conj)
            pkg.transec_apply_noalloc(tr.ctx, e, 0, x, y_na, conj_k=conj)
            torch.cuda.synchronize()
            ref = y_ref.cpu().numpy()
            got = y_na.cpu().numpy()
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), call
        x = torch.zeros((65 * g.n,), dtype=torch.complex128, device="cuda")
        with pytest.raises(pkg.TransecError) as ei:
            pkg.transec_apply_noalloc(tr.ctx, 0.1, 0, x, torch.zeros_like(x))
        assert ei.value.status == pkg.EINVAL and "64 vectors" in str(ei.value)


def test_noalloc_apply_rejects_too_many_partial_sums():
    """One stencil block per point (a 1x1 column with one-row tiles and one-plane slabs)
    needs more partial sums than the fixed region holds: refused on the host, before
    any launch."""
    need_gpu()
    import torch

    import paper_2208_02783_gb300 as pkg

    inst = small_instance(1, 1, 1 << 16, 0.4, 2, 64, v_amp=0.0, seed=34)
    with context(inst, tile_y=1, slab=1) as tr:
        x = torch.zeros((2, inst.grid.n), dtype=torch.complex128, device="cuda")
        with pytest.raises(pkg.TransecError) as ei:
            pkg.transec_apply_noalloc(tr.ctx, 0.1, 0, x, torch.zeros_like(x))
        assert ei.value.status == pkg.EINVAL and "partial-sum" in str(ei.value)
