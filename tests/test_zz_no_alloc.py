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
