"""The stencil and trace kernels on their own, against the CPU oracle.

The operator apply y = A(E, k) x (and A(E, -k) = A(E, k)^T) is compared with the
oracle's CSR matrix times the same seeded complex vectors, for every stencil order,
complex k, cells narrower than the stencil, ragged tiles and several vectors; the
bar is the rounding of a 37-term complex sum in FP64.  The trace reduction is
compared with the oracle's column_contributions.
"""

import numpy as np
import pytest

from tests.gpu_util import context, need_gpu
from workloads import random_complex, small_instance
from oracle.hamiltonian import system_matrix
from oracle.transmission import column_contributions, left_support

pytestmark = pytest.mark.gpu

CASES = [
    # nx, ny, nz, h, order, kfrac
    (8, 8, 20, 0.5, 2, (0.0, 0.0)),
    (7, 5, 23, 0.45, 4, (0.31, -0.17)),
    (20, 20, 40, 0.341, 12, (0.4375, -0.3125)),
    (4, 3, 30, 0.5, 12, (0.23, 0.41)),      # stencil wider than the cell: multi-wrap
    (37, 9, 18, 0.4, 8, (-0.12, 0.5)),      # ragged x tiles (nx > 32)
    (33, 41, 14, 0.38, 10, (0.5, 0.5)),     # ragged in both, real phases
    (1, 1, 40, 0.5, 6, (0.3, 0.1)),         # a single lateral point
]


@pytest.mark.parametrize("nx,ny,nz,h,order,kf", CASES)
@pytest.mark.parametrize("conj", [False, True])
def test_apply_matches_csr(nx, ny, nz, h, order, kf, conj):
    need_gpu()
    inst = small_instance(nx, ny, nz, h, order, max(2, nz // 5), kfrac=(kf,), seed=nx * 100 + order)
    g = inst.grid
    e = 0.37
    x = random_complex((3, g.n), seed=order)
    with context(inst) as tr:
        y = tr.apply(e, 0, x, conj_k=conj)
    kref = (-kf[0], -kf[1]) if conj else kf
    a = system_matrix(g, inst.v, inst.gamma_l, inst.gamma_r, e, kref)
    ref = (a @ x.T).T
    scale = np.abs(ref).max()
    assert np.abs(y - ref).max() <= 1e-13 * scale


def test_apply_transpose_identity():
    # A(E, -k) = A(E, k)^T: u^T A(k) v == (A(-k) u)^T v on the GPU results alone
    need_gpu()
    inst = small_instance(9, 6, 30, 0.42, 12, 6, kfrac=((0.29, -0.41),), seed=3)
    u = random_complex(inst.grid.n, seed=1)
    v = random_complex(inst.grid.n, seed=2)
    with context(inst) as tr:
        av = tr.apply(0.2, 0, v[None])[0]
        au = tr.apply(0.2, 0, u[None], conj_k=True)[0]
    lhs, rhs = u @ av, au @ v
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("nx,ny,nz", [(5, 4, 30), (20, 20, 64)])
def test_trace_matches_oracle(nx, ny, nz):
    need_gpu()
    inst = small_instance(nx, ny, nz, 0.4, 4, 7, seed=5)
    g = inst.grid
    cols_all = left_support(g, inst.gamma_l)
    pos = np.array([0, 3, len(cols_all) - 1, len(cols_all) // 2])
    x = random_complex((len(pos), g.n), seed=11)
    with context(inst) as tr:
        t = tr.trace(x, pos)
    ref = column_contributions(g, inst.gamma_l, inst.gamma_r, cols_all[pos], x.T)
    assert np.allclose(t, ref, rtol=1e-13, atol=0)


def test_trace_out_of_range_column_is_nan():
    need_gpu()
    inst = small_instance(4, 4, 20, 0.5, 2, 4, seed=6)
    with context(inst) as tr:
        t = tr.trace(random_complex((1, inst.grid.n), 1), np.array([10**6]))
    assert np.isnan(t[0])
