"""The eigen route's per-energy stage on the GPU (transec_eigen_transmission, paper
Sec. II.A Eqs. transmission-eigenbasis, Gamma-tilde, G-diag), through the C ABI.

The eigenpairs come from the oracle (dense LAPACK eigensolution of H_k - i Gamma with
biorthogonal left vectors); the GPU forms the transformed CAPs and the eigen-sum.
With every eigenpair T must equal the dense-LU trace; with the p eigenpairs nearest an
energy it must equal the oracle's truncated sum with the same pairs (1e-10 relative,
FP64 Gram and sum in another order).
"""

import numpy as np
import pytest

from tests.gpu_util import context, library, need_gpu
from oracle.eigen import eigenpairs, nearest, transformed_caps, transmission_eigen
from oracle.hamiltonian import gamma_points
from oracle.transmission import transmission_dense
from workloads import small_instance

pytestmark = pytest.mark.gpu


def _rows(g, inst, v, w):
    gl = gamma_points(g, inst.gamma_l)
    gr = gamma_points(g, inst.gamma_r)
    return v[gr > 0], w[gl > 0]


@pytest.mark.parametrize("kf", [(0.0, 0.0), (0.23, -0.37)])
def test_eigen_sum_matches_dense_lu_and_truncation(kf):
    need_gpu()
    inst = small_instance(4, 4, 24, 0.45, 4, 6, v_amp=0.7, kfrac=(kf,), energies=(0.3,), seed=4)
    g = inst.grid
    lam, v, w = eigenpairs(g, inst.v, inst.gamma_l, inst.gamma_r, kf)
    energies = np.linspace(0.1, 0.8, 11)
    with context(inst) as tr:
        vr, wl = _rows(g, inst, v, w)
        t_all = tr.eigen_transmission(lam, vr, wl, energies)
        for s, e in enumerate(energies):
            td, _ = transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, kf)
            assert abs(t_all[s] - td) <= 1e-9 * max(1.0, abs(td)), (e, t_all[s], td)
        sel = nearest(lam, 0.45, g.n // 3)
        vr, wl = _rows(g, inst, v[:, sel], w[:, sel])
        t_p = tr.eigen_transmission(lam[sel], vr, wl, energies)
        want = transmission_eigen(lam[sel], *transformed_caps(g, inst.gamma_l, inst.gamma_r, v[:, sel], w[:, sel]),
                                  energies)
        assert np.abs(t_p - want).max() <= 1e-10 * max(1.0, np.abs(want).max())


def test_eigen_argument_checks():
    need_gpu()
    pkg = library()
    inst = small_instance(4, 4, 24, 0.45, 4, 6, kfrac=((0.0, 0.0),), energies=(0.3,), seed=4)
    with context(inst) as tr:
        with pytest.raises(pkg.TransecError) as ei:
            pkg.binding.transec_eigen_transmission(tr.ctx, np.zeros(0, complex), np.zeros((96, 0), complex),
                                                   np.zeros((96, 0), complex), [0.3])
        assert ei.value.status == pkg.EINVAL
