"""Multi-shift transpose BiCG (one Krylov run for a column at many energies) against
the oracle's dense LU, through the C ABI.

Every energy's column contribution t_j (and the shadow system's t_j at -k) must match
dense LU to the solver's 1e-6 bar; the run takes as many seed iterations as its slowest
energy, far fewer than the separate solves together."""

import numpy as np
import pytest

from tests.gpu_util import library, need_gpu
from workloads import small_instance
from oracle.transmission import left_support, transmission_dense

pytestmark = pytest.mark.gpu

TOL_T = 1e-6


def test_shifted_column_matches_dense_lu():
    need_gpu()
    pkg = library()
    kf = (0.21, -0.34)
    inst = small_instance(6, 6, 40, 0.45, 8, 8, v_amp=0.7, kfrac=(kf, (-kf[0], -kf[1])), energies=(0.3,),
                          seed=5)
    g = inst.grid
    energies = np.linspace(0.15, 0.75, 8)
    sup = left_support(g, inst.gamma_l)
    col = 17
    j = sup[col]
    ref_p = np.array([transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, kf, [j])[1][0]
                      for e in energies])
    ref_m = np.array([transmission_dense(g, inst.v, inst.gamma_l, inst.gamma_r, e, (-kf[0], -kf[1]), [j])[1][0]
                      for e in energies])
    with pkg.Transec.from_instance(inst) as tr:
        t, tm, its, st = pkg.binding.transec_shifted_column(tr.ctx, energies, 0, col)
        assert np.all(st == 0), st
        assert np.abs(t - ref_p).max() <= TOL_T, (t, ref_p)
        assert np.abs(tm - ref_m).max() <= TOL_T, (tm, ref_m)
        # separate solves of the same column at each energy, for the iteration count
        sep = tr.column_contributions(energies, np.zeros(energies.size, np.int32), np.full(energies.size, col))
        assert np.all(sep["status"] == 0)
        assert np.abs(sep["t"] - t).max() <= TOL_T
        assert its.max() <= 1.2 * sep["iters"].max()
        assert its.max() < 0.5 * sep["iters"].sum()


def test_shifted_column_argument_checks():
    need_gpu()
    pkg = library()
    inst = small_instance(4, 4, 24, 0.5, 2, 6, energies=(0.3,), seed=1)
    with pkg.Transec.from_instance(inst) as tr:
        with pytest.raises(pkg.TransecError):
            pkg.binding.transec_shifted_column(tr.ctx, [0.3], 0, inst.n_rhs)  # column out of range
        with pytest.raises(pkg.TransecError):
            pkg.binding.transec_shifted_column(tr.ctx, [0.3], 5, 0)  # k index out of range
        with pytest.raises(pkg.TransecError):
            pkg.binding.transec_shifted_column(tr.ctx, [np.nan], 0, 0)
