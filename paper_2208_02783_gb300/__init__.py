"""GB300 library for CAP-terminated Landauer transmission T(E, k).

The compute lives in ``_native/libtransec.so`` (hand-written CUDA for sm_103a,
C ABI in include/transec.h).  ``binding`` mirrors that ABI one function per entry
point; ``Transec`` below is a small convenience wrapper over the same calls.
"""

from __future__ import annotations

import numpy as np

from .binding import (  # noqa: F401
    EBREAKDOWN, ECUDA, EINVAL, ENOCONV, ENOMEM, ESTATE, ETIMEOUT, METHOD_AUTO, METHOD_BICG,
    METHOD_COCG, OK, PREC_DF64, PREC_FP64, PREC_MIXED, SolverOpts, TransecError, load,
    transec_apply, transec_apply_noalloc, transec_autotune, transec_batch_column_contributions,
    transec_column_contributions, transec_create, transec_destroy,
    transec_get_solver, transec_last_error, transec_n_rhs, transec_set_abc,
    transec_set_kmesh, transec_set_potential, transec_set_solver, transec_stats,
    transec_stats_reset, transec_status_string, transec_trace, transec_transmission,
    transec_version, transec_fgmres_columns, transec_shifted_column, transec_shifted_columns,
    transec_sweep_stats, transec_transmission_sketch, transec_unet_create, transec_unet_destroy,
    transec_unet_dims, transec_unet_forward, transec_unet_get_params, transec_unet_n_params,
    transec_unet_set_params, transec_unet_set_path, transec_unet_train_operator, transec_unet_train_step,
    transec_eigen_transmission, transec_unet_zero_output,
)


def batch_column_contributions(contexts, ictx, energies, ik, cols):
    """Sampled columns of several ``Transec`` contexts (cells of uneven size) in one
    solve on the first context's device and options; host arrays in and out."""
    energies = np.ascontiguousarray(energies, np.float64)
    n = energies.size
    t = np.zeros(n)
    tm = np.zeros(n)
    it = np.zeros(n, np.int32)
    st = np.zeros(n, np.int32)
    rc = transec_batch_column_contributions([c.ctx for c in contexts], np.asarray(ictx, np.int32),
                                            energies, np.asarray(ik, np.int32),
                                            np.asarray(cols, np.int64), t, tm, it, st)
    return {"t": t, "t_minus": tm, "iters": it, "status": st, "rc": rc}


class Transec:
    """One library context: a grid, its potential, CAPs, k-mesh and solver options."""

    def __init__(self, nx, ny, nz, hx, hy, hz, order, device=0, stream=None):
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        self.ctx = transec_create(nx, ny, nz, hx, hy, hz, order, device, stream)

    @classmethod
    def from_instance(cls, inst, device=0, stream=None, **solver):
        g = inst.grid
        t = cls(g.nx, g.ny, g.nz, g.hx, g.hy, g.hz, g.order, device, stream)
        t.set_potential(inst.v)
        t.set_abc(inst.gamma_l, inst.gamma_r)
        t.set_kmesh(inst.kfrac, inst.kweights)
        if solver:
            t.set_solver(**solver)
        return t

    def set_potential(self, v):
        if isinstance(v, np.ndarray):
            v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
        transec_set_potential(self.ctx, v)

    def set_abc(self, gamma_l, gamma_r):
        transec_set_abc(self.ctx, gamma_l, gamma_r)

    def set_kmesh(self, kfrac, weights=None):
        transec_set_kmesh(self.ctx, kfrac, weights)

    def set_solver(self, **kw):
        o = transec_get_solver(self.ctx)
        for k, v in kw.items():
            if not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, v)
        transec_set_solver(self.ctx, o)

    def solver(self) -> dict:
        o = transec_get_solver(self.ctx)
        return {f: getattr(o, f) for f, _ in o._fields_}

    def autotune(self, energy, ik=0) -> dict:
        """Pick tile height, slab depth and columns in flight for this operator."""
        return transec_autotune(self.ctx, energy, ik)

    @property
    def n_rhs(self) -> int:
        return transec_n_rhs(self.ctx)

    def transmission(self, energies, nk):
        energies = np.ascontiguousarray(energies, dtype=np.float64)
        ne = energies.size
        t = np.zeros((ne, nk))
        ta = np.zeros(ne)
        st = np.zeros((ne, nk), np.int32)
        it = np.zeros((ne, nk), np.int32)
        rc = transec_transmission(self.ctx, energies, t, ta, st, it)
        return {"T": t, "T_avg": ta, "status": st, "iters": it, "rc": rc}

    def column_contributions(self, energies, ik, cols):
        """Host or device arrays in; results come back on the same side."""
        if hasattr(energies, "is_cuda") and energies.is_cuda:
            import torch

            n = energies.numel()
            dev = energies.device
            t = torch.empty(n, dtype=torch.float64, device=dev)
            tm = torch.empty(n, dtype=torch.float64, device=dev)
            it = torch.empty(n, dtype=torch.int32, device=dev)
            st = torch.empty(n, dtype=torch.int32, device=dev)
        else:
            energies = np.ascontiguousarray(energies, np.float64)
            n = energies.size
            t = np.zeros(n)
            tm = np.zeros(n)
            it = np.zeros(n, np.int32)
            st = np.zeros(n, np.int32)
        rc = transec_column_contributions(self.ctx, energies, ik, cols, t, tm, it, st)
        return {"t": t, "t_minus": tm, "iters": it, "status": st, "rc": rc}

    def shifted_column(self, energies, ik, col):
        """One left-CAP column at many energies in one multi-shift Krylov run."""
        t, tm, it, st = transec_shifted_column(self.ctx, energies, ik, col)
        return {"t": t, "t_minus": tm, "iters": it, "status": st}

    def eigen_transmission(self, lam, v_right, w_left, energies):
        """T(E, k) by the paper's eigenbasis trace from a supplied (partial) eigensolution."""
        return transec_eigen_transmission(self.ctx, lam, v_right, w_left, energies)

    def shifted_columns(self, energies, ik, cols):
        """Sampled left-CAP columns, each at every energy of the window, by the
        multi-shift engine: arrays of shape (len(cols), len(energies))."""
        t, tm, it, st = transec_shifted_columns(self.ctx, energies, ik, cols)
        return {"t": t, "t_minus": tm, "iters": it, "status": st}

    def transmission_sketch(self, energies, ik, s_left=16, s_right=32, seed=0):
        """Full-trace T(E, k) and T(E, -k) for the k indices ``ik`` over a window of
        energies from the two-sided sketch: arrays of shape (len(ik), len(energies))."""
        T, tm, rk, st, it, ms = transec_transmission_sketch(self.ctx, energies, ik, s_left, s_right, seed)
        return {"T": T, "T_minus": tm, "rank": rk, "status": st, "iters": it, "miss": ms}

    def sweep_stats(self) -> dict:
        return transec_sweep_stats(self.ctx)

    def apply(self, energy, ik, x, conj_k=False):
        x = np.ascontiguousarray(x, np.complex128)
        y = np.zeros_like(x)
        transec_apply(self.ctx, energy, ik, x, y, conj_k)
        return y

    def trace(self, x, cols):
        x = np.ascontiguousarray(x, np.complex128)
        cols = np.ascontiguousarray(cols, np.int64)
        t = np.zeros(cols.size)
        transec_trace(self.ctx, x, cols, t)
        return t

    def stats(self) -> dict:
        return transec_stats(self.ctx)

    def stats_reset(self):
        transec_stats_reset(self.ctx)

    def close(self):
        if self.ctx:
            transec_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LearnedPreconditioner:
    """The U-Net right preconditioner for one ``Transec`` context's volume: fitted to
    that operator family on the GPU, then used by FGMRES(restart) for sampled columns."""

    def __init__(self, transec: Transec, seed=0, device=0):
        nz, ny, nx = transec.shape
        self.transec = transec
        self.net = transec_unet_create(device, nx, ny, nz, seed)
        transec_unet_zero_output(self.net)

    def train(self, steps, e_lo, e_hi, lr=1e-3, seed=0, source="krylov"):
        """Adam steps on pairs (r = A e, e) from Krylov iterates ("krylov") or random
        fields ("random"); returns the per-step relative losses."""
        src = {"random": 0, "krylov": 1}[source]
        return transec_unet_train_operator(self.transec.ctx, self.net, steps, e_lo, e_hi, lr, seed, src)

    def params(self):
        return transec_unet_get_params(self.net)

    def set_params(self, p):
        transec_unet_set_params(self.net, p)

    def fgmres_columns(self, energies, ik, cols, restart=30, maxit=20000, precondition=True, net_every=2):
        t, it, st, fb = transec_fgmres_columns(self.transec.ctx, self.net if precondition else None,
                                               energies, ik, cols, restart, maxit, net_every)
        return {"t": t, "iters": it, "status": st, "fallback": fb}

    def close(self):
        if self.net:
            transec_unet_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
