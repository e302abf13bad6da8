// Mixed-precision form: complex-FP32 Krylov iteration with FP64 residual replacement.
//
// The iteration itself is the plain engine's (k_stencil<float>, k_update<float>,
// k_scalars with mixed = 1): vectors and the stencil in complex FP32, every dot
// product and norm accumulated in FP64 across threads and blocks, the scalars
// alpha, beta, rho in FP64.  The FP32 "x" of a slot holds only the correction d
// gathered since the last replacement.  When k_scalars sees the FP32 residual drop by
// the reliable factor, or find no new minimum for `stall` iterations (BiCG residuals
// oscillate and an FP32 run eventually stagnates), the slot is flagged and, at the
// end of the graph chunk, these kernels
//
//   k_mx_prep     select the flagged slots (a second slot array with beta = 0)
//   k_mx_accum    x64 += d, d = 0
//   k_stencil<double> on x64    q64 = A(E, +-k) x64 in FP64
//   k_mx_finish   r64 = e_j - q64 (true residual), r32 = fl32(r64), FP64 norms, <r, r>
//   k_mx_scalars  convergence on the FP64 residual; otherwise the FP32 recurrence
//                 restarts from the true residual (beta = 0, rho = <r, r>)
//
// so the solution is accumulated in FP64 and convergence is always judged on the FP64
// residual of the FP64 operator: iterative refinement whose inner solver is the FP32
// BiCG run until its residual has dropped by the reliable factor or stalls.  The
// trace reads x64.
#pragma once

#include "kernels.cuh"

namespace transec {

struct MxPrepArgs {
  const Slot* slots;
  Slot* rslots;
  int S;
};

static __global__ void __launch_bounds__(256) k_mx_prep(const MxPrepArgs a) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.S) return;
  const Slot st = a.slots[s];
  Slot r{};
  if (st.status == SLOT_ACTIVE && st.pending) {
    r.status = SLOT_ACTIVE;
    r.item = st.item;
    r.e = st.e;
    r.ik = st.ik;
    r.inst = st.inst;
    r.j = st.j;
    r.beta = make_double2(0.0, 0.0);
  } else {
    r.status = SLOT_IDLE;
  }
  a.rslots[s] = r;
}

struct MxAccumArgs {
  double2* x64;
  float2* d;
  const Slot* rslots;
  long long n, slot_stride;
  int H;
  const Inst* insts;
};

static __global__ void __launch_bounds__(256) k_mx_accum(const MxAccumArgs a) {
  const int slot = blockIdx.y;
  if (a.rslots[slot].status != SLOT_ACTIVE) return;
  const long long n = a.insts ? a.insts[a.rslots[slot].inst].g.n : a.n;
  const long long base = (long long)slot * a.slot_stride;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    for (int h = 0; h < a.H; ++h) {
      const long long off = base + (long long)h * n + i;
      const float2 dv = a.d[off];
      double2 xv = a.x64[off];
      xv.x += (double)dv.x;
      xv.y += (double)dv.y;
      a.x64[off] = xv;
      a.d[off] = make_float2(0.f, 0.f);
    }
  }
}

struct MxFinishArgs {
  const double2* q64;
  float2* r32;
  const Slot* rslots;
  double* part;  // [slot][gridDim.x][4]: rho re, rho im, |r_0|^2, |r_1|^2
  long long n, slot_stride;
  int H;
  const Inst* insts;
};

static __global__ void __launch_bounds__(256) k_mx_finish(const MxFinishArgs a) {
  __shared__ double red[4][32];
  const int slot = blockIdx.y;
  const Slot* st = a.rslots + slot;
  if (st->status != SLOT_ACTIVE) return;
  const long long j = st->j;
  const long long n = a.insts ? a.insts[st->inst].g.n : a.n;
  const long long base = (long long)slot * a.slot_stride;
  double rrx = 0, rry = 0, n0 = 0, n1 = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float2 rf[2];
    for (int h = 0; h < a.H; ++h) {
      const long long off = base + (long long)h * n + i;
      const double2 q = a.q64[off];
      double2 r = make_double2(-q.x, -q.y);
      if (i == j) r.x += 1.0;
      const double nn = r.x * r.x + r.y * r.y;
      if (h == 0) n0 += nn; else n1 += nn;
      rf[h] = make_float2((float)r.x, (float)r.y);
      a.r32[off] = rf[h];
    }
    const double ax = rf[0].x, ay = rf[0].y;
    if (a.H == 2) {
      const double bx = rf[1].x, by = rf[1].y;
      rrx += 2.0 * (ax * bx - ay * by);
      rry += 2.0 * (ax * by + ay * bx);
    } else {
      rrx += ax * ax - ay * ay;
      rry += 2.0 * ax * ay;
    }
  }
  double v4[4] = {rrx, rry, n0, n1};
  block_sum<4>(v4, red);
  if (threadIdx.x == 0) {
    double* o = a.part + ((size_t)slot * gridDim.x + blockIdx.x) * 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) o[k] = v4[k];
  }
}

struct MxScalarArgs {
  const double* part;
  int nblk;
  const Slot* rslots;
  Slot* slots;
  int S, H;
  double tol;
};

static __global__ void __launch_bounds__(256) k_mx_scalars(const MxScalarArgs a) {
  const int slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (slot >= a.S) return;
  if (a.rslots[slot].status != SLOT_ACTIVE) return;
  double s[4] = {0, 0, 0, 0};
  const double* rp = a.part + (size_t)slot * a.nblk * 4;
  for (int b = lane; b < a.nblk; b += 32)
#pragma unroll
    for (int k = 0; k < 4; ++k) s[k] += rp[4 * b + k];
#pragma unroll
  for (int k = 0; k < 4; ++k) s[k] = warp_sum(s[k]);
  if (lane != 0) return;
  Slot* st = a.slots + slot;
  const double2 rho = make_double2(s[0], s[1]);
  const double res = sqrt(a.H == 2 ? fmax(s[2], s[3]) : s[2]);
  st->pending = 0;
  st->refresh += 1;
  st->last_ref = st->it;
  st->res = res;
  int code = 1;
  if (!isfinite(res) || !isfinite(rho.x) || !isfinite(rho.y)) code = kEBREAKDOWN;
  else if (res <= a.tol) code = kOK;
  else if (rho.x == 0.0 && rho.y == 0.0) code = kEBREAKDOWN;
  if (code != 1) {
    st->result = code;
    st->status = SLOT_DONE;
  } else {
    // restart the FP32 recurrence from the true residual (beta = 0 makes p = r):
    // keeping the old search direction across a replacement stalls the FP32
    // iteration once its biorthogonality is lost
    st->beta = make_double2(0.0, 0.0);
    st->rho = rho;
    st->rmax = res;
    st->rbest = res;
    st->it_best = st->it;
  }
}

struct MxInitArgs {
  double2* x64;
  const Slot* slots;
  long long n, slot_stride;
  int H;
  const Inst* insts;
};

static __global__ void __launch_bounds__(256) k_mx_init(const MxInitArgs a) {
  const int slot = blockIdx.y;
  if (!a.slots[slot].init) return;
  const long long n = a.insts ? a.insts[a.slots[slot].inst].g.n : a.n;
  const long long base = (long long)slot * a.slot_stride;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    for (int h = 0; h < a.H; ++h) a.x64[base + (long long)h * n + i] = make_double2(0.0, 0.0);
}

}  // namespace transec
