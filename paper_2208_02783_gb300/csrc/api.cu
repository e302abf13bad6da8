// C ABI of the transmission library (include/transec.h) and the slot-engine driver.
//
// A solve is a queue of work items (E, k, left-CAP column).  The engine keeps S
// "slots" in flight on the GPU; each slot runs its own Krylov recurrence and, once
// converged (or failed), has its column contribution t_j traced, is released and is
// refilled from the queue by a device kernel.  Iterations are issued as a CUDA graph
// of `chunk` iterations (stencil, update, scalars per iteration) followed by the
// trace / assign / init kernels; the host only polls the harvested-item counter
// between graph launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "engine.cuh"
#include "mixed.cuh"

using namespace transec;

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(d);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int fail(transec_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      cudaGetLastError();                                                             \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? TRANSEC_ENOMEM : TRANSEC_ECUDA, \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                \
    }                                                                                 \
  } while (0)

#define CHECK_LAUNCH()                                                                \
  do {                                                                                \
    cudaError_t e_ = cudaGetLastError();                                              \
    if (e_ != cudaSuccess)                                                            \
      return fail(ctx, TRANSEC_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

// Central finite-difference coefficients of d^2/dx^2 of order 2N (the standard
// closed form): c_0 = -2 sum_{m<=N} 1/m^2, c_m = 2 (-1)^(m+1) (N!)^2 /
// (m^2 (N-m)! (N+m)!).  Numerators and denominators are exact 64-bit integers, so
// each coefficient is one correctly rounded division.
void fd_coefficients(int order, double* c) {
  const int N = order / 2;
  long long f[13];
  f[0] = 1;
  for (int i = 1; i <= 12; ++i) f[i] = f[i - 1] * i;
  const long long fn2 = f[N] * f[N];
  long long s = 0;  // sum (N!)^2 / m^2, each term an integer for m <= N
  for (int m = 1; m <= N; ++m) s += fn2 / ((long long)m * m);
  c[0] = -2.0 * (double)s / (double)fn2;
  for (int m = 1; m <= N; ++m) {
    const long long den = (long long)m * m * f[N - m] * f[N + m];
    const double v = (double)(2 * fn2) / (double)den;
    c[m] = (m % 2 == 1) ? v : -v;
  }
}

int severity(int code) {
  switch (code) {
    case TRANSEC_OK: return 0;
    case TRANSEC_ENOCONV: return 1;
    case TRANSEC_EBREAKDOWN: return 2;
    case TRANSEC_ETIMEOUT: return 3;
    default: return 4;
  }
}

void default_opts(transec_solver_opts* o) {
  if (o->tol <= 0) o->tol = 1e-10;
  if (o->maxit <= 0) o->maxit = 100000;
  if (o->chunk <= 0) o->chunk = 16;
  if (o->chunk % 2) o->chunk += 1;  // the p ping-pong must end where it started
  if (o->reliable <= 0 || o->reliable >= 1) o->reliable = 1e-5;
  if (o->mixed_maxit <= 0) o->mixed_maxit = 8000;
  if (o->mixed_decade_its == 0) o->mixed_decade_its = 1000;
  if (o->df_stall_its == 0) o->df_stall_its = 8000;
  if (o->sketch_guard == 0) o->sketch_guard = 1e-7;
}

// Bloch phase exp(2 pi i kappa w) with the argument reduced before the cosine.
double2 bloch(double kappa, int w) {
  const double f = kappa * w - std::nearbyint(kappa * w);
  return make_double2(std::cos(2.0 * M_PI * f), std::sin(2.0 * M_PI * f));
}

bool real_phase(double ka, double kb) {
  auto is_half = [](double k) { double t = 2.0 * k; return std::fabs(t - std::nearbyint(t)) < 1e-15; };
  return is_half(ka) && is_half(kb);
}

int partner_of(const transec_ctx* c, int k) {
  for (int p = 0; p < c->nk; ++p) {
    if (p == k) continue;
    const double da = c->kfrac[2 * p] + c->kfrac[2 * k], db = c->kfrac[2 * p + 1] + c->kfrac[2 * k + 1];
    if (std::fabs(da - std::nearbyint(da)) < 1e-12 && std::fabs(db - std::nearbyint(db)) < 1e-12)
      return p;
  }
  return -1;
}

}  // namespace

// ---------------------------------------------------------------------------------
// launch shape
// ---------------------------------------------------------------------------------

namespace transec {

TileShape choose_tiles(const Geometry& g, int H, int elem_bytes, int max_threads, int tile_y,
                       int slab) {
  TileShape t{};
  const int R = g.R;
  // tile width: the whole row when it fits a warp, else the width in [16, 32] that
  // wastes the fewest padded columns
  if (g.nx <= 32) {
    t.TX = g.nx;
  } else {
    int best = 32;
    long long bestc = 1LL << 60;
    for (int w = 16; w <= 32; ++w) {
      const long long cost = (long long)((g.nx + w - 1) / w) * (w + 2 * R);
      if (cost < bestc) { bestc = cost; best = w; }
    }
    t.TX = best;
  }
  int ylim = std::max(1, max_threads / (t.TX * H));
  ylim = std::min(ylim, g.ny);
  if (tile_y > 0) {
    t.TY = std::min(tile_y, ylim);
  } else {
    int best = ylim;
    long long bestc = 1LL << 60;
    for (int h = 1; h <= ylim; ++h) {
      const long long cost = (long long)((g.ny + h - 1) / h) * (h + 2 * R);
      if (cost < bestc) { bestc = cost; best = h; }
    }
    t.TY = best;
  }
  t.ntx = (g.nx + t.TX - 1) / t.TX;
  t.nty = (g.ny + t.TY - 1) / t.TY;
  t.D = slab > 0 ? slab : (elem_bytes >= 16 ? 32 : 64);
  t.D = std::min(t.D, g.nz);
  t.nslab = (g.nz + t.D - 1) / t.D;
  // the requested depth is an upper bound: slabs of equal depth keep the blocks of a
  // launch equally long (480 planes at depth 64 become 8 slabs of 60, not 7 of 64 and
  // one of 32)
  t.D = (g.nz + t.nslab - 1) / t.nslab;
  t.threads = ((t.TX * t.TY * H + 31) / 32) * 32;
  t.smem = (size_t)H * (t.TX + 2 * R) * (t.TY + 2 * R) * elem_bytes;
  return t;
}

template <typename T>
void launch_stencil(int R, dim3 grid, int threads, size_t smem, cudaStream_t s,
                    const StencilArgs<T>& a) {
  switch (R) {
    case 1: k_stencil<T, 1><<<grid, threads, smem, s>>>(a); break;
    case 2: k_stencil<T, 2><<<grid, threads, smem, s>>>(a); break;
    case 3: k_stencil<T, 3><<<grid, threads, smem, s>>>(a); break;
    case 4: k_stencil<T, 4><<<grid, threads, smem, s>>>(a); break;
    case 5: k_stencil<T, 5><<<grid, threads, smem, s>>>(a); break;
    case 6: k_stencil<T, 6><<<grid, threads, smem, s>>>(a); break;
    default: break;
  }
}

template <typename T>
cudaError_t prepare_stencil(int R, size_t smem) {
  const int bytes = (int)smem;
  switch (R) {
    case 1: return cudaFuncSetAttribute(k_stencil<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    case 2: return cudaFuncSetAttribute(k_stencil<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    case 3: return cudaFuncSetAttribute(k_stencil<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    case 4: return cudaFuncSetAttribute(k_stencil<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    case 5: return cudaFuncSetAttribute(k_stencil<T, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    case 6: return cudaFuncSetAttribute(k_stencil<T, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t prepare_stencil<double>(int, size_t);
template cudaError_t prepare_stencil<float>(int, size_t);
template void launch_stencil<double>(int, dim3, int, size_t, cudaStream_t, const StencilArgs<double>&);
template void launch_stencil<float>(int, dim3, int, size_t, cudaStream_t, const StencilArgs<float>&);

template <typename T>
void Engine<T>::release() {
  cudaFree(X); cudaFree(R); cudaFree(P0); cudaFree(P1); cudaFree(Q);
  cudaFree(sig_part); cudaFree(rho_part); cudaFree(slots); cudaFree(queue);
  X = R = P0 = P1 = Q = nullptr;
  sig_part = rho_part = nullptr;
  slots = nullptr;
  queue = nullptr;
  S = H = 0;
  n = 0;
}

template struct Engine<double>;
template struct Engine<float>;

}  // namespace transec

namespace {

// Columns in flight: enough point-halves per iteration to fill the GPU, bounded by
// memory (at most half of what is free) and by the number of items.
int choose_slots(long long n_mean, int H, size_t bytes_per_slot, long long nitems, int requested) {
  long long s;
  if (requested > 0) {
    s = requested;
  } else {
    const long long target = 24LL << 20;  // point-halves per iteration
    s = (target + n_mean * H - 1) / (n_mean * H);
    s = std::max(1LL, std::min(s, 4096LL));
  }
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && bytes_per_slot > 0) {
    const long long cap = (long long)(fr / 2 / bytes_per_slot);
    s = std::min(s, std::max(1LL, cap));
  }
  s = std::min(s, std::max(1LL, nitems));
  return (int)s;
}

template <typename T> Engine<T>& engine_of(transec_ctx* ctx);
template <> [[maybe_unused]] Engine<double>& engine_of<double>(transec_ctx* ctx) { return ctx->e64; }
template <> [[maybe_unused]] Engine<float>& engine_of<float>(transec_ctx* ctx) { return ctx->e32; }

template <typename T>
int engine_ensure(transec_ctx* ctx, Engine<T>& eng, int S, int H, long long n, int nblk2,
                  int nblk3) {
  using CT = typename Cx<T>::type;
  const bool same = eng.S >= S && eng.H == H && eng.n >= n && eng.nblk2 >= nblk2 &&
                    eng.nblk3 >= nblk3 && eng.X != nullptr;
  if (!same) {
    eng.release();
    const size_t vec = (size_t)S * H * n * sizeof(CT);
    CK(cudaMalloc(&eng.X, vec));
    CK(cudaMalloc(&eng.R, vec));
    CK(cudaMalloc(&eng.P0, vec));
    CK(cudaMalloc(&eng.P1, vec));
    CK(cudaMalloc(&eng.Q, vec));
    CK(cudaMalloc(&eng.sig_part, (size_t)S * nblk2 * 2 * sizeof(double)));
    CK(cudaMalloc(&eng.rho_part, (size_t)S * nblk3 * 4 * sizeof(double)));
    CK(cudaMalloc(&eng.slots, (size_t)S * sizeof(Slot)));
    CK(cudaMalloc(&eng.queue, sizeof(Queue)));
    eng.S = S;
    eng.H = H;
    eng.n = n;
    eng.nblk2 = nblk2;
    eng.nblk3 = nblk3;
  }
  return TRANSEC_OK;
}

// The operators of one solve and their launch shapes for H halves: the driver
// context alone, or every member of a batch (same device and stencil order).
struct BatchPlan {
  std::vector<Inst> insts;
  long long n_max = 0;
  double n_mean = 0;
  int R = 0;
  // per arithmetic (0: FP64 kernel, 1: FP32 kernel): the launch covering every member
  int grid_x[2] = {0, 0}, grid_y[2] = {0, 0}, threads[2] = {0, 0};
  size_t smem[2] = {0, 0};
  int nblk3 = 1;
};

BatchPlan plan_batch(const transec_ctx* driver, const std::vector<transec_ctx*>& members, int H,
                     bool fp32_iteration) {
  BatchPlan b;
  b.R = driver->g.R;
  for (const transec_ctx* m : members) {
    Inst in{};
    in.g = m->g;
    in.v = m->d_v;
    in.v32 = m->d_v32;
    in.gam = m->d_gam;
    in.gl = m->d_gl;
    in.gr = m->d_gr;
    in.phase = m->d_phase;
    in.gam32 = m->d_gam32;
    in.phase32 = m->d_phase32;
    in.lplanes = m->d_lplanes;
    in.rplanes = m->d_rplanes;
    in.nlp = (int)m->lplanes.size();
    in.nrp = (int)m->rplanes.size();
    in.nk = m->nk;
    // the iteration kernel takes the driver's tile options; the FP64 residual
    // replacement of the mixed form uses the default shape
    const int ty = driver->opts.tile_y, sl = driver->opts.slab;
    in.tile[0] = choose_tiles(m->g, H, sizeof(double2), StencilMax<double>::threads,
                              fp32_iteration ? 0 : ty, fp32_iteration ? 0 : sl);
    in.tile[1] = choose_tiles(m->g, H, sizeof(float2), StencilMax<float>::threads,
                              fp32_iteration ? ty : 0, fp32_iteration ? sl : 0);
    for (int k = 0; k < 2; ++k) {
      b.grid_x[k] = std::max(b.grid_x[k], in.tile[k].ntx * in.tile[k].nty);
      b.grid_y[k] = std::max(b.grid_y[k], in.tile[k].nslab);
      b.threads[k] = std::max(b.threads[k], in.tile[k].threads);
      b.smem[k] = std::max(b.smem[k], in.tile[k].smem);
    }
    b.n_max = std::max(b.n_max, m->g.n);
    b.n_mean += (double)m->g.n / members.size();
    b.nblk3 = std::max(b.nblk3, (int)std::min(1024LL, (m->g.n + 256 * 8 - 1) / (256 * 8)));
    b.insts.push_back(in);
  }
  return b;
}

int ensure_events(transec_ctx* ctx, int n) {
  while ((int)ctx->prof_ev.size() < n) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    ctx->prof_ev.push_back(e);
  }
  return TRANSEC_OK;
}

void accumulate_events(transec_ctx* ctx, int C, bool fp32) {
  for (int i = 0; i < C; ++i) {
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, ctx->prof_ev[4 * i], ctx->prof_ev[4 * i + 1]) == cudaSuccess) {
      if (fp32) {
        ctx->stencil32_ms += a;
        ctx->stencil32_launches += 1;
      } else {
        ctx->stencil_ms += a;
        ctx->stencil_launches += 1;
      }
    }
    if (cudaEventElapsedTime(&b, ctx->prof_ev[4 * i + 2], ctx->prof_ev[4 * i + 3]) == cudaSuccess) {
      ctx->update_ms += b;
      ctx->update_launches += 1;
    }
  }
  cudaGetLastError();
}

// FP64 buffers of the mixed-precision residual replacement (see mixed.cuh).
int mixed_ensure(transec_ctx* ctx, int S, int H, long long n, long long nblk_sig,
                 long long nblk_part) {
  const long long elems = (long long)S * H * n;
  if (ctx->mx_elems < elems) {
    cudaFree(ctx->mx_x); cudaFree(ctx->mx_q); cudaFree(ctx->mx_p);
    ctx->mx_x = ctx->mx_q = ctx->mx_p = nullptr;
    ctx->mx_elems = 0;
    CK(cudaMalloc(&ctx->mx_x, elems * sizeof(double2)));
    CK(cudaMalloc(&ctx->mx_q, elems * sizeof(double2)));
    CK(cudaMalloc(&ctx->mx_p, elems * sizeof(double2)));
    ctx->mx_elems = elems;
  }
  if (ctx->mx_sig_elems < S * nblk_sig * 2) {
    cudaFree(ctx->mx_sig);
    ctx->mx_sig = nullptr;
    ctx->mx_sig_elems = 0;
    CK(cudaMalloc(&ctx->mx_sig, S * nblk_sig * 2 * sizeof(double)));
    ctx->mx_sig_elems = S * nblk_sig * 2;
  }
  if (ctx->mx_part_elems < S * nblk_part * 4) {
    cudaFree(ctx->mx_part);
    ctx->mx_part = nullptr;
    ctx->mx_part_elems = 0;
    CK(cudaMalloc(&ctx->mx_part, S * nblk_part * 4 * sizeof(double)));
    ctx->mx_part_elems = S * nblk_part * 4;
  }
  if (ctx->mx_S < S) {
    cudaFree(ctx->mx_slots);
    ctx->mx_slots = nullptr;
    ctx->mx_S = 0;
    CK(cudaMalloc(&ctx->mx_slots, S * sizeof(Slot)));
    ctx->mx_S = S;
  }
  return TRANSEC_OK;
}

// Solve nitems (E, k, column) items with the slot engine of arithmetic type T and H
// halves: plain (T = double) or mixed precision (T = float, with FP64 residual
// replacement).  Item and result arrays are device pointers.
template <typename T>
int run_engine(transec_ctx* ctx, const std::vector<transec_ctx*>& members, const int* d_item_inst,
               int H, bool mixed, int nitems, const double* d_e, const int* d_ik,
               const long long* d_col, double* d_t, double* d_tm, int* d_it, int* d_st) {
  using CT = typename Cx<T>::type;
  Engine<T>& eng = engine_of<T>(ctx);
  const BatchPlan bp = plan_batch(ctx, members, H, !std::is_same<T, double>::value);
  const int ti = std::is_same<T, double>::value ? 0 : 1;  // tile set of the iteration kernel
  const long long nmax = bp.n_max;
  const size_t per_slot = (size_t)5 * H * nmax * sizeof(CT) +
                          (mixed ? (size_t)3 * H * nmax * sizeof(double2) : 0);
  const int S = choose_slots((long long)bp.n_mean, H, per_slot, nitems, ctx->opts.slots);
  int rc = engine_ensure<T>(ctx, eng, S, H, nmax, bp.grid_x[ti] * bp.grid_y[ti], bp.nblk3);
  if (rc) return rc;
  CK(prepare_stencil<T>(bp.R, bp.smem[ti]));
  if (mixed) {
    rc = mixed_ensure(ctx, S, H, nmax, (long long)bp.grid_x[0] * bp.grid_y[0], bp.nblk3);
    if (rc) return rc;
    CK(prepare_stencil<double>(bp.R, bp.smem[0]));
  }
  const int ninst = (int)bp.insts.size();
  if (ctx->insts_cap < ninst) {
    cudaFree(ctx->d_insts);
    ctx->d_insts = nullptr;
    ctx->insts_cap = 0;
    CK(cudaMalloc(&ctx->d_insts, ninst * sizeof(Inst)));
    ctx->insts_cap = ninst;
  }
  cudaStream_t s = ctx->s;
  CK(cudaMemcpyAsync(ctx->d_insts, bp.insts.data(), ninst * sizeof(Inst), cudaMemcpyHostToDevice, s));
  const Inst* dI = ctx->d_insts;
  const int Sl = eng.S;  // may exceed S when reusing larger buffers; extra slots stay idle
  Queue q0{};
  q0.nitems = nitems;
  CK(cudaMemcpyAsync(eng.queue, &q0, sizeof(Queue), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(eng.slots, 0, (size_t)Sl * sizeof(Slot), s));
  const long long n = nmax;
  const long long stride = (long long)H * nmax;

  AssignArgs aa{};
  aa.slots = eng.slots; aa.S = std::min(Sl, S); aa.H = H; aa.queue = eng.queue;
  aa.item_e = d_e; aa.item_ik = d_ik; aa.item_col = d_col;
  aa.item_inst = d_item_inst; aa.insts = dI; aa.ninst = ninst;

  InitArgs<T> ia{};
  ia.x = eng.X; ia.r = eng.R; ia.p = eng.P0; ia.slots = eng.slots; ia.n = n; ia.slot_stride = stride;
  ia.H = H; ia.insts = dI;
  const dim3 ig((unsigned)bp.nblk3, (unsigned)aa.S);

  StencilArgs<T> sa{};
  sa.r = eng.R; sa.q = eng.Q; sa.part = eng.sig_part; sa.slots = eng.slots; sa.H = H; sa.conj = 0;
  sa.slot_stride = stride; sa.insts = dI; sa.tile_idx = ti;
  const dim3 sg((unsigned)bp.grid_x[ti], (unsigned)bp.grid_y[ti], (unsigned)aa.S);
  const int sthreads = bp.threads[ti];
  const size_t ssmem = bp.smem[ti];

  UpdateArgs<T> ua{};
  ua.x = eng.X; ua.r = eng.R; ua.q = eng.Q; ua.sig_part = eng.sig_part;
  ua.sig_nblk = bp.grid_x[ti] * bp.grid_y[ti]; ua.rho_part = eng.rho_part; ua.slots = eng.slots;
  ua.n = n; ua.slot_stride = stride; ua.H = H; ua.insts = dI;
  const dim3 ug((unsigned)bp.nblk3, (unsigned)aa.S);

  ScalarArgs ca{};
  ca.rho_part = eng.rho_part; ca.nblk = bp.nblk3; ca.slots = eng.slots; ca.S = aa.S; ca.H = H;
  ca.maxit = mixed ? std::min(ctx->opts.maxit, ctx->opts.mixed_maxit) : ctx->opts.maxit;
  ca.tol = ctx->opts.tol;
  // the FP32 cycle restarts only on progress (no stall rule: BiCG residuals wander for
  // thousands of iterations before they fall, and a restart there loses the progress)
  ca.mixed = mixed ? 1 : 0; ca.reliable = ctx->opts.reliable; ca.stall = 1 << 30;
  ca.max_gap = 1 << 30;
  ca.decade_its = mixed ? ctx->opts.mixed_decade_its : 0;
  const int cgrid = (aa.S + 7) / 8;

  // the trace reads the FP64 solution: the engine's x (plain) or x64 (mixed)
  TraceArgs<double> ta{};
  ta.x = mixed ? ctx->mx_x : reinterpret_cast<const double2*>(eng.X);
  ta.slots = eng.slots; ta.queue = eng.queue; ta.res_t = d_t; ta.res_tm = d_tm; ta.res_it = d_it;
  ta.res_status = d_st; ta.slot_stride = stride; ta.H = H; ta.insts = dI;

  // mixed precision: residual replacement stage
  MxPrepArgs mp{eng.slots, ctx->mx_slots, aa.S};
  MxAccumArgs mac{ctx->mx_x, reinterpret_cast<float2*>(eng.X), ctx->mx_slots, n, stride, H, dI};
  StencilArgs<double> s64{};
  s64.r = ctx->mx_x; s64.p_in = ctx->mx_x; s64.p_out = ctx->mx_p; s64.q = ctx->mx_q;
  s64.part = ctx->mx_sig; s64.slots = ctx->mx_slots; s64.H = H; s64.conj = 0;
  s64.slot_stride = stride; s64.insts = dI; s64.tile_idx = 0;
  const dim3 sg64((unsigned)bp.grid_x[0], (unsigned)bp.grid_y[0], (unsigned)aa.S);
  MxFinishArgs mf{ctx->mx_q, reinterpret_cast<float2*>(eng.R), ctx->mx_slots, ctx->mx_part, n,
                  stride, H, dI};
  MxScalarArgs ms{ctx->mx_part, bp.nblk3, ctx->mx_slots, eng.slots, aa.S, H, ctx->opts.tol};
  MxInitArgs mi{ctx->mx_x, eng.slots, n, stride, H, dI};

  k_assign<<<1, 1024, 0, s>>>(aa);
  k_init<T><<<ig, 256, 0, s>>>(ia);
  if (mixed) k_mx_init<<<ig, 256, 0, s>>>(mi);
  CHECK_LAUNCH();

  const int C = ctx->opts.chunk;
  const bool prof = ctx->opts.profile != 0;
  if (prof) {
    rc = ensure_events(ctx, 4 * C);
    if (rc) return rc;
  }
  // One chunk: C iterations, the mixed form's residual replacement, trace, refill.
  // Default: the chunk is the body of a device-side WHILE loop (a conditional graph
  // node), so a whole solve is one graph launch; with profiling (event records are not
  // allowed in conditional bodies) or opts.host_loop the host launches chunk by chunk.
  const bool device_loop = !prof && !ctx->opts.host_loop;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle loop{};
  if (device_loop) {
    CK(cudaGraphCreate(&graph, 0));
    cudaError_t eh = cudaGraphConditionalHandleCreate(&loop, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (eh == cudaSuccess) eh = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    if (eh == cudaSuccess)
      eh = cudaStreamBeginCaptureToGraph(s, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal);
    if (eh != cudaSuccess) {
      cudaGraphDestroy(graph);
      cudaGetLastError();
      return fail(ctx, TRANSEC_ECUDA, std::string("device loop set-up: ") + cudaGetErrorString(eh));
    }
  } else {
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  }
  for (int i = 0; i < C; ++i) {
    sa.p_in = (i % 2 == 0) ? eng.P0 : eng.P1;
    sa.p_out = (i % 2 == 0) ? eng.P1 : eng.P0;
    if (prof) cudaEventRecordWithFlags(ctx->prof_ev[4 * i + 0], s, cudaEventRecordExternal);
    launch_stencil<T>(bp.R, sg, sthreads, ssmem, s, sa);
    if (prof) cudaEventRecordWithFlags(ctx->prof_ev[4 * i + 1], s, cudaEventRecordExternal);
    ua.p = sa.p_out;
    if (prof) cudaEventRecordWithFlags(ctx->prof_ev[4 * i + 2], s, cudaEventRecordExternal);
    k_update<T><<<ug, 256, 0, s>>>(ua);
    if (prof) cudaEventRecordWithFlags(ctx->prof_ev[4 * i + 3], s, cudaEventRecordExternal);
    k_scalars<<<cgrid, 256, 0, s>>>(ca);
  }
  if (mixed) {
    k_mx_prep<<<(aa.S + 255) / 256, 256, 0, s>>>(mp);
    k_mx_accum<<<ig, 256, 0, s>>>(mac);
    launch_stencil<double>(bp.R, sg64, bp.threads[0], bp.smem[0], s, s64);
    k_mx_finish<<<ig, 256, 0, s>>>(mf);
    k_mx_scalars<<<cgrid, 256, 0, s>>>(ms);
  }
  k_trace<double><<<aa.S, 256, 0, s>>>(ta);
  k_assign<<<1, 1024, 0, s>>>(aa);
  k_init<T><<<ig, 256, 0, s>>>(ia);
  if (mixed) k_mx_init<<<ig, 256, 0, s>>>(mi);
  if (device_loop) {
    k_continue<<<1, 1, 0, s>>>(loop, eng.queue);
  } else {
    cudaMemcpyAsync(ctx->h_harvest, &eng.queue->harvested, sizeof(int), cudaMemcpyDeviceToHost, s);
  }
  {
    cudaGraph_t captured = nullptr;
    cudaError_t e1 = cudaStreamEndCapture(s, &captured);
    if (!device_loop) graph = captured;
    if (e1 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return fail(ctx, TRANSEC_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e1));
    }
  }
  {
    cudaError_t e2 = cudaGraphInstantiate(&exec, graph, 0);
    if (e2 != cudaSuccess) {
      cudaGraphDestroy(graph);
      cudaGetLastError();
      return fail(ctx, TRANSEC_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
    }
  }
  const long long per_chunk = 3LL * C + 3 + (mixed ? 6 : 0) + (device_loop ? 1 : 0);
  const long long max_chunks =
      ((long long)nitems / std::max(1, aa.S) + 2) * ((long long)ctx->opts.maxit / C + 2) + 16;
  // chunks per device-loop launch: a launch always ends, and the host re-checks
  const int per_launch = 4096;
  long long chunks = 0;
  int rcode = TRANSEC_OK;
  *ctx->h_harvest = 0;
  while (true) {
    cudaError_t e3 = cudaSuccess;
    if (device_loop) {
      const int lim = (int)std::min<long long>(chunks + per_launch, 1LL << 30);
      e3 = cudaMemcpyAsync(&eng.queue->limit, &lim, sizeof(int), cudaMemcpyHostToDevice, s);
      if (e3 == cudaSuccess) e3 = cudaGraphLaunch(exec, s);
      Queue qh{};
      if (e3 == cudaSuccess) e3 = cudaMemcpyAsync(&qh, eng.queue, sizeof(Queue), cudaMemcpyDeviceToHost, s);
      if (e3 == cudaSuccess) e3 = cudaStreamSynchronize(s);
      if (e3 == cudaSuccess) {
        chunks = qh.chunks;
        *ctx->h_harvest = qh.harvested;
      }
    } else {
      e3 = cudaGraphLaunch(exec, s);
      if (e3 == cudaSuccess) e3 = cudaStreamSynchronize(s);
      if (e3 == cudaSuccess) ++chunks;
    }
    if (e3 != cudaSuccess) {
      cudaGetLastError();
      rcode = fail(ctx, TRANSEC_ECUDA, std::string("solver chunk: ") + cudaGetErrorString(e3));
      break;
    }
    if (prof) accumulate_events(ctx, C, !std::is_same<T, double>::value);
    if (*ctx->h_harvest >= nitems) break;
    if (chunks > max_chunks) {
      rcode = fail(ctx, TRANSEC_ETIMEOUT, "solver did not drain its work queue within the iteration bound");
      break;
    }
  }
  ctx->launches += (mixed ? 3 : 2) + chunks * per_chunk;
  if (rcode == TRANSEC_OK && d_it) {
    std::vector<int> its(nitems), inst(nitems, 0);
    bool ok = cudaMemcpy(its.data(), d_it, nitems * sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
    if (ok && d_item_inst)
      ok = cudaMemcpy(inst.data(), d_item_inst, nitems * sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
    if (ok) {
      for (int i = 0; i < nitems; ++i) {
        const int ii = (inst[i] >= 0 && inst[i] < ninst) ? inst[i] : 0;
        const long long pa = (long long)its[i] * H * bp.insts[ii].g.n;
        if (std::is_same<T, double>::value) ctx->point_applies += pa;
        else ctx->point_applies32 += pa;
      }
    }
    cudaGetLastError();
  }
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  return rcode;
}

// Device scratch for host-pointer calls.
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};

int begin_call(transec_ctx* ctx) {
  CK(cudaEventRecord(ctx->ev_in, ctx->user));
  CK(cudaStreamWaitEvent(ctx->s, ctx->ev_in, 0));
  return TRANSEC_OK;
}

int end_call(transec_ctx* ctx) {
  CK(cudaEventRecord(ctx->ev_out, ctx->s));
  CK(cudaStreamWaitEvent(ctx->user, ctx->ev_out, 0));
  CK(cudaStreamSynchronize(ctx->s));
  return TRANSEC_OK;
}

int check_ready(transec_ctx* ctx) {
  if (!ctx) return TRANSEC_EINVAL;
  if (!ctx->have_v) return fail(ctx, TRANSEC_ESTATE, "potential not set");
  if (!ctx->have_abc) return fail(ctx, TRANSEC_ESTATE, "absorbing boundary not set");
  if (!ctx->have_k) return fail(ctx, TRANSEC_ESTATE, "k-mesh not set");
  return TRANSEC_OK;
}

// Items with device-resident arrays -> results in device arrays, for one method group.
// Items of a batch (members[item_inst[i]], or ctx alone when item_inst is NULL), solved
// in one engine run with the driver context's options, buffers and stream.
int solve_batch(transec_ctx* ctx, const std::vector<transec_ctx*>& members, const int* d_inst,
                int H, int nitems, const double* d_e, const int* d_ik, const long long* d_col,
                double* d_t, double* d_tm, int* d_it, int* d_st) {
  if (nitems == 0) return TRANSEC_OK;
  if (ctx->opts.precision != TRANSEC_PREC_MIXED)
    return run_engine<double>(ctx, members, d_inst, H, false, nitems, d_e, d_ik, d_col, d_t, d_tm,
                              d_it, d_st);
  int rc = run_engine<float>(ctx, members, d_inst, H, true, nitems, d_e, d_ik, d_col, d_t, d_tm,
                             d_it, d_st);
  if (rc != TRANSEC_OK) return rc;
  // Columns the mixed form could not finish (not converged, or a breakdown of the
  // FP32 recurrence) are solved again with the plain FP64 engine.
  std::vector<int> st(nitems);
  CK(cudaMemcpyAsync(st.data(), d_st, nitems * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  std::vector<int> redo;
  for (int i = 0; i < nitems; ++i)
    if (st[i] == TRANSEC_ENOCONV || st[i] == TRANSEC_EBREAKDOWN) redo.push_back(i);
  if (redo.empty()) return TRANSEC_OK;
  const int m = (int)redo.size();
  std::vector<double> he(nitems);
  std::vector<int> hk(nitems), hit(nitems), hi(nitems, 0);
  std::vector<long long> hc(nitems);
  if (d_inst)
    CK(cudaMemcpyAsync(hi.data(), d_inst, nitems * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaMemcpyAsync(he.data(), d_e, nitems * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaMemcpyAsync(hk.data(), d_ik, nitems * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaMemcpyAsync(hc.data(), d_col, nitems * sizeof(long long), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaMemcpyAsync(hit.data(), d_it, nitems * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  std::vector<double> re(m);
  std::vector<int> rk(m), ri(m);
  std::vector<long long> rcl(m);
  for (int u = 0; u < m; ++u) {
    re[u] = he[redo[u]];
    rk[u] = hk[redo[u]];
    rcl[u] = hc[redo[u]];
    ri[u] = hi[redo[u]];
  }
  DevBuf be, bk, bc, bt, btm, bit, bst, bi;
  CK(cudaMalloc(&bi.p, m * sizeof(int)));
  CK(cudaMemcpyAsync(bi.p, ri.data(), m * sizeof(int), cudaMemcpyHostToDevice, ctx->s));
  CK(cudaMalloc(&be.p, m * sizeof(double)));
  CK(cudaMalloc(&bk.p, m * sizeof(int)));
  CK(cudaMalloc(&bc.p, m * sizeof(long long)));
  CK(cudaMalloc(&bt.p, m * sizeof(double)));
  CK(cudaMalloc(&btm.p, m * sizeof(double)));
  CK(cudaMalloc(&bit.p, m * sizeof(int)));
  CK(cudaMalloc(&bst.p, m * sizeof(int)));
  CK(cudaMemcpyAsync(be.p, re.data(), m * sizeof(double), cudaMemcpyHostToDevice, ctx->s));
  CK(cudaMemcpyAsync(bk.p, rk.data(), m * sizeof(int), cudaMemcpyHostToDevice, ctx->s));
  CK(cudaMemcpyAsync(bc.p, rcl.data(), m * sizeof(long long), cudaMemcpyHostToDevice, ctx->s));
  rc = run_engine<double>(ctx, members, d_inst ? (const int*)bi.p : nullptr, H, false, m,
                          (double*)be.p, (int*)bk.p, (long long*)bc.p, (double*)bt.p,
                          (double*)btm.p, (int*)bit.p, (int*)bst.p);
  if (rc != TRANSEC_OK) return rc;
  std::vector<double> t(m), tm(m);
  std::vector<int> it(m), s2(m);
  CK(cudaMemcpyAsync(t.data(), bt.p, m * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaMemcpyAsync(tm.data(), btm.p, m * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaMemcpyAsync(it.data(), bit.p, m * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaMemcpyAsync(s2.data(), bst.p, m * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  for (int u = 0; u < m; ++u) {
    const int i = redo[u];
    CK(cudaMemcpyAsync(d_t + i, &t[u], sizeof(double), cudaMemcpyHostToDevice, ctx->s));
    CK(cudaMemcpyAsync(d_tm + i, &tm[u], sizeof(double), cudaMemcpyHostToDevice, ctx->s));
    const int tot = hit[i] + it[u];  // iterations of both attempts
    CK(cudaMemcpyAsync(d_it + i, &tot, sizeof(int), cudaMemcpyHostToDevice, ctx->s));
    CK(cudaMemcpyAsync(d_st + i, &s2[u], sizeof(int), cudaMemcpyHostToDevice, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
  }
  ctx->fallbacks += m;
  return TRANSEC_OK;
}

int solve_items(transec_ctx* ctx, int H, int nitems, const double* d_e, const int* d_ik,
                const long long* d_col, double* d_t, double* d_tm, int* d_it, int* d_st) {
  return solve_batch(ctx, {ctx}, nullptr, H, nitems, d_e, d_ik, d_col, d_t, d_tm, d_it, d_st);
}

// Host item lists -> host results (one method group); `inst` (may be empty) holds the
// batch member of each item.
int solve_host_items(transec_ctx* ctx, const std::vector<transec_ctx*>& members,
                     const std::vector<int>& inst, int H, const std::vector<double>& e,
                     const std::vector<int>& ik, const std::vector<long long>& col,
                     std::vector<double>& t, std::vector<double>& tm, std::vector<int>& it,
                     std::vector<int>& st) {
  const int nitems = (int)e.size();
  t.assign(nitems, 0.0);
  tm.assign(nitems, 0.0);
  it.assign(nitems, 0);
  st.assign(nitems, 0);
  if (nitems == 0) return TRANSEC_OK;
  DevBuf be, bk, bc, bt, btm, bit, bst;
  CK(cudaMalloc(&be.p, nitems * sizeof(double)));
  CK(cudaMalloc(&bk.p, nitems * sizeof(int)));
  CK(cudaMalloc(&bc.p, nitems * sizeof(long long)));
  CK(cudaMalloc(&bt.p, nitems * sizeof(double)));
  CK(cudaMalloc(&btm.p, nitems * sizeof(double)));
  CK(cudaMalloc(&bit.p, nitems * sizeof(int)));
  CK(cudaMalloc(&bst.p, nitems * sizeof(int)));
  CK(cudaMemcpyAsync(be.p, e.data(), nitems * sizeof(double), cudaMemcpyHostToDevice, ctx->s));
  CK(cudaMemcpyAsync(bk.p, ik.data(), nitems * sizeof(int), cudaMemcpyHostToDevice, ctx->s));
  CK(cudaMemcpyAsync(bc.p, col.data(), nitems * sizeof(long long), cudaMemcpyHostToDevice, ctx->s));
  DevBuf bi;
  if (!inst.empty()) {
    CK(cudaMalloc(&bi.p, nitems * sizeof(int)));
    CK(cudaMemcpyAsync(bi.p, inst.data(), nitems * sizeof(int), cudaMemcpyHostToDevice, ctx->s));
  }
  int rc = solve_batch(ctx, members, (const int*)bi.p, H, nitems, (double*)be.p, (int*)bk.p,
                       (long long*)bc.p, (double*)bt.p, (double*)btm.p, (int*)bit.p, (int*)bst.p);
  if (rc != TRANSEC_OK && rc != TRANSEC_ENOCONV && rc != TRANSEC_EBREAKDOWN) return rc;
  CK(cudaMemcpyAsync(t.data(), bt.p, nitems * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaMemcpyAsync(tm.data(), btm.p, nitems * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaMemcpyAsync(it.data(), bit.p, nitems * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaMemcpyAsync(st.data(), bst.p, nitems * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  return rc;
}

// Number of halves for k index ik under the configured method, or -1 if invalid.
int halves_for(const transec_ctx* ctx, int ik) {
  const bool rp = real_phase(ctx->kfrac[2 * ik], ctx->kfrac[2 * ik + 1]);
  switch (ctx->opts.method) {
    case TRANSEC_METHOD_COCG: return rp ? 1 : -1;
    case TRANSEC_METHOD_BICG: return 2;
    default: return rp ? 1 : 2;
  }
}

}  // namespace

namespace {
__global__ void k_to_float(const double* a, float* b, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void k_count_nonfinite(const double* a, long long n, int* bad) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(a[i])) atomicAdd(bad, 1);
}
// out[0] = max |V(x, y, z) - V(-x mod nx, -y mod ny, z)|, out[1] = max |V|, as the bit
// patterns of non-negative doubles (which order like the values)
__global__ void k_inversion_gap(const double* v, int nx, int ny, long long n, unsigned long long* out) {
  const long long nxy = (long long)nx * ny;
  double gap = 0.0, mx = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long z = i / nxy;
    const int w = (int)(i - z * nxy);
    const int y = w / nx, x = w - y * nx;
    const long long im = z * nxy + (x ? nx - x : 0) + (long long)nx * (y ? ny - y : 0);
    gap = fmax(gap, fabs(v[i] - v[im]));
    mx = fmax(mx, fabs(v[i]));
  }
  atomicMax(out, (unsigned long long)__double_as_longlong(gap));
  atomicMax(out + 1, (unsigned long long)__double_as_longlong(mx));
}
}  // namespace

// ---------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------

extern "C" {

int transec_version(void) { return 10000; }

const char* transec_status_string(int status) {
  switch (status) {
    case TRANSEC_OK: return "ok";
    case TRANSEC_EINVAL: return "invalid argument";
    case TRANSEC_ENOMEM: return "out of memory";
    case TRANSEC_ECUDA: return "CUDA error";
    case TRANSEC_ENOCONV: return "not converged within maxit";
    case TRANSEC_EBREAKDOWN: return "Krylov breakdown";
    case TRANSEC_ETIMEOUT: return "bounded wait timed out";
    case TRANSEC_ESTATE: return "call order violated";
    default: return "unknown status";
  }
}

int transec_create(transec_ctx** out, int nx, int ny, int nz, double hx, double hy, double hz,
                   int fd_order, int device, void* cuda_stream) {
  if (!out) return TRANSEC_EINVAL;
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 2 || !(hx > 0) || !(hy > 0) || !(hz > 0) || !std::isfinite(hx) ||
      !std::isfinite(hy) || !std::isfinite(hz) || fd_order < 2 || fd_order > 12 || fd_order % 2)
    return TRANSEC_EINVAL;
  if ((long long)nx * ny * nz > (1LL << 31)) return TRANSEC_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return TRANSEC_ECUDA;
  }
  transec_ctx* ctx = new transec_ctx();
  DeviceGuard dg(device);
  ctx->device = device;
  ctx->user = (cudaStream_t)cuda_stream;
  ctx->order = fd_order;
  ctx->hx = hx; ctx->hy = hy; ctx->hz = hz;
  Geometry& g = ctx->g;
  g.nx = nx; g.ny = ny; g.nz = nz; g.R = fd_order / 2;
  g.nxy = (long long)nx * ny;
  g.n = g.nxy * nz;
  double c[kMaxR + 1];
  fd_coefficients(fd_order, c);
  for (int m = 0; m <= kMaxR; ++m) {
    const double cm = m <= g.R ? c[m] : 0.0;
    g.kx[m] = cm / (2.0 * hx * hx);
    g.ky[m] = cm / (2.0 * hy * hy);
    g.kz[m] = cm / (2.0 * hz * hz);
  }
  g.diag_c = 0.5 * c[0] * (1.0 / (hx * hx) + 1.0 / (hy * hy) + 1.0 / (hz * hz));
  ctx->opts = transec_solver_opts{};
  default_opts(&ctx->opts);
  if (cudaStreamCreateWithFlags(&ctx->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost(&ctx->h_harvest, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&ctx->d_v, g.n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ctx->d_v32, g.n * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    transec_destroy(ctx);
    return TRANSEC_ECUDA;
  }
  *out = ctx;
  return TRANSEC_OK;
}

int transec_set_potential(transec_ctx* ctx, const double* v_ks, int on_device) {
  if (!ctx) return TRANSEC_EINVAL;
  if (!v_ks) return fail(ctx, TRANSEC_EINVAL, "v_ks is NULL");
  DeviceGuard dg(ctx->device);
  int rc = begin_call(ctx);
  if (rc) return rc;
  const long long n = ctx->g.n;
  CK(cudaMemcpyAsync(ctx->d_v, v_ks, n * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->s));
  DevBuf bad;
  CK(cudaMalloc(&bad.p, sizeof(int)));
  CK(cudaMemsetAsync(bad.p, 0, sizeof(int), ctx->s));
  k_count_nonfinite<<<256, 256, 0, ctx->s>>>(ctx->d_v, n, (int*)bad.p);
  k_to_float<<<1024, 256, 0, ctx->s>>>(ctx->d_v, ctx->d_v32, n);
  DevBuf gapb;
  CK(cudaMalloc(&gapb.p, 2 * sizeof(unsigned long long)));
  CK(cudaMemsetAsync(gapb.p, 0, 2 * sizeof(unsigned long long), ctx->s));
  k_inversion_gap<<<256, 256, 0, ctx->s>>>(ctx->d_v, ctx->g.nx, ctx->g.ny, n, (unsigned long long*)gapb.p);
  CHECK_LAUNCH();
  int hbad = 0;
  double hgap[2] = {0.0, 0.0};
  CK(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaMemcpyAsync(hgap, gapb.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  rc = end_call(ctx);
  if (rc) return rc;
  if (hbad) {
    ctx->have_v = false;
    ctx->v_inversion_gap = std::nan("");
    return fail(ctx, TRANSEC_EINVAL, "v_ks holds non-finite values");
  }
  ctx->v_inversion_gap = hgap[1] > 0.0 ? hgap[0] / hgap[1] : 0.0;
  ctx->have_v = true;
  return TRANSEC_OK;
}

int transec_set_abc(transec_ctx* ctx, const double* gamma_l, const double* gamma_r) {
  if (!ctx) return TRANSEC_EINVAL;
  if (!gamma_l || !gamma_r) return fail(ctx, TRANSEC_EINVAL, "gamma array is NULL");
  const int nz = ctx->g.nz;
  std::vector<int> lp, rp;
  std::vector<double> gam(nz);
  for (int l = 0; l < nz; ++l) {
    if (!std::isfinite(gamma_l[l]) || !std::isfinite(gamma_r[l]) || gamma_l[l] < 0 || gamma_r[l] < 0)
      return fail(ctx, TRANSEC_EINVAL, "gamma values must be finite and non-negative");
    if (gamma_l[l] > 0) lp.push_back(l);
    if (gamma_r[l] > 0) rp.push_back(l);
    gam[l] = gamma_l[l] + gamma_r[l];
  }
  if (lp.empty()) return fail(ctx, TRANSEC_EINVAL, "left absorbing profile is zero everywhere");
  DeviceGuard dg(ctx->device);
  cudaFree(ctx->d_gl); cudaFree(ctx->d_gr); cudaFree(ctx->d_gam); cudaFree(ctx->d_gam32);
  cudaFree(ctx->d_lplanes); cudaFree(ctx->d_rplanes);
  ctx->d_gl = ctx->d_gr = ctx->d_gam = nullptr;
  ctx->d_gam32 = nullptr;
  ctx->d_lplanes = ctx->d_rplanes = nullptr;
  ctx->have_abc = false;
  CK(cudaMalloc(&ctx->d_gl, nz * sizeof(double)));
  CK(cudaMalloc(&ctx->d_gr, nz * sizeof(double)));
  CK(cudaMalloc(&ctx->d_gam, nz * sizeof(double)));
  CK(cudaMalloc(&ctx->d_lplanes, lp.size() * sizeof(int)));
  CK(cudaMalloc(&ctx->d_rplanes, std::max<size_t>(1, rp.size()) * sizeof(int)));
  CK(cudaMemcpy(ctx->d_gl, gamma_l, nz * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_gr, gamma_r, nz * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_gam, gam.data(), nz * sizeof(double), cudaMemcpyHostToDevice));
  {
    std::vector<float> g32(gam.begin(), gam.end());
    CK(cudaMalloc(&ctx->d_gam32, nz * sizeof(float)));
    CK(cudaMemcpy(ctx->d_gam32, g32.data(), nz * sizeof(float), cudaMemcpyHostToDevice));
  }
  CK(cudaMemcpy(ctx->d_lplanes, lp.data(), lp.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!rp.empty())
    CK(cudaMemcpy(ctx->d_rplanes, rp.data(), rp.size() * sizeof(int), cudaMemcpyHostToDevice));
  ctx->gl.assign(gamma_l, gamma_l + nz);
  ctx->gr.assign(gamma_r, gamma_r + nz);
  ctx->lplanes = lp;
  ctx->rplanes = rp;
  ctx->have_abc = true;
  return TRANSEC_OK;
}

int transec_set_kmesh(transec_ctx* ctx, int nk, const double* kfrac, const double* weights) {
  if (!ctx) return TRANSEC_EINVAL;
  if (nk < 1 || !kfrac) return fail(ctx, TRANSEC_EINVAL, "nk must be >= 1 and kfrac non-NULL");
  for (int i = 0; i < 2 * nk; ++i)
    if (!std::isfinite(kfrac[i])) return fail(ctx, TRANSEC_EINVAL, "non-finite k");
  std::vector<double> w(nk, 1.0 / nk);
  if (weights) {
    for (int i = 0; i < nk; ++i) {
      if (!std::isfinite(weights[i])) return fail(ctx, TRANSEC_EINVAL, "non-finite weight");
      w[i] = weights[i];
    }
  }
  // phase table [k][sign][axis][w]
  std::vector<double2> tab((size_t)nk * 2 * 2 * kPhaseN);
  for (int k = 0; k < nk; ++k)
    for (int sgn = 0; sgn < 2; ++sgn)
      for (int ax = 0; ax < 2; ++ax)
        for (int wi = 0; wi < kPhaseN; ++wi) {
          const double kap = (sgn ? -1.0 : 1.0) * kfrac[2 * k + ax];
          tab[(((size_t)k * 2 + sgn) * 2 + ax) * kPhaseN + wi] = bloch(kap, wi - kPhaseW);
        }
  DeviceGuard dg(ctx->device);
  cudaFree(ctx->d_phase);
  cudaFree(ctx->d_phase32);
  ctx->d_phase = nullptr;
  ctx->d_phase32 = nullptr;
  ctx->have_k = false;
  CK(cudaMalloc(&ctx->d_phase, tab.size() * sizeof(double2)));
  CK(cudaMemcpy(ctx->d_phase, tab.data(), tab.size() * sizeof(double2), cudaMemcpyHostToDevice));
  {
    std::vector<float2> t32(tab.size());
    for (size_t u = 0; u < tab.size(); ++u) t32[u] = make_float2((float)tab[u].x, (float)tab[u].y);
    CK(cudaMalloc(&ctx->d_phase32, t32.size() * sizeof(float2)));
    CK(cudaMemcpy(ctx->d_phase32, t32.data(), t32.size() * sizeof(float2), cudaMemcpyHostToDevice));
  }
  ctx->nk = nk;
  ctx->kfrac.assign(kfrac, kfrac + 2 * nk);
  ctx->kw = w;
  ctx->have_k = true;
  return TRANSEC_OK;
}

int transec_set_solver(transec_ctx* ctx, const transec_solver_opts* opts) {
  if (!ctx || !opts) return TRANSEC_EINVAL;
  transec_solver_opts o = *opts;
  if (o.method < 0 || o.method > 2 || o.precision < 0 || o.precision > 2 || o.tol < 0 ||
      o.maxit < 0 || o.slots < 0 || o.chunk < 0 || o.tile_y < 0 || o.slab < 0 || o.mixed_maxit < 0 ||
      o.psym < 0 || o.psym > 1 || !std::isfinite(o.sketch_guard) ||
      !std::isfinite(o.tol) || !std::isfinite(o.reliable))
    return fail(ctx, TRANSEC_EINVAL, "invalid solver options");
  default_opts(&o);
  ctx->opts = o;
  return TRANSEC_OK;
}

int transec_get_solver(const transec_ctx* ctx, transec_solver_opts* opts) {
  if (!ctx || !opts) return TRANSEC_EINVAL;
  *opts = ctx->opts;
  return TRANSEC_OK;
}

int transec_n_rhs(const transec_ctx* ctx, int64_t* n_rhs) {
  if (!ctx || !n_rhs) return TRANSEC_EINVAL;
  *n_rhs = ctx->have_abc ? (int64_t)ctx->lplanes.size() * ctx->g.nxy : 0;
  return TRANSEC_OK;
}

int transec_column_contributions(transec_ctx* ctx, int nitems, const double* energies,
                                 const int* ik, const int64_t* cols, double* t_out,
                                 double* t_minus_out, int* iters_out, int* status_out,
                                 int on_device) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (nitems < 0) return fail(ctx, TRANSEC_EINVAL, "nitems < 0");
  if (nitems == 0) return TRANSEC_OK;
  if (!energies || !ik || !cols || !t_out) return fail(ctx, TRANSEC_EINVAL, "NULL item or output array");
  DeviceGuard dg(ctx->device);
  rc = begin_call(ctx);
  if (rc) return rc;
  // One method group per call on the device path: the k-points of the items decide it.
  std::vector<int> hik;
  if (on_device) {
    hik.resize(nitems);
    CK(cudaMemcpyAsync(hik.data(), ik, nitems * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
  } else {
    hik.assign(ik, ik + nitems);
  }
  int H = 0;
  for (int i = 0; i < nitems; ++i) {
    if (hik[i] < 0 || hik[i] >= ctx->nk) return fail(ctx, TRANSEC_EINVAL, "k index out of range");
    const int h = halves_for(ctx, hik[i]);
    if (h < 0) return fail(ctx, TRANSEC_EINVAL, "COCG requested for a k-point with complex Bloch phase");
    H = std::max(H, h);
  }
  int worst = TRANSEC_OK;
  if (on_device) {
    DevBuf btm, bit, bst;
    double* dtm = t_minus_out;
    int* dit = iters_out;
    int* dst = status_out;
    if (!dtm) { CK(cudaMalloc(&btm.p, nitems * sizeof(double))); dtm = (double*)btm.p; }
    if (!dit) { CK(cudaMalloc(&bit.p, nitems * sizeof(int))); dit = (int*)bit.p; }
    if (!dst) { CK(cudaMalloc(&bst.p, nitems * sizeof(int))); dst = (int*)bst.p; }
    rc = solve_items(ctx, H, nitems, energies, ik, (const long long*)cols, t_out, dtm, dit, dst);
    if (rc != TRANSEC_OK) return rc;
    std::vector<int> hs(nitems);
    CK(cudaMemcpyAsync(hs.data(), dst, nitems * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    for (int v : hs)
      if (severity(v) > severity(worst)) worst = v;
  } else {
    std::vector<double> e(energies, energies + nitems);
    std::vector<long long> c(cols, cols + nitems);
    std::vector<double> t, tm;
    std::vector<int> it, st;
    rc = solve_host_items(ctx, {ctx}, {}, H, e, hik, c, t, tm, it, st);
    if (rc != TRANSEC_OK && rc != TRANSEC_ENOCONV && rc != TRANSEC_EBREAKDOWN) return rc;
    std::memcpy(t_out, t.data(), nitems * sizeof(double));
    if (t_minus_out) std::memcpy(t_minus_out, tm.data(), nitems * sizeof(double));
    if (iters_out) std::memcpy(iters_out, it.data(), nitems * sizeof(int));
    if (status_out) std::memcpy(status_out, st.data(), nitems * sizeof(int));
    for (int v : st)
      if (severity(v) > severity(worst)) worst = v;
  }
  rc = end_call(ctx);
  if (rc) return rc;
  if (worst != TRANSEC_OK) ctx->err = std::string("some columns failed: ") + transec_status_string(worst);
  return worst;
}

int transec_batch_column_contributions(int nctx, transec_ctx* const* ctxs, int nitems,
                                       const int* ictx, const double* energies, const int* ik,
                                       const int64_t* cols, double* t_out, double* t_minus_out,
                                       int* iters_out, int* status_out, int on_device) {
  if (nctx < 1 || !ctxs || !ctxs[0]) return TRANSEC_EINVAL;
  transec_ctx* ctx = ctxs[0];
  std::vector<transec_ctx*> members(ctxs, ctxs + nctx);
  for (transec_ctx* m : members) {
    if (!m) return fail(ctx, TRANSEC_EINVAL, "NULL context in batch");
    int rc = check_ready(m);
    if (rc) return fail(ctx, rc, std::string("batch member not ready: ") + m->err);
    if (m->device != ctx->device) return fail(ctx, TRANSEC_EINVAL, "batch contexts on different devices");
    if (m->g.R != ctx->g.R) return fail(ctx, TRANSEC_EINVAL, "batch contexts with different stencil orders");
  }
  if (nitems < 0) return fail(ctx, TRANSEC_EINVAL, "nitems < 0");
  if (nitems == 0) return TRANSEC_OK;
  if (!ictx || !energies || !ik || !cols || !t_out) return fail(ctx, TRANSEC_EINVAL, "NULL item or output array");
  DeviceGuard dg(ctx->device);
  int rc = begin_call(ctx);
  if (rc) return rc;
  std::vector<int> hik(nitems), hic(nitems);
  if (on_device) {
    CK(cudaMemcpyAsync(hik.data(), ik, nitems * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaMemcpyAsync(hic.data(), ictx, nitems * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
  } else {
    hik.assign(ik, ik + nitems);
    hic.assign(ictx, ictx + nitems);
  }
  int H = 0;
  for (int i = 0; i < nitems; ++i) {
    if (hic[i] < 0 || hic[i] >= nctx) return fail(ctx, TRANSEC_EINVAL, "context index out of range");
    const transec_ctx* m = members[hic[i]];
    if (hik[i] < 0 || hik[i] >= m->nk) return fail(ctx, TRANSEC_EINVAL, "k index out of range");
    const bool rp = real_phase(m->kfrac[2 * hik[i]], m->kfrac[2 * hik[i] + 1]);
    const int h = ctx->opts.method == TRANSEC_METHOD_BICG ? 2 : (rp ? 1 : 2);
    if (ctx->opts.method == TRANSEC_METHOD_COCG && !rp)
      return fail(ctx, TRANSEC_EINVAL, "COCG requested for a k-point with complex Bloch phase");
    H = std::max(H, h);
  }
  int worst = TRANSEC_OK;
  if (on_device) {
    DevBuf btm, bit, bst;
    double* dtm = t_minus_out;
    int* dit = iters_out;
    int* dst = status_out;
    if (!dtm) { CK(cudaMalloc(&btm.p, nitems * sizeof(double))); dtm = (double*)btm.p; }
    if (!dit) { CK(cudaMalloc(&bit.p, nitems * sizeof(int))); dit = (int*)bit.p; }
    if (!dst) { CK(cudaMalloc(&bst.p, nitems * sizeof(int))); dst = (int*)bst.p; }
    rc = solve_batch(ctx, members, ictx, H, nitems, energies, ik, (const long long*)cols, t_out,
                     dtm, dit, dst);
    if (rc != TRANSEC_OK) return rc;
    std::vector<int> hs(nitems);
    CK(cudaMemcpyAsync(hs.data(), dst, nitems * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    for (int v : hs)
      if (severity(v) > severity(worst)) worst = v;
  } else {
    std::vector<double> e(energies, energies + nitems);
    std::vector<long long> c(cols, cols + nitems);
    std::vector<double> t, tm;
    std::vector<int> it, st;
    rc = solve_host_items(ctx, members, hic, H, e, hik, c, t, tm, it, st);
    if (rc != TRANSEC_OK && rc != TRANSEC_ENOCONV && rc != TRANSEC_EBREAKDOWN) return rc;
    std::memcpy(t_out, t.data(), nitems * sizeof(double));
    if (t_minus_out) std::memcpy(t_minus_out, tm.data(), nitems * sizeof(double));
    if (iters_out) std::memcpy(iters_out, it.data(), nitems * sizeof(int));
    if (status_out) std::memcpy(status_out, st.data(), nitems * sizeof(int));
    for (int v : st)
      if (severity(v) > severity(worst)) worst = v;
  }
  rc = end_call(ctx);
  if (rc) return rc;
  if (worst != TRANSEC_OK) ctx->err = std::string("some columns failed: ") + transec_status_string(worst);
  return worst;
}

int transec_autotune(transec_ctx* ctx, double energy, int ik, int* tile_y_out, int* slab_out,
                     int* slots_out) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (ik < 0 || ik >= ctx->nk || !std::isfinite(energy)) return fail(ctx, TRANSEC_EINVAL, "bad autotune arguments");
  DeviceGuard dg(ctx->device);
  const transec_solver_opts saved = ctx->opts;
  const int H = halves_for(ctx, ik);
  if (H < 0) return fail(ctx, TRANSEC_EINVAL, "COCG requested for a k-point with complex Bloch phase");
  const bool fp64 = saved.precision == TRANSEC_PREC_FP64;
  const int maxthreads = fp64 ? StencilMax<double>::threads : StencilMax<float>::threads;
  const int tx = std::min(ctx->g.nx, 32);
  const int ylim = std::max(1, std::min(ctx->g.ny, maxthreads / (tx * H)));
  std::vector<int> tys = {0};
  for (int v : {ylim, ylim / 2, 8, 4})
    if (v >= 1 && v <= ylim && std::find(tys.begin(), tys.end(), v) == tys.end()) tys.push_back(v);
  std::vector<int> slabs = {16, 32, 64, 128};
  const long long target = 24LL << 20;
  const int s0 = (int)std::max(1LL, std::min(4096LL, (target + ctx->g.n * H - 1) / (ctx->g.n * H)));
  std::vector<int> slots = {std::max(1, s0 / 2), s0, std::min(4096, 2 * s0)};
  const long long nrhs = (long long)ctx->lplanes.size() * ctx->g.nxy;
  double best = -1.0;
  int by = 0, bs = 0, bS = s0;
  for (int ty : tys)
    for (int sl : slabs)
      for (int S : slots) {
        ctx->opts = saved;
        ctx->opts.tile_y = ty;
        ctx->opts.slab = sl;
        ctx->opts.slots = S;
        ctx->opts.maxit = 32;
        ctx->opts.mixed_maxit = 32;
        ctx->opts.profile = 1;
        ctx->opts.host_loop = 1;
        std::vector<double> e(S, energy);
        std::vector<int> k(S, ik);
        std::vector<long long> c(S);
        for (int u = 0; u < S; ++u) c[u] = (long long)u % std::max(1LL, nrhs);
        std::vector<double> t, tm;
        std::vector<int> it, st;
        transec_stats_reset(ctx);
        rc = begin_call(ctx);
        if (rc == TRANSEC_OK) rc = solve_host_items(ctx, {ctx}, {}, H, e, k, c, t, tm, it, st);
        if (rc == TRANSEC_OK || rc == TRANSEC_ENOCONV || rc == TRANSEC_EBREAKDOWN) rc = end_call(ctx);
        if (rc != TRANSEC_OK) {
          ctx->opts = saved;
          return rc;
        }
        const double ms = ctx->stencil_ms + ctx->stencil32_ms + ctx->update_ms;
        const double rate =
            ms > 0 ? (double)(ctx->point_applies + ctx->point_applies32) / ms : 0.0;
        if (rate > best) {
          best = rate;
          by = ty;
          bs = sl;
          bS = S;
        }
      }
  ctx->opts = saved;
  ctx->opts.tile_y = by;
  ctx->opts.slab = bs;
  ctx->opts.slots = bS;
  transec_stats_reset(ctx);
  if (tile_y_out) *tile_y_out = by;
  if (slab_out) *slab_out = bs;
  if (slots_out) *slots_out = bS;
  return TRANSEC_OK;
}

int transec_transmission(transec_ctx* ctx, int ne, const double* energies, double* T_out,
                         double* T_avg_out, int* status_out, int* iters_out) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (ne < 0 || (ne > 0 && (!energies || !T_out))) return fail(ctx, TRANSEC_EINVAL, "bad energies/T_out");
  if (ne == 0) return TRANSEC_OK;
  for (int e = 0; e < ne; ++e)
    if (!std::isfinite(energies[e])) return fail(ctx, TRANSEC_EINVAL, "non-finite energy");
  DeviceGuard dg(ctx->device);
  rc = begin_call(ctx);
  if (rc) return rc;
  const int nk = ctx->nk;
  const long long nrhs = (long long)ctx->lplanes.size() * ctx->g.nxy;
  // representative k-points: with BiCG a k whose mirror was already chosen is read
  // from that mirror's shadow columns (A(E, -k) = A(E, k)^T)
  std::vector<int> H(nk), rep(nk, -1), from_shadow(nk, 0);
  for (int k = 0; k < nk; ++k) {
    H[k] = halves_for(ctx, k);
    if (H[k] < 0) return fail(ctx, TRANSEC_EINVAL, "COCG requested for a k-point with complex Bloch phase");
  }
  for (int k = 0; k < nk; ++k) {
    if (rep[k] >= 0) continue;
    rep[k] = k;
    if (H[k] == 2) {
      const int p = partner_of(ctx, k);
      if (p > k && rep[p] < 0) { rep[p] = k; from_shadow[p] = 1; }
    }
  }
  std::vector<double> T((size_t)ne * nk, 0.0);
  std::vector<int> St((size_t)ne * nk, TRANSEC_OK), It((size_t)ne * nk, 0);
  // process per halves group, in batches of (E, k) pairs
  const long long max_items = 1LL << 22;
  for (int hgrp = 1; hgrp <= 2; ++hgrp) {
    std::vector<std::pair<int, int>> pairs;  // (e, k representative)
    for (int e = 0; e < ne; ++e)
      for (int k = 0; k < nk; ++k)
        if (rep[k] == k && H[k] == hgrp) pairs.push_back({e, k});
    const long long per_batch = std::max(1LL, max_items / std::max(1LL, nrhs));
    for (size_t b0 = 0; b0 < pairs.size(); b0 += per_batch) {
      const size_t b1 = std::min(pairs.size(), (size_t)(b0 + per_batch));
      std::vector<double> ie;
      std::vector<int> ik;
      std::vector<long long> ic;
      for (size_t pi = b0; pi < b1; ++pi)
        for (long long c = 0; c < nrhs; ++c) {
          ie.push_back(energies[pairs[pi].first]);
          ik.push_back(pairs[pi].second);
          ic.push_back(c);
        }
      std::vector<double> t, tm;
      std::vector<int> it, st;
      rc = solve_host_items(ctx, {ctx}, {}, hgrp, ie, ik, ic, t, tm, it, st);
      if (rc != TRANSEC_OK && rc != TRANSEC_ENOCONV && rc != TRANSEC_EBREAKDOWN) return rc;
      size_t u = 0;
      for (size_t pi = b0; pi < b1; ++pi) {
        const int e = pairs[pi].first, k = pairs[pi].second;
        int partner = -1;
        for (int kk = 0; kk < nk; ++kk)
          if (kk != k && rep[kk] == k && from_shadow[kk]) partner = kk;
        double sum = 0.0, sum_m = 0.0;
        int worst = TRANSEC_OK, itmax = 0;
        for (long long c = 0; c < nrhs; ++c, ++u) {
          sum += t[u];
          sum_m += tm[u];
          if (severity(st[u]) > severity(worst)) worst = st[u];
          itmax = std::max(itmax, it[u]);
        }
        const double nan = std::nan("");
        T[(size_t)e * nk + k] = worst == TRANSEC_OK ? sum : nan;
        St[(size_t)e * nk + k] = worst;
        It[(size_t)e * nk + k] = itmax;
        if (partner >= 0) {
          T[(size_t)e * nk + partner] = worst == TRANSEC_OK ? sum_m : nan;
          St[(size_t)e * nk + partner] = worst;
          It[(size_t)e * nk + partner] = itmax;
        }
      }
    }
  }
  rc = end_call(ctx);
  if (rc) return rc;
  int worst = TRANSEC_OK;
  for (int e = 0; e < ne; ++e) {
    double avg = 0.0;
    for (int k = 0; k < nk; ++k) {
      const size_t i = (size_t)e * nk + k;
      T_out[i] = T[i];
      if (status_out) status_out[i] = St[i];
      if (iters_out) iters_out[i] = It[i];
      if (severity(St[i]) > severity(worst)) worst = St[i];
      avg += ctx->kw[k] * T[i];
    }
    if (T_avg_out) T_avg_out[e] = avg;
  }
  if (worst != TRANSEC_OK) ctx->err = std::string("some (E, k) failed: ") + transec_status_string(worst);
  return worst;
}

int transec_apply(transec_ctx* ctx, double energy, int ik, int conj_k, int nvec, const double* x,
                  double* y, int on_device) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (nvec < 0 || ik < 0 || ik >= ctx->nk || !std::isfinite(energy))
    return fail(ctx, TRANSEC_EINVAL, "bad apply arguments");
  if (nvec == 0) return TRANSEC_OK;
  if (!x || !y) return fail(ctx, TRANSEC_EINVAL, "NULL vector");
  DeviceGuard dg(ctx->device);
  rc = begin_call(ctx);
  if (rc) return rc;
  const long long n = ctx->g.n;
  const size_t bytes = (size_t)nvec * n * sizeof(double2);
  DevBuf bx, by, bp, bpart, bslot;
  const double2* dx = (const double2*)x;
  double2* dy = (double2*)y;
  if (!on_device) {
    CK(cudaMalloc(&bx.p, bytes));
    CK(cudaMalloc(&by.p, bytes));
    CK(cudaMemcpyAsync(bx.p, x, bytes, cudaMemcpyHostToDevice, ctx->s));
    dx = (const double2*)bx.p;
    dy = (double2*)by.p;
  }
  const TileShape ts = choose_tiles(ctx->g, 1, sizeof(double2), StencilMax<double>::threads,
                                    ctx->opts.tile_y, ctx->opts.slab);
  CK(prepare_stencil<double>(ctx->g.R, ts.smem));
  CK(cudaMalloc(&bp.p, bytes));
  CK(cudaMalloc(&bpart.p, (size_t)nvec * ts.ntx * ts.nty * ts.nslab * 2 * sizeof(double)));
  std::vector<Slot> hs(nvec);
  for (int v = 0; v < nvec; ++v) {
    hs[v] = Slot{};
    hs[v].status = SLOT_ACTIVE;
    hs[v].ik = ik;
    hs[v].e = energy;
    hs[v].beta = make_double2(0.0, 0.0);
  }
  CK(cudaMalloc(&bslot.p, nvec * sizeof(Slot)));
  CK(cudaMemcpyAsync(bslot.p, hs.data(), nvec * sizeof(Slot), cudaMemcpyHostToDevice, ctx->s));
  StencilArgs<double> sa{};
  sa.r = dx; sa.p_in = dx; sa.p_out = (double2*)bp.p; sa.q = dy; sa.part = (double*)bpart.p;
  sa.slots = (const Slot*)bslot.p; sa.phase = ctx->d_phase; sa.v = ctx->d_v; sa.gam = ctx->d_gam;
  sa.g = ctx->g; sa.H = 1; sa.TX = ts.TX; sa.TY = ts.TY; sa.D = ts.D; sa.ntx = ts.ntx;
  sa.conj = conj_k ? 1 : 0; sa.slot_stride = n;
  launch_stencil<double>(ctx->g.R, dim3(ts.ntx * ts.nty, ts.nslab, nvec), ts.threads, ts.smem, ctx->s, sa);
  CHECK_LAUNCH();
  if (!on_device) CK(cudaMemcpyAsync(y, by.p, bytes, cudaMemcpyDeviceToHost, ctx->s));
  return end_call(ctx);
}

int transec_trace(transec_ctx* ctx, int nvec, const double* x, const int64_t* cols, double* t_out,
                  int on_device) {
  if (!ctx) return TRANSEC_EINVAL;
  if (!ctx->have_abc) return fail(ctx, TRANSEC_ESTATE, "absorbing boundary not set");
  if (nvec < 0) return fail(ctx, TRANSEC_EINVAL, "nvec < 0");
  if (nvec == 0) return TRANSEC_OK;
  if (!x || !cols || !t_out) return fail(ctx, TRANSEC_EINVAL, "NULL argument");
  DeviceGuard dg(ctx->device);
  int rc = begin_call(ctx);
  if (rc) return rc;
  const long long n = ctx->g.n;
  DevBuf bx, bc, bt;
  const double2* dx = (const double2*)x;
  const long long* dc = (const long long*)cols;
  double* dt = t_out;
  if (!on_device) {
    const size_t bytes = (size_t)nvec * n * sizeof(double2);
    CK(cudaMalloc(&bx.p, bytes));
    CK(cudaMalloc(&bc.p, nvec * sizeof(long long)));
    CK(cudaMalloc(&bt.p, nvec * sizeof(double)));
    CK(cudaMemcpyAsync(bx.p, x, bytes, cudaMemcpyHostToDevice, ctx->s));
    CK(cudaMemcpyAsync(bc.p, cols, nvec * sizeof(long long), cudaMemcpyHostToDevice, ctx->s));
    dx = (const double2*)bx.p;
    dc = (const long long*)bc.p;
    dt = (double*)bt.p;
  }
  VecTraceArgs va{};
  va.x = dx; va.cols = dc; va.lplanes = ctx->d_lplanes; va.rplanes = ctx->d_rplanes;
  va.nlp = (int)ctx->lplanes.size(); va.nrp = (int)ctx->rplanes.size(); va.gl = ctx->d_gl;
  va.gr = ctx->d_gr; va.t_out = dt; va.nxy = ctx->g.nxy; va.n = n;
  k_vec_trace<<<nvec, 256, 0, ctx->s>>>(va);
  CHECK_LAUNCH();
  if (!on_device) CK(cudaMemcpyAsync(t_out, bt.p, nvec * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  return end_call(ctx);
}

int transec_stats(const transec_ctx* ctx, long long* launches, long long* point_applies,
                  double* stencil_ms, long long* stencil_launches, double* update_ms,
                  long long* update_launches, long long* fallbacks, long long* point_applies32,
                  double* stencil32_ms, long long* stencil32_launches) {
  if (!ctx) return TRANSEC_EINVAL;
  if (fallbacks) *fallbacks = ctx->fallbacks;
  if (point_applies32) *point_applies32 = ctx->point_applies32;
  if (stencil32_ms) *stencil32_ms = ctx->stencil32_ms;
  if (stencil32_launches) *stencil32_launches = ctx->stencil32_launches;
  if (launches) *launches = ctx->launches;
  if (point_applies) *point_applies = ctx->point_applies;
  if (stencil_ms) *stencil_ms = ctx->stencil_ms;
  if (stencil_launches) *stencil_launches = ctx->stencil_launches;
  if (update_ms) *update_ms = ctx->update_ms;
  if (update_launches) *update_launches = ctx->update_launches;
  return TRANSEC_OK;
}

int transec_stats_reset(transec_ctx* ctx) {
  if (!ctx) return TRANSEC_EINVAL;
  ctx->launches = 0;
  ctx->point_applies = 0;
  ctx->stencil_ms = ctx->update_ms = 0;
  ctx->stencil_launches = ctx->update_launches = 0;
  ctx->fallbacks = 0;
  ctx->stencil32_ms = 0;
  ctx->stencil32_launches = ctx->point_applies32 = 0;
  ctx->sweep_iters = ctx->sweep_shift_points = 0;
  ctx->sweep_stencil_ms = ctx->sweep_shift_ms = ctx->sweep_update_ms = ctx->sweep_reduce_ms = 0;
  ctx->sweep_stencil_launches = ctx->sweep_shift_launches = 0;
  ctx->sweep_fp64_redone = 0;
  ctx->sweep_guard_redone = 0;
  ctx->eig_gram_ms = 0;
  ctx->eig_sum_ms = 0;
  ctx->sweep_stencil_df_ms = ctx->sweep_shift_df_ms = 0;
  ctx->sweep_stencil_df_launches = ctx->sweep_shift_df_launches = 0;
  return TRANSEC_OK;
}

int transec_sweep_stats(const transec_ctx* ctx, long long* iters, long long* shift_points,
                        double* stencil_ms, long long* stencil_launches, double* shift_ms,
                        long long* shift_launches, double* stencil_df_ms, long long* stencil_df_launches,
                        double* shift_df_ms, long long* shift_df_launches, double* reduce_ms,
                        long long* fp64_redone, long long* guard_redone) {
  if (!ctx) return TRANSEC_EINVAL;
  if (guard_redone) *guard_redone = ctx->sweep_guard_redone;
  if (stencil_df_ms) *stencil_df_ms = ctx->sweep_stencil_df_ms;
  if (stencil_df_launches) *stencil_df_launches = ctx->sweep_stencil_df_launches;
  if (shift_df_ms) *shift_df_ms = ctx->sweep_shift_df_ms;
  if (shift_df_launches) *shift_df_launches = ctx->sweep_shift_df_launches;
  if (fp64_redone) *fp64_redone = ctx->sweep_fp64_redone;
  if (iters) *iters = ctx->sweep_iters;
  if (shift_points) *shift_points = ctx->sweep_shift_points;
  if (stencil_ms) *stencil_ms = ctx->sweep_stencil_ms;
  if (stencil_launches) *stencil_launches = ctx->sweep_stencil_launches;
  if (shift_ms) *shift_ms = ctx->sweep_shift_ms;
  if (shift_launches) *shift_launches = ctx->sweep_shift_launches;
  if (reduce_ms) *reduce_ms = ctx->sweep_reduce_ms;
  return TRANSEC_OK;
}

const char* transec_last_error(const transec_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

void transec_destroy(transec_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard dg(ctx->device);
  if (ctx->s) cudaStreamSynchronize(ctx->s);
  transec::sweep_release(ctx);
  ctx->e64.release();
  ctx->e32.release();
  cudaFree(ctx->mx_x); cudaFree(ctx->mx_q); cudaFree(ctx->mx_p);
  cudaFree(ctx->mx_sig); cudaFree(ctx->mx_part); cudaFree(ctx->mx_slots);
  cudaFree(ctx->d_insts);
  cudaFree(ctx->d_v); cudaFree(ctx->d_v32);
  cudaFree(ctx->d_gl); cudaFree(ctx->d_gr); cudaFree(ctx->d_gam);
  cudaFree(ctx->d_lplanes); cudaFree(ctx->d_rplanes); cudaFree(ctx->d_phase);
  cudaFree(ctx->d_gam32); cudaFree(ctx->d_phase32);
  if (ctx->h_harvest) cudaFreeHost(ctx->h_harvest);
  for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  if (ctx->s) cudaStreamDestroy(ctx->s);
  cudaGetLastError();
  delete ctx;
}

}  // extern "C"
