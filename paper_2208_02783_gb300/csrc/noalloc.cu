// transec_apply_noalloc: the operator apply without any device allocation.
//
// Some callers cannot let a library call cudaMalloc or cudaFree: a serving process
// whose device memory is owned and budgeted by another allocator (a framework's
// caching allocator), or a latency-critical loop where cudaFree's implicit device
// synchronisation (and cudaMalloc's unpredictable latency) cannot be tolerated.  For
// them this entry point runs the same stencil kernel as transec_apply, with the
// kernel's scratch -- the p-buffer written by the fused p <- r + beta p update, the
// per-block partial sums and the per-vector solver state -- placed in one file-scope
// static device array instead of memory allocated per call.
//
// The array is part of the library image, so every GPU that loads the library holds
// it (kNoAllocScratchBytes, about 17 MiB) until the process exits.  It is shared by all
// calls and keeps the last call's contents: everything the kernel reads from it is
// written earlier in the same call, and calls that overlap on the GPU race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "engine.cuh"

namespace transec {
template <typename T>
cudaError_t prepare_stencil(int R, size_t smem);
}

namespace {

using transec::Slot;

// Largest workload one call may pass: nvec * nx * ny * nz complex values in the
// p-scratch, at most kNoAllocMaxVec vectors, and their partial sums in kPartBytes.
constexpr long long kNoAllocMaxPoints = 1LL << 20;  // 16 MiB of double2
constexpr int kNoAllocMaxVec = 64;
constexpr size_t kPBytes = (size_t)kNoAllocMaxPoints * sizeof(double2);
constexpr size_t kPartBytes = (size_t)1 << 20;
constexpr size_t kSlotBytes = ((kNoAllocMaxVec * sizeof(Slot) + 255) / 256) * 256;
constexpr size_t kNoAllocScratchBytes = kPBytes + kPartBytes + kSlotBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on `device` (which must be current).  The
// name g_noalloc_scratch in host code is only a stand-in for the symbol, so the
// address is looked up once per device and cached.
cudaError_t scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

// Per-vector state for the apply: active, energy, k index, beta = 0 (so the fused
// update leaves p = x).
__global__ void k_noalloc_slots(Slot* slots, int nvec, double energy, int ik) {
  const int v = threadIdx.x;
  if (v >= nvec) return;
  Slot s{};
  s.status = transec::SLOT_ACTIVE;
  s.item = v;
  s.ik = ik;
  s.e = energy;
  s.beta = make_double2(0.0, 0.0);
  s.rho = make_double2(1.0, 0.0);
  slots[v] = s;
}

struct Guard {
  int prev = -1;
  explicit Guard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(d);
  }
  ~Guard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int fail(transec_ctx* ctx, int code, const std::string& msg) {
  ctx->err = msg;
  return code;
}

int cuda_fail(transec_ctx* ctx, const char* what, cudaError_t e) {
  cudaGetLastError();
  return fail(ctx, TRANSEC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" int transec_apply_noalloc(transec_ctx* ctx, double energy, int ik, int conj_k,
                                     int nvec, const double* x, double* y) {
  using namespace transec;
  if (!ctx) return TRANSEC_EINVAL;
  if (!ctx->have_v || !ctx->have_abc || !ctx->have_k)
    return fail(ctx, TRANSEC_ESTATE, "potential, absorbing boundary and k-mesh must be set first");
  if (nvec < 0 || ik < 0 || ik >= ctx->nk || !std::isfinite(energy))
    return fail(ctx, TRANSEC_EINVAL, "bad apply arguments");
  if (nvec == 0) return TRANSEC_OK;
  if (!x || !y) return fail(ctx, TRANSEC_EINVAL, "NULL vector");
  if (nvec > kNoAllocMaxVec)
    return fail(ctx, TRANSEC_EINVAL,
                "transec_apply_noalloc: nvec exceeds the fixed scratch limit of 64 vectors");
  if ((long long)nvec * ctx->g.n > kNoAllocMaxPoints)
    return fail(ctx, TRANSEC_EINVAL,
                "transec_apply_noalloc: nvec * nx * ny * nz exceeds the fixed scratch limit of "
                "1048576 complex values");
  const TileShape ts = choose_tiles(ctx->g, 1, sizeof(double2), StencilMax<double>::threads,
                                    ctx->opts.tile_y, ctx->opts.slab);
  const long long nblk = (long long)ts.ntx * ts.nty * ts.nslab;
  if ((size_t)nvec * nblk * 2 * sizeof(double) > kPartBytes)
    return fail(ctx, TRANSEC_EINVAL,
                "transec_apply_noalloc: too many stencil blocks for the fixed partial-sum scratch");
  Guard guard(ctx->device);
  void* base = nullptr;
  cudaError_t e = scratch_address(ctx->device, &base);
  if (e != cudaSuccess) return cuda_fail(ctx, "cudaGetSymbolAddress", e);
  double2* p_scratch = reinterpret_cast<double2*>(base);
  double* part = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kPBytes);
  Slot* slots = reinterpret_cast<Slot*>(static_cast<unsigned char*>(base) + kPBytes + kPartBytes);

  e = prepare_stencil<double>(ctx->g.R, ts.smem);
  if (e != cudaSuccess) return cuda_fail(ctx, "stencil set-up", e);
  e = cudaEventRecord(ctx->ev_in, ctx->user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s, ctx->ev_in, 0);
  if (e != cudaSuccess) return cuda_fail(ctx, "stream ordering", e);

  k_noalloc_slots<<<1, kNoAllocMaxVec, 0, ctx->s>>>(slots, nvec, energy, ik);
  StencilArgs<double> sa{};
  sa.r = reinterpret_cast<const double2*>(x);
  sa.p_in = reinterpret_cast<const double2*>(x);
  sa.p_out = p_scratch;
  sa.q = reinterpret_cast<double2*>(y);
  sa.part = part;
  sa.slots = slots;
  sa.phase = ctx->d_phase;
  sa.v = ctx->d_v;
  sa.gam = ctx->d_gam;
  sa.g = ctx->g;
  sa.H = 1;
  sa.TX = ts.TX;
  sa.TY = ts.TY;
  sa.D = ts.D;
  sa.ntx = ts.ntx;
  sa.conj = conj_k ? 1 : 0;
  sa.slot_stride = ctx->g.n;
  launch_stencil<double>(ctx->g.R, dim3(ts.ntx * ts.nty, ts.nslab, nvec), ts.threads, ts.smem,
                         ctx->s, sa);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, "kernel launch", e);
  e = cudaEventRecord(ctx->ev_out, ctx->s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->user, ctx->ev_out, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->s);
  if (e != cudaSuccess) return cuda_fail(ctx, "apply", e);
  return TRANSEC_OK;
}
