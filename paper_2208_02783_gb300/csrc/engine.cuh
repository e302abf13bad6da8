// Host-side declarations shared by the C ABI and the solver engines.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/transec.h"
#include "kernels.cuh"

struct transec_ctx;

namespace transec {

// Device buffers of the multi-shift engine (sweep.cu), kept between calls.
struct SweepBufs;
void sweep_release(transec_ctx* ctx);

// Device buffers and launch shape of one slot engine (one arithmetic type T, one
// number of halves H).  Buffers are kept between calls and grown on demand.
template <typename T>
struct Engine {
  using CT = typename Cx<T>::type;
  int S = 0, H = 0;
  long long n = 0;
  CT* X = nullptr;
  CT* R = nullptr;
  CT* P0 = nullptr;
  CT* P1 = nullptr;
  CT* Q = nullptr;
  double* sig_part = nullptr;
  double* rho_part = nullptr;
  Slot* slots = nullptr;
  Queue* queue = nullptr;
  // stencil launch shape
  int TX = 0, TY = 0, D = 0, ntx = 0, nty = 0, nslab = 0, threads = 0;
  size_t smem = 0;
  int nblk2 = 0, nblk3 = 0;
  void release();
};

TileShape choose_tiles(const Geometry& g, int H, int elem_bytes, int max_threads, int tile_y,
                       int slab);

template <typename T>
void launch_stencil(int R, dim3 grid, int threads, size_t smem, cudaStream_t s,
                    const StencilArgs<T>& a);

}  // namespace transec

// The context behind the opaque C handle.
struct transec_ctx {
  int device = 0;
  cudaStream_t user = nullptr;  // caller's stream (may be the legacy default stream)
  cudaStream_t s = nullptr;     // the context's own stream (graph capture happens here)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  transec::Geometry g{};
  int order = 0;
  double hx = 0, hy = 0, hz = 0;
  // operator data
  double* d_v = nullptr;
  float* d_v32 = nullptr;
  bool have_v = false;
  // max |V(x, y, z) - V(-x, -y, z)| / max |V| over the cell (in-plane inversion about
  // grid point (0, 0), coordinates taken modulo the cell); NaN before a potential is set
  double v_inversion_gap = __builtin_nan("");
  std::vector<double> gl, gr;
  double* d_gl = nullptr;
  double* d_gr = nullptr;
  double* d_gam = nullptr;
  float* d_gam32 = nullptr;
  int* d_lplanes = nullptr;
  int* d_rplanes = nullptr;
  std::vector<int> lplanes, rplanes;
  bool have_abc = false;
  int nk = 0;
  std::vector<double> kfrac, kw;
  double2* d_phase = nullptr;
  float2* d_phase32 = nullptr;
  bool have_k = false;
  transec_solver_opts opts{};
  std::string err;
  // solver engines
  transec::Engine<double> e64;
  transec::Engine<float> e32;
  // mixed precision extra state: FP64 solution, FP64 A*x and the stencil's p copy per
  // slot and half, their partial sums, and the slot array of the replacement pass
  double2* mx_x = nullptr;
  double2* mx_q = nullptr;
  double2* mx_p = nullptr;
  double* mx_sig = nullptr;
  double* mx_part = nullptr;
  transec::Slot* mx_slots = nullptr;
  long long mx_elems = 0;
  long long mx_sig_elems = 0;
  long long mx_part_elems = 0;
  int mx_S = 0;
  // operator table of the last solve (one entry, or one per member of a batch)
  transec::Inst* d_insts = nullptr;
  int insts_cap = 0;
  // pinned host word for the harvested counter
  int* h_harvest = nullptr;
  // counters since the last transec_stats_reset
  long long launches = 0;
  long long point_applies = 0;
  double stencil_ms = 0, update_ms = 0;
  long long stencil_launches = 0, update_launches = 0;
  long long fallbacks = 0;  // mixed-precision columns re-solved in FP64
  // the same for the FP32 kernels of the mixed form (the FP64 fields then hold the
  // residual replacements' and fallbacks' FP64 work only)
  double stencil32_ms = 0;
  long long stencil32_launches = 0, point_applies32 = 0;
  std::vector<cudaEvent_t> prof_ev;  // 4 per iteration of a chunk when profiling
  transec::SweepBufs* sweep = nullptr;  // multi-shift engine buffers (sweep.cu)
  // multi-shift engine counters since the last transec_stats_reset: seed iterations
  // summed over runs, per-shift point updates, and event-timed kernel ms (profile)
  long long sweep_iters = 0, sweep_shift_points = 0;
  double sweep_stencil_ms = 0, sweep_shift_ms = 0, sweep_update_ms = 0, sweep_reduce_ms = 0;
  long long sweep_stencil_launches = 0, sweep_shift_launches = 0;
  long long sweep_fp64_redone = 0;  // double-float results solved again in FP64
  long long sweep_guard_redone = 0;  // sketch results computed again with a larger sketch
  double eig_gram_ms = 0, eig_sum_ms = 0;  // eigen route (profile): Gram matrices, eigen-sums
  double sweep_stencil_df_ms = 0, sweep_shift_df_ms = 0;  // the double-float runs' kernels
  long long sweep_stencil_df_launches = 0, sweep_shift_df_launches = 0;
};
