// Shared device-side types of the transmission library.
//
// Complex values are stored interleaved (re, im) as double2 / float2.  Vectors of a
// slot block are laid out [slot][half][point], point = i + nx*(j + ny*l): one
// contiguous complex vector per (slot, half), so a converged slot can be retired and
// refilled without touching the others.  half 0 carries +k, half 1 the shadow (-k)
// system of the transpose BiCG; COCG slots have one half.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace transec {

constexpr int kMaxR = 6;     // order 12 stencil reaches 6 neighbours per side
constexpr int kPhaseW = 8;   // Bloch phase table covers wrap counts -8..8 (any nx >= 1 at order <= 12)
constexpr int kPhaseN = 2 * kPhaseW + 1;

template <typename T> struct Cx;
template <> struct Cx<double> { using type = double2; };
template <> struct Cx<float> { using type = float2; };

// Slot life cycle: IDLE -> (assign) ACTIVE -> (converged / failed) DONE -> (trace) IDLE
enum SlotStatus : int { SLOT_IDLE = 0, SLOT_ACTIVE = 1, SLOT_DONE = 2 };

// Grid and operator constants shared by every kernel of a context.
struct Geometry {
  int nx, ny, nz, R;
  long long nxy, n;
  double kx[kMaxR + 1], ky[kMaxR + 1], kz[kMaxR + 1];  // c_m / (2 h^2), m = 1..R
  double diag_c;  // c_0/2 * (1/hx^2 + 1/hy^2 + 1/hz^2)
};

// Launch shape of the stencil for one geometry.
struct TileShape {
  int TX, TY, D, ntx, nty, nslab, threads;
  size_t smem;
};

// One operator of a solve: geometry, its device arrays and the stencil's launch
// shapes (tile[0] for the FP64 kernel, tile[1] for the FP32 one).  A batch of
// operators of different sizes shares one slot engine through a table of these.
struct Inst {
  Geometry g;
  const double* v;
  const float* v32;
  const double* gam;     // Gamma_L + Gamma_R per plane
  const double* gl;      // Gamma_L per plane
  const double* gr;      // Gamma_R per plane
  const double2* phase;  // [nk][2][2][kPhaseN]
  const int* lplanes;    // planes with Gamma_L > 0
  const int* rplanes;    // planes with Gamma_R > 0
  int nlp, nrp, nk, pad;
  TileShape tile[2];
  const float* gam32;    // FP32 copies for the FP32 stencil (no conversions per point)
  const float2* phase32;
};

// Per-slot solver state (device resident).
struct Slot {
  int status;     // SlotStatus
  int item;       // work item being solved, -1 when idle
  int it;         // operator applications so far (per half)
  int result;     // per-item status code once DONE (0 = converged)
  int ik;         // k-point index
  int init;       // set by assign when the vectors must be (re)initialised
  int inst;       // operator (index into the Inst table) of the item
  int pad0;
  long long j;    // grid index of the right-hand side e_j
  double e;       // energy (Hartree)
  double2 rho;    // <r, r> in the pairing form
  double2 beta;   // p <- r + beta p
  double res;     // last residual norm (max over halves)
  int refresh;    // mixed precision: number of FP64 residual replacements
  int pending;    // mixed precision: a residual replacement is requested
  double rmax;    // mixed precision: true residual norm at the last replacement
  int last_ref;   // mixed precision: iteration of the last replacement
  int it_best;    // mixed precision: iteration of the smallest residual of this cycle
  double rbest;   // mixed precision: smallest FP32 residual of this cycle
};

// Work queue bookkeeping (device resident).
struct Queue {
  int next;       // next unassigned item
  int harvested;  // items whose result has been written
  int nitems;
  int chunks;     // chunks run so far (device-side loop)
  int limit;      // the device-side loop stops at this chunk count
  int pad[3];
};

// --- small complex helpers -------------------------------------------------------
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cdiv(double2 a, double2 b) {
  // Smith's algorithm keeps the scaling safe for wide exponent ranges.
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  } else {
    double r = b.x / b.y, d = b.x * r + b.y;
    return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
}
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

template <typename CT> __host__ __device__ inline CT czero();
template <> __host__ __device__ inline double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __host__ __device__ inline float2 czero<float2>() { return make_float2(0.f, 0.f); }

template <typename CT> __host__ __device__ inline CT cfrom(double2 a);
template <> __host__ __device__ inline double2 cfrom<double2>(double2 a) { return a; }
template <> __host__ __device__ inline float2 cfrom<float2>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}

}  // namespace transec
