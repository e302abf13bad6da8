// CUDA kernels of the transmission hot path (sm_103a).
//
//   k_stencil   Bloch-phased stencil apply fused with the Krylov pre-update:
//               p <- r + beta p, q <- A(E, +-k) p, sigma += <p, q> (pairing form)
//   k_update    x += alpha p, r -= alpha q, rho' = <r, r>, ||r_h||^2 per half
//   k_scalars   per slot: reduce the partial sums, convergence, beta = rho'/rho
//   k_trace     t_j = 4 Gamma_L(j) sum_i Gamma_R(i) |x_j(i)|^2 for finished slots
//   k_assign    hand queued (E, k, column) items to idle slots
//   k_init      x = 0, r = e_j, p = 0 for newly assigned slots
//
// The operator (paper Sec. II.A, Eqs. Bloch and H_k) is
//   A(E, k) p = (E - V + c_0/2 sum_a h_a^-2 + i Gamma) p
//             + sum_a sum_{m=1..R} c_m/(2 h_a^2) (p(n + m e_a) + p(n - m e_a)),
// a lateral neighbour that leaves the cell re-entering on the other side with the
// Bloch factor exp(2 pi i kappa_a w) (w = wrap count), z-neighbours outside the grid
// being zero.  half 1 of a transpose-BiCG slot applies A(E, -k) = A(E, k)^T, i.e.
// the conjugate phases (Sec. II.B, H_{-k} = H_k^*).
//
// Reductions are deterministic: every block writes one partial per quantity and
// the consumer sums the partials in a fixed order.
#pragma once

#include "common.cuh"

namespace transec {

// ---------------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------------

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of NV doubles per thread; the result is valid in thread 0.
template <int NV>
__device__ inline void block_sum(double (&v)[NV], double (*red)[32]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[k][wid] = v[k];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = lane < nw ? red[k][lane] : 0.0;
      v[k] = warp_sum(s);
    }
  }
}

__device__ inline int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Per-thread accumulator of a complex bilinear form sum_i a_i b_i (no conjugate).
// FP64: plain FP64 sums.  FP32: the compensated dot product of Ogita, Rump & Oishi
// ("Accurate sum and dot product", SIAM J. Sci. Comput. 2005, algorithm Dot2): each
// product is split exactly into p + e with an FMA, p is added with an error-free
// TwoSum, and the rounding errors are gathered in a second float, so the result is as
// accurate as a dot product computed in twice the working precision.  The bilinear
// forms of COCG/BiCG cancel heavily for oscillatory vectors, which plain FP32 sums
// do not survive.  The _rn intrinsics keep the compiler from contracting the
// error-free transformations.
template <typename T> struct DotAcc;

template <> struct DotAcc<double> {
  double re = 0.0, im = 0.0;
  __device__ inline void add(double2 a, double2 b) {
    re += a.x * b.x - a.y * b.y;
    im += a.x * b.y + a.y * b.x;
  }
  __device__ inline double2 value() const { return make_double2(re, im); }
};

template <> struct DotAcc<float> {
  float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
  __device__ static inline void acc(float& s, float& c, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float e = __fmaf_rn(x, y, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(q, e));
  }
  __device__ inline void add(float2 a, float2 b) {
    acc(sr, cr, a.x, b.x);
    acc(sr, cr, -a.y, b.y);
    acc(si, ci, a.x, b.y);
    acc(si, ci, a.y, b.x);
  }
  __device__ inline double2 value() const {
    return make_double2((double)sr + (double)cr, (double)si + (double)ci);
  }
};

// ---------------------------------------------------------------------------------
// stencil apply fused with p <- r + beta p
// ---------------------------------------------------------------------------------

template <typename T>
struct StencilArgs {
  using CT = typename Cx<T>::type;
  const CT* r;          // [slot][half][n]
  const CT* p_in;       // previous search direction
  CT* p_out;            // p_in + beta... written as r + beta p_in
  CT* q;                // A p_out
  double* part;         // [slot][nblk][2] partial sums of <p, A p>
  const Slot* slots;
  const double2* phase; // [nk][2 (sign of k)][2 (axis)][kPhaseN]
  const T* v;           // potential in the arithmetic type
  const double* gam;    // Gamma_L + Gamma_R per plane
  Geometry g;
  int H, TX, TY, D, ntx;
  int conj;             // 1: swap the phase tables (apply A^T to half 0)
  long long slot_stride;  // H * n (the largest n of a batch)
  // batch mode: when insts is set, each slot's operator, arrays and launch shape
  // come from insts[slot.inst] (tile[tile_idx]) instead of the fields above; blocks
  // past that operator's tiles or slabs only write zero partial sums
  const Inst* insts;
  int tile_idx;
};

template <typename T> __device__ inline const T* inst_potential(const Inst& in);
template <> __device__ inline const double* inst_potential<double>(const Inst& in) { return in.v; }
template <> __device__ inline const float* inst_potential<float>(const Inst& in) { return in.v32; }
// Gamma profile and Bloch phase table in the arithmetic type of the kernel
template <typename T> __device__ inline const T* inst_gamma(const Inst& in);
template <> __device__ inline const double* inst_gamma<double>(const Inst& in) { return in.gam; }
template <> __device__ inline const float* inst_gamma<float>(const Inst& in) { return in.gam32; }
template <typename T> __device__ inline const typename Cx<T>::type* inst_phase(const Inst& in);
template <> __device__ inline const double2* inst_phase<double>(const Inst& in) { return in.phase; }
template <> __device__ inline const float2* inst_phase<float>(const Inst& in) { return in.phase32; }
// argument-mode tables (the stand-alone apply paths run in FP64 only)
template <typename T> __device__ inline const T* args_gamma(const double* g);
template <> __device__ inline const double* args_gamma<double>(const double* g) { return g; }
template <> __device__ inline const float* args_gamma<float>(const double*) { return nullptr; }
template <typename T> __device__ inline const typename Cx<T>::type* args_phase(const double2* p);
template <> __device__ inline const double2* args_phase<double>(const double2* p) { return p; }
template <> __device__ inline const float2* args_phase<float>(const double2*) { return nullptr; }

// Block = TX*TY*H threads (rounded up to whole warps), one grid point (x, y) per thread and half, marching over
// the z-slab [z0, z0 + D) with a register queue of the 2R+1 planes around the
// centre plane; the centre plane (plus lateral halos, Bloch-phased when wrapped)
// sits in shared memory for the x/y neighbours.  Grid = (tiles, slabs, slots).
// Threads per stencil block: FP64 keeps the 13-plane queue in 128 registers (one
// block per SM); FP32 is held to 64 registers so that two blocks share an SM, since
// the HBM-bound FP32 kernel needs the warps to cover its per-plane loads.
template <typename T> struct StencilMax { static constexpr int threads = 512, blocks = 2; };
template <> struct StencilMax<double> { static constexpr int threads = 448, blocks = 1; };

template <typename T, int R>
__global__ void __launch_bounds__(StencilMax<T>::threads, StencilMax<T>::blocks)
    k_stencil(const StencilArgs<T> a) {
  using CT = typename Cx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[2][32];
  CT* sm = reinterpret_cast<CT*>(smem_raw);

  const int slot = blockIdx.z;
  const Slot* stp = a.slots + slot;
  if (stp->status != SLOT_ACTIVE) return;  // uniform over the block
  const double2 beta_d = stp->beta;
  const double e = stp->e;
  const int ik = stp->ik;

  // operator and launch shape: kernel arguments, or the slot's batch entry
  const Geometry* gp = &a.g;
  const T* vp = a.v;
  const T* gamp = args_gamma<T>(a.gam);
  const CT* phase = args_phase<T>(a.phase);
  int TX = a.TX, TY = a.TY, D = a.D, ntx = a.ntx;
  bool beyond = false;
  if (a.insts) {
    const Inst& in = a.insts[stp->inst];
    gp = &in.g;
    vp = inst_potential<T>(in);
    gamp = inst_gamma<T>(in);
    phase = inst_phase<T>(in);
    const TileShape& ts = in.tile[a.tile_idx];
    TX = ts.TX; TY = ts.TY; D = ts.D; ntx = ts.ntx;
    beyond = (int)blockIdx.x >= ts.ntx * ts.nty || (int)blockIdx.y >= ts.nslab;
  }
  if (beyond) {
    if (threadIdx.x == 0) {
      double* o = a.part + ((size_t)slot * gridDim.x * gridDim.y + blockIdx.x + gridDim.x * blockIdx.y) * 2;
      o[0] = 0.0;
      o[1] = 0.0;
    }
    return;
  }
  const int nx = gp->nx, ny = gp->ny, nz = gp->nz;
  const long long nxy = gp->nxy;
  const int npt = TX * TY;
  const int t = threadIdx.x;
  // the block is rounded up to whole warps (and, in a batch, to the largest tile);
  // threads past TX*TY*H only join the barriers and the reductions
  const bool worker = t < npt * a.H;
  const int half = worker ? t / npt : 0;
  const int lt = worker ? t - half * npt : 0;
  const int tx = lt % TX, ty = lt / TX;
  const int x0 = (blockIdx.x % ntx) * TX, y0 = (blockIdx.x / ntx) * TY;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool inside = worker && (gx < nx) && (gy < ny);
  const int z0 = blockIdx.y * D;
  const int z1 = min(z0 + D, nz);
  const int SW = TX + 2 * R;
  const int SHt = TY + 2 * R;
  CT* my = sm + half * SW * SHt;
  const long long base = (long long)slot * a.slot_stride + (long long)half * gp->n;
  const CT* __restrict__ r = a.r + base;
  const CT* __restrict__ pin = a.p_in + base;
  CT* __restrict__ pout = a.p_out + base;
  CT* __restrict__ q = a.q + base;
  const CT beta = cfrom<CT>(beta_d);
  const CT* ph = phase + (size_t)(ik * 2 + (half ^ a.conj)) * 2 * kPhaseN;
  const long long pidx = (long long)gx + (long long)nx * gy;

  T kx[R + 1], ky[R + 1], kz[R + 1];
#pragma unroll
  for (int m = 1; m <= R; ++m) {
    kx[m] = (T)gp->kx[m];
    ky[m] = (T)gp->ky[m];
    kz[m] = (T)gp->kz[m];
  }
  const T ediag = (T)(e + gp->diag_c);

  auto pnew = [&](long long off) -> CT {
    const CT rr = r[off], pp = pin[off];
    CT o;
    o.x = rr.x + beta.x * pp.x - beta.y * pp.y;
    o.y = rr.y + beta.x * pp.y + beta.y * pp.x;
    return o;
  };
  // p_new at an arbitrary lateral position of plane zc, wrapped into the cell with
  // its Bloch factor (Eq. Bloch: phi(x + L) = exp(i k L) phi(x)).
  auto wrapped = [&](int xx, int yy, int zc) -> CT {
    int wx = 0, wy = 0;
    if (xx < 0 || xx >= nx) { wx = floordiv(xx, nx); xx -= wx * nx; }
    if (yy < 0 || yy >= ny) { wy = floordiv(yy, ny); yy -= wy * ny; }
    CT v = pnew((long long)zc * nxy + xx + (long long)nx * yy);
    if (wx) v = cmul(v, ph[kPhaseW + wx]);
    if (wy) v = cmul(v, ph[kPhaseN + kPhaseW + wy]);
    return v;
  };

  CT qv[2 * R + 1];
  qv[0] = czero<CT>();
#pragma unroll
  for (int m = 1; m <= 2 * R; ++m) {
    const int z = z0 - R + m - 1;
    qv[m] = (inside && z >= 0 && z < nz) ? pnew((long long)z * nxy + pidx) : czero<CT>();
  }

  DotAcc<T> sg;
  const int nh = 2 * R * (TX + TY);
  for (int zc = z0; zc < z1; ++zc) {
#pragma unroll
    for (int m = 0; m < 2 * R; ++m) qv[m] = qv[m + 1];
    {
      const int z = zc + R;
      qv[2 * R] = (inside && z < nz) ? pnew((long long)z * nxy + pidx) : czero<CT>();
    }
    const CT c = qv[R];
    if (worker) my[(ty + R) * SW + tx + R] = inside ? c : wrapped(gx, gy, zc);
    for (int h = worker ? lt : nh; h < nh; h += npt) {
      int hx, hy;
      if (h < 2 * R * TY) {
        const int row = h / (2 * R), k = h - row * 2 * R;
        hy = row + R;
        hx = (k < R) ? k : TX + k;
      } else {
        const int h2 = h - 2 * R * TY;
        const int col = h2 / (2 * R), k = h2 - col * 2 * R;
        hx = col + R;
        hy = (k < R) ? k : TY + k;
      }
      my[hy * SW + hx] = wrapped(x0 + hx - R, y0 + hy - R, zc);
    }
    __syncthreads();
    if (inside) {
      const long long off = (long long)zc * nxy + pidx;
      const T dr = ediag - vp[off];
      const T di = gamp[zc];
      CT acc;
      acc.x = dr * c.x - di * c.y;
      acc.y = dr * c.y + di * c.x;
      const CT* ctr = my + (ty + R) * SW + (tx + R);
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        const CT xa = ctr[m], xb = ctr[-m], ya = ctr[m * SW], yb = ctr[-m * SW];
        const CT za = qv[R + m], zb = qv[R - m];
        acc.x += kx[m] * (xa.x + xb.x) + ky[m] * (ya.x + yb.x) + kz[m] * (za.x + zb.x);
        acc.y += kx[m] * (xa.y + xb.y) + ky[m] * (ya.y + yb.y) + kz[m] * (za.y + zb.y);
      }
      q[off] = acc;
      pout[off] = c;
      // pairing form: half h pairs with half 1-h at the same point (or itself)
      const CT o = (a.H == 2) ? sm[(1 - half) * SW * SHt + (ty + R) * SW + tx + R] : c;
      sg.add(o, acc);
    }
    __syncthreads();
  }
  const double2 sgv = sg.value();
  double v2[2] = {sgv.x, sgv.y};
  block_sum<2>(v2, red);
  if (threadIdx.x == 0) {
    const int nblk = gridDim.x * gridDim.y;
    const int b = blockIdx.x + gridDim.x * blockIdx.y;
    double* o = a.part + ((size_t)slot * nblk + b) * 2;
    o[0] = v2[0];
    o[1] = v2[1];
  }
}

// ---------------------------------------------------------------------------------
// vector update: x += alpha p, r -= alpha q, partial <r, r> and ||r_h||^2
// ---------------------------------------------------------------------------------

// alpha = rho / sigma of one slot, sigma summed from the stencil's per-block partials
// in a fixed order; called by one full warp, the value is valid in every lane.
__device__ inline double2 slot_alpha(const double* sp, int nblk, double2 rho) {
  const int lane = threadIdx.x & 31;
  double sx = 0.0, sy = 0.0;
  for (int b = lane; b < nblk; b += 32) {
    sx += sp[2 * b];
    sy += sp[2 * b + 1];
  }
  sx = warp_sum(sx);
  sy = warp_sum(sy);
  sx = __shfl_sync(0xffffffffu, sx, 0);
  sy = __shfl_sync(0xffffffffu, sy, 0);
  return cdiv(rho, make_double2(sx, sy));
}

template <typename T>
struct UpdateArgs {
  using CT = typename Cx<T>::type;
  CT* x;                   // NULL: no solution update (multi-shift seed)
  CT* r;
  const CT* p;
  const CT* q;
  const double* sig_part;  // [slot][sig_nblk][2]
  int sig_nblk;
  double* rho_part;        // [slot][gridDim.x][4]: rho re, rho im, |r_0|^2, |r_1|^2
  const Slot* slots;
  long long n, slot_stride;
  int H;
  const Inst* insts;       // batch mode: the slot's grid size comes from its operator
};

template <typename T>
__global__ void __launch_bounds__(256) k_update(const UpdateArgs<T> a) {
  using CT = typename Cx<T>::type;
  __shared__ double red[4][32];
  __shared__ double2 s_alpha;
  const int slot = blockIdx.y;
  const Slot* stp = a.slots + slot;
  if (stp->status != SLOT_ACTIVE) return;
  const long long n = a.insts ? a.insts[stp->inst].g.n : a.n;
  if (threadIdx.x < 32) {
    const double2 al = slot_alpha(a.sig_part + (size_t)slot * a.sig_nblk * 2, a.sig_nblk, stp->rho);
    if (threadIdx.x == 0) s_alpha = al;
  }
  __syncthreads();
  const CT al = cfrom<CT>(s_alpha);
  const long long base = (long long)slot * a.slot_stride;
  DotAcc<T> rr;
  T n0 = 0, n1 = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    CT rv[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h >= a.H) break;
      const long long off = base + (long long)h * n + i;
      const CT qq = a.q[off];
      CT rr = a.r[off];
      if (a.x) {  // the multi-shift engine keeps no seed solution
        const CT pp = a.p[off];
        CT xx = a.x[off];
        xx.x += al.x * pp.x - al.y * pp.y;
        xx.y += al.x * pp.y + al.y * pp.x;
        a.x[off] = xx;
      }
      rr.x -= al.x * qq.x - al.y * qq.y;
      rr.y -= al.x * qq.y + al.y * qq.x;
      a.r[off] = rr;
      rv[h] = rr;
    }
    n0 += rv[0].x * rv[0].x + rv[0].y * rv[0].y;
    if (a.H == 2) {
      n1 += rv[1].x * rv[1].x + rv[1].y * rv[1].y;
      rr.add(rv[0], rv[1]);  // <r, r> = r_+ . r_- + r_- . r_+ = 2 r_+ . r_-
    } else {
      rr.add(rv[0], rv[0]);
    }
  }
  const double2 rrv = rr.value();
  const double rscale = a.H == 2 ? 2.0 : 1.0;
  double v4[4] = {rscale * rrv.x, rscale * rrv.y, (double)n0, (double)n1};
  block_sum<4>(v4, red);
  if (threadIdx.x == 0) {
    double* o = a.rho_part + ((size_t)slot * gridDim.x + blockIdx.x) * 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) o[k] = v4[k];
  }
}

// ---------------------------------------------------------------------------------
// per-slot scalars: one warp per slot
// ---------------------------------------------------------------------------------

struct ScalarArgs {
  const double* rho_part;  // [slot][nblk][4]
  int nblk;
  Slot* slots;
  int S, H, maxit;
  double tol;
  int mixed;               // 1: FP32 iteration; convergence is judged on the FP64
                           // residual, this kernel only requests replacements
  double reliable;         // replacement when the residual dropped by this factor,
  int stall;               // ... or found no new minimum for this many iterations,
  int max_gap;             // ... or after this many iterations without one
  int decade_its;          // mixed: give up (ENOCONV, FP64 fallback) once the residual
                           // has fallen by less than one decade per this many iterations
};

// Status codes written to Slot::result (same values as the C ABI).
constexpr int kOK = 0, kEINVAL = -1, kENOCONV = -4, kEBREAKDOWN = -5;

static __global__ void __launch_bounds__(256) k_scalars(const ScalarArgs a) {
  const int slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (slot >= a.S) return;
  Slot* st = a.slots + slot;
  if (st->status != SLOT_ACTIVE) return;
  double s[4] = {0, 0, 0, 0};
  const double* rp = a.rho_part + (size_t)slot * a.nblk * 4;
  for (int b = lane; b < a.nblk; b += 32)
#pragma unroll
    for (int k = 0; k < 4; ++k) s[k] += rp[4 * b + k];
#pragma unroll
  for (int k = 0; k < 4; ++k) s[k] = warp_sum(s[k]);
  if (lane != 0) return;
  const double2 rho_new = make_double2(s[0], s[1]);
  const int it = st->it + 1;
  const double res = sqrt(a.H == 2 ? fmax(s[2], s[3]) : s[2]);
  int code = 1;  // still running
  if (!isfinite(rho_new.x) || !isfinite(rho_new.y) || !isfinite(res)) code = kEBREAKDOWN;
  else if (!a.mixed && res <= a.tol) code = kOK;
  else if (rho_new.x == 0.0 && rho_new.y == 0.0) code = kEBREAKDOWN;
  else if (it >= a.maxit) code = kENOCONV;
  st->it = it;
  st->res = res;
  if (code != 1) {
    st->result = code;
    st->status = SLOT_DONE;
  } else {
    st->beta = cdiv(rho_new, st->rho);
    st->rho = rho_new;
    if (a.mixed) {
      if (res < st->rbest) {
        st->rbest = res;
        st->it_best = it;
      }
      if (res <= a.reliable * st->rmax || res <= a.tol || it - st->it_best >= a.stall ||
          it - st->last_ref >= a.max_gap)
        st->pending = 1;
      // the FP32 iteration stagnates on the hard columns (FP32 rounding of the search
      // directions, amplified by the high end of the spectrum); hand them over early
      if (a.decade_its > 0 && it >= a.decade_its &&
          fmin(st->rbest, st->rmax) > exp10(-(double)it / a.decade_its)) {
        st->result = kENOCONV;
        st->status = SLOT_DONE;
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// trace of finished slots, results, slot release
// ---------------------------------------------------------------------------------

template <typename TX>
struct TraceArgs {
  using CT = typename Cx<TX>::type;
  const CT* x;             // [slot][half][n]
  Slot* slots;
  Queue* queue;
  const int* rplanes;      // planes with Gamma_R > 0
  int nrp;
  const double* gl;        // Gamma_L per plane
  const double* gr;        // Gamma_R per plane
  double* res_t;
  double* res_tm;
  int* res_it;
  int* res_status;
  long long nxy, n, slot_stride;
  int H;
  const Inst* insts;       // batch mode: planes, profiles and sizes of the slot's operator
};

template <typename TX>
__global__ void __launch_bounds__(256) k_trace(const TraceArgs<TX> a) {
  using CT = typename Cx<TX>::type;
  __shared__ double red[2][32];
  const int slot = blockIdx.x;
  Slot* st = a.slots + slot;
  if (st->status != SLOT_DONE) return;
  const int* rplanes = a.rplanes;
  const double* gl = a.gl;
  const double* gr = a.gr;
  int nrp = a.nrp;
  long long nxy = a.nxy, n = a.n;
  if (a.insts) {
    const Inst& in = a.insts[st->inst];
    rplanes = in.rplanes; gl = in.gl; gr = in.gr; nrp = in.nrp; nxy = in.g.nxy; n = in.g.n;
  }
  double acc[2] = {0.0, 0.0};
  const long long tot = (long long)nrp * nxy;
  for (int h = 0; h < a.H; ++h) {
    const CT* x = a.x + (long long)slot * a.slot_stride + (long long)h * n;
    double s = 0.0;
    for (long long u = threadIdx.x; u < tot; u += blockDim.x) {
      const int pl = rplanes[u / nxy];
      const CT v = x[(long long)pl * nxy + (u % nxy)];
      const double vx = (double)v.x, vy = (double)v.y;
      s += gr[pl] * (vx * vx + vy * vy);
    }
    acc[h] = s;
  }
  block_sum<2>(acc, red);
  if (threadIdx.x == 0) {
    const int item = st->item;
    const double glj = gl[st->j / nxy];
    double t0 = 4.0 * glj * acc[0];
    double t1 = a.H == 2 ? 4.0 * glj * acc[1] : t0;
    if (st->result != kOK) {
      t0 = __longlong_as_double(0x7ff8000000000000LL);
      t1 = t0;
    }
    a.res_t[item] = t0;
    if (a.res_tm) a.res_tm[item] = t1;
    if (a.res_it) a.res_it[item] = st->it;
    if (a.res_status) a.res_status[item] = st->result;
    st->status = SLOT_IDLE;
    st->item = -1;
    atomicAdd(&a.queue->harvested, 1);
  }
}

// ---------------------------------------------------------------------------------
// work assignment (single block, deterministic slot order)
// ---------------------------------------------------------------------------------

struct AssignArgs {
  Slot* slots;
  int S, H;
  Queue* queue;
  const double* item_e;
  const int* item_ik;
  const long long* item_col;
  const int* lplanes;   // planes with Gamma_L > 0
  int nlp, nk;
  long long nxy;
  const int* item_inst; // batch mode: operator of each item (NULL: all items use insts[0])
  const Inst* insts;    // batch mode: when set, lplanes / nlp / nk / nxy come from here
  int ninst;
};

static __global__ void __launch_bounds__(1024) k_assign(const AssignArgs a) {
  __shared__ int s_next, s_tot;
  __shared__ int s_warp[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_next = a.queue->next;
  __syncthreads();
  const int nitems = a.queue->nitems;
  for (int base = 0; base < a.S; base += blockDim.x) {
    const int s = base + tid;
    int need = 0;
    if (s < a.S) {
      a.slots[s].init = 0;
      need = a.slots[s].status == SLOT_IDLE;
    }
    // block exclusive scan of need
    unsigned m = __ballot_sync(0xffffffffu, need);
    int wrank = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) s_warp[wid] = __popc(m);
    __syncthreads();
    if (tid == 0) {
      int acc = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        int c = s_warp[w];
        s_warp[w] = acc;
        acc += c;
      }
      s_tot = acc;
    }
    __syncthreads();
    const int item = s_next + s_warp[wid] + wrank;
    if (need && item < nitems) {
      Slot* st = a.slots + s;
      const double e = a.item_e[item];
      const int ik = a.item_ik[item];
      const long long col = a.item_col[item];
      const int ii = a.item_inst ? a.item_inst[item] : 0;
      const bool ii_ok = !a.insts || (ii >= 0 && ii < a.ninst);
      const int* lplanes = a.lplanes;
      int nk = a.nk;
      long long nxy = a.nxy, nrhs = (long long)a.nlp * a.nxy;
      if (a.insts && ii_ok) {
        const Inst& in = a.insts[ii];
        lplanes = in.lplanes; nk = in.nk; nxy = in.g.nxy; nrhs = (long long)in.nlp * in.g.nxy;
      }
      st->inst = ii_ok ? ii : 0;
      st->item = item;
      st->it = 0;
      st->refresh = 0;
      st->pending = 0;
      st->last_ref = 0;
      st->it_best = 0;
      st->rbest = 1.0;
      st->rmax = 1.0;
      st->res = 1.0;
      st->beta = make_double2(0.0, 0.0);
      st->rho = make_double2(a.H == 2 ? 2.0 : 1.0, 0.0);  // <e_j, e_j> in the pairing form
      if (!ii_ok || !isfinite(e) || ik < 0 || ik >= nk || col < 0 || col >= nrhs) {
        st->ik = 0;
        st->e = 0.0;
        st->j = 0;
        st->result = kEINVAL;
        st->status = SLOT_DONE;
      } else {
        st->ik = ik;
        st->e = e;
        st->j = (long long)lplanes[col / nxy] * nxy + col % nxy;
        st->result = 0;
        st->status = SLOT_ACTIVE;
        st->init = 1;
      }
    }
    __syncthreads();
    if (tid == 0) s_next = min(s_next + s_tot, nitems);
    __syncthreads();
  }
  if (tid == 0) a.queue->next = s_next;
}

// ---------------------------------------------------------------------------------
// device-side loop control: ends the graph's WHILE loop once every item is harvested
// or the per-launch chunk limit is reached (so a launch always ends)
// ---------------------------------------------------------------------------------

static __global__ void k_continue(cudaGraphConditionalHandle h, Queue* q) {
  const int c = q->chunks + 1;
  q->chunks = c;
  const bool more = q->harvested < q->nitems && c < q->limit;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

// ---------------------------------------------------------------------------------
// vector initialisation of newly assigned slots: x = 0, r = e_j, p = 0
// ---------------------------------------------------------------------------------

template <typename T>
struct InitArgs {
  using CT = typename Cx<T>::type;
  CT* x;
  CT* r;
  CT* p;
  const Slot* slots;
  long long n, slot_stride;
  int H;
  const Inst* insts;
};

template <typename T>
__global__ void __launch_bounds__(256) k_init(const InitArgs<T> a) {
  using CT = typename Cx<T>::type;
  const int slot = blockIdx.y;
  const Slot* st = a.slots + slot;
  if (!st->init) return;
  const long long n = a.insts ? a.insts[st->inst].g.n : a.n;
  const long long j = st->j;
  const long long base = (long long)slot * a.slot_stride;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    for (int h = 0; h < a.H; ++h) {
      const long long off = base + (long long)h * n + i;
      a.x[off] = czero<CT>();
      a.p[off] = czero<CT>();
      CT rv = czero<CT>();
      if (i == j) rv.x = (T)1;
      a.r[off] = rv;
    }
  }
}

// ---------------------------------------------------------------------------------
// stand-alone trace of given vectors (checks the reduction on its own)
// ---------------------------------------------------------------------------------

struct VecTraceArgs {
  const double2* x;  // [v][n]
  const long long* cols;
  const int* lplanes;
  const int* rplanes;
  int nlp, nrp;
  const double* gl;
  const double* gr;
  double* t_out;
  long long nxy, n;
};

static __global__ void __launch_bounds__(256) k_vec_trace(const VecTraceArgs a) {
  __shared__ double red[1][32];
  const int v = blockIdx.x;
  const double2* x = a.x + (long long)v * a.n;
  const long long tot = (long long)a.nrp * a.nxy;
  double s[1] = {0.0};
  for (long long u = threadIdx.x; u < tot; u += blockDim.x) {
    const int pl = a.rplanes[u / a.nxy];
    const double2 val = x[(long long)pl * a.nxy + (u % a.nxy)];
    s[0] += a.gr[pl] * (val.x * val.x + val.y * val.y);
  }
  block_sum<1>(s, red);
  if (threadIdx.x == 0) {
    const long long col = a.cols[v];
    const long long nrhs = (long long)a.nlp * a.nxy;
    if (col < 0 || col >= nrhs) {
      a.t_out[v] = __longlong_as_double(0x7ff8000000000000LL);
    } else {
      const int pl = a.lplanes[col / a.nxy];
      a.t_out[v] = 4.0 * a.gl[pl] * s[0];
    }
  }
}

}  // namespace transec
