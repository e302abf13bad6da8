// Multi-shift slot engine: many transpose-BiCG runs in flight on the GPU, each run
// serving a whole window of energies at once.
//
// For fixed k, A(E, k) = A(E0, k) + (E - E0) 1 (Sec. II.A: G(E) = [E - H_k + i Gamma]^-1),
// so every energy of a window shares the Krylov space of a seed energy E0.  A run
// iterates the seed's transpose BiCG (A x = b with the shadow system A^T y = b;
// A(E, k)^T = A(E, -k), Sec. II.B) and carries, for every shift sigma = E - E0, the
// collinear-residual scalars pi_sigma and the shifted iterates, kept only on the grid
// planes the result reads:
//
//   pi_{n+1}     = (1 + alpha_n sigma) pi_n + (alpha_n beta_{n-1} / alpha_{n-1}) (pi_n - pi_{n-1})
//   p_sigma,n    = r_n / pi_n + (pi_{n-1} / pi_n)^2 beta_{n-1} p_sigma,n-1
//   x_sigma,n+1  = x_sigma,n + (alpha_n pi_n / pi_{n+1}) p_sigma,n
//
// (the shadow iterates y_sigma likewise from the seed's shadow residual).  A shift is
// converged once max(||r||, ||r~||) / |pi_sigma| <= tol ||b||; it then stops changing.
// The seed runs until every shift of its window has converged.
//
// Runs are items of a device-side queue (slots retire and refill as in the plain
// engine) of three kinds:
//   UNIT   b = e_j for a left-CAP column j; the result is t_j(E) and t_j(E, -k) for
//          every energy of the window (read on the Gamma_R planes);
//   LEFT   b = Gamma_L^1/2 omega for a random phase vector omega on the left-CAP
//          support; the Gamma_R planes of x and y are kept;
//   RIGHT  b = Gamma_R^1/2 psi on the right-CAP support; the Gamma_L planes are kept.
// LEFT and RIGHT runs of one k form a two-sided sketch of M = Gamma_R^1/2 G Gamma_L^1/2
// (Sec. II.A: T = 4 Tr[Gamma_L G^dagger Gamma_R G] = 4 ||M||_F^2): the primal halves of
// the LEFT runs give Y = M Omega, the shadow halves of the RIGHT runs give
// W = Psi^T M (both at +k; the other halves give the same pair at -k).  k_ms_gn then
// forms, per energy and sign of k, the low-rank estimate of Tropp, Yurtsever, Udell &
// Cevher (SIAM J. Matrix Anal. Appl. 38, 2017): Q = orth(Y), X = (Psi^T Q)^+ W,
// T = 4 ||X||_F^2, exact when the numerical rank of M (about the number of open
// channels) is below the sketch size.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "engine.cuh"
#include "stencil_df.cuh"

namespace transec {
template <typename T>
cudaError_t prepare_stencil(int R, size_t smem);
}

using namespace transec;

namespace transec {

enum RunKind : int { RUN_UNIT = 0, RUN_LEFT = 1, RUN_RIGHT = 2 };

// Largest relative inversion gap of V (max |V(r) - V(R_{z,pi} r)| / max |V|) accepted for
// P-symmetric runs: the operator's own rounding, far below what moves T at 1e-6.
constexpr double kPsymTol = 1e-12;

// Per-run state beside the seed's Slot.
struct MsSlot {
  double2 alpha;       // alpha_n of the current iteration
  double2 alpha_prev;  // alpha_{n-1} (1 before the first iteration)
  double bnorm;        // ||b||_2
  int kind;            // RunKind
  int rep;             // sketch: group (k representative) of the run
  int idx;             // sketch: index of the random vector within its kind
  int pad[3];
};

// Per-run, per-shift state.
struct MsShift {
  double2 pi, pi_prev, pi_next;
  int active;   // 1 while the shift iterates
  int status;   // kOK, kENOCONV or kEBREAKDOWN once the shift stopped
  int conv_it;  // seed iteration at which it stopped
  int pad;
};

// Coefficients of one iteration's shifted update (k_ms_coef -> k_ms_shift).
struct MsCoef {
  double2 inv_pi, beta_s, alpha_s;
  float4 inv_pi_df, beta_s_df, alpha_s_df;  // the same in double-float
};

// One queued run.
struct MsItem {
  int ik, kind, rep, idx;
  long long col;  // UNIT: left-CAP column
};

struct SweepBufs {
  int S = 0, ne = 0;
  long long n = 0, no = 0;
  int nblk_st = 0, nblk3 = 0, nitems = 0, nrnd = 0;
  double2 *R = nullptr, *P0 = nullptr, *P1 = nullptr, *Q = nullptr;
  double2 *XS = nullptr, *PS = nullptr;
  double *sig_part = nullptr, *rho_part = nullptr;
  Slot* slots = nullptr;
  MsSlot* ms = nullptr;
  MsShift* sh = nullptr;
  MsCoef* coef = nullptr;
  Queue* queue = nullptr;
  MsItem* items = nullptr;
  double* energies = nullptr;
  double2* rnd = nullptr;
  int *lrank = nullptr, *rrank = nullptr;
  int* escale = nullptr;       // [S] double-float form: 2^k scaling of the bilinear forms
  float2* v_df = nullptr;      // V, Gamma and Bloch phases in double-float
  float2* gam_df = nullptr;
  float4* phase_df = nullptr;
  size_t cap_n = 0, cap_ph = 0;
  // capacities (elements) of the buffers above, kept between calls
  size_t cap_vec = 0, cap_shv = 0, cap_sig = 0, cap_rho = 0, cap_slots = 0, cap_shs = 0;
  size_t cap_items = 0, cap_ene = 0, cap_rnd = 0, cap_nz = 0;
  void release() {
    cudaFree(R); cudaFree(P0); cudaFree(P1); cudaFree(Q); cudaFree(XS); cudaFree(PS);
    cudaFree(sig_part); cudaFree(rho_part); cudaFree(slots); cudaFree(ms); cudaFree(sh);
    cudaFree(coef); cudaFree(queue); cudaFree(items); cudaFree(energies); cudaFree(rnd);
    cudaFree(lrank); cudaFree(rrank); cudaFree(escale); cudaFree(v_df); cudaFree(gam_df);
    cudaFree(phase_df);
    *this = SweepBufs{};
  }
};

void sweep_release(transec_ctx* ctx) {
  if (ctx && ctx->sweep) {
    ctx->sweep->release();
    delete ctx->sweep;
    ctx->sweep = nullptr;
  }
}

}  // namespace transec

namespace {

// ---------------------------------------------------------------------------------
// random phases: splitmix64 (Steele, Lea & Flood, OOPSLA 2014) of a counter built
// from the seed, the run group, the kind, the vector index and the point
// ---------------------------------------------------------------------------------

__host__ __device__ inline unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

struct RandomArgs {
  double2* rnd;  // [rep][2 kinds][smax][np]
  int nrep, smax;
  long long np;
  unsigned long long seed;
};

// rnd[rep][kind][i][u] = exp(2 pi i theta), theta uniform in [0, 1) (53 bits)
__global__ void __launch_bounds__(256) k_ms_random(const RandomArgs a) {
  const long long total = (long long)a.nrep * 2 * a.smax * a.np;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const unsigned long long h = splitmix64(a.seed ^ splitmix64((unsigned long long)e));
    const double theta = (double)(h >> 11) * 0x1.0p-53;
    double s, c;
    sincospi(2.0 * theta, &s, &c);
    a.rnd[e] = make_double2(c, s);
  }
}

// ---------------------------------------------------------------------------------
// storage of the vectors: complex FP64 (double2) or double-float (float4); the
// kernels off the hot path read and write them through FP64 values
// ---------------------------------------------------------------------------------

__device__ inline double2 vload(const double2* p, long long i) { return p[i]; }
__device__ inline double2 vload(const float4* p, long long i) { return dfc_to_double2(p[i]); }
__device__ inline void vstore(double2* p, long long i, double2 v) { p[i] = v; }
__device__ inline void vstore(float4* p, long long i, double2 v) { p[i] = dfc_from_double2(v); }

// exponent k with 2^k x of order one (clamped to the float range)
__device__ inline int unit_exponent(double x) {
  if (!(x > 0.0) || !isfinite(x)) return 0;
  return max(-120, min(120, -ilogb(x)));
}

// ---------------------------------------------------------------------------------
// queue: assignment, vector initialisation, rho_0
// ---------------------------------------------------------------------------------

struct MsArgs {
  Slot* slots;
  MsSlot* ms;
  MsShift* sh;
  MsCoef* coef;
  Queue* queue;
  const MsItem* items;
  const double* energies;  // ne
  double e0;               // seed energy
  int S, ne, nk;
  double2* R;
  double2* P0;
  double2* XS;
  double2* PS;
  const double2* rnd;      // [rep][2][smax][np]
  int smax;
  long long np;            // points per random vector (largest CAP support)
  long long n, no, nxy;
  const int* lplanes;
  const int* rplanes;
  const int* lrank;        // per plane: index among the left-CAP planes, or -1
  const int* rrank;
  int nlp, nrp;
  const double* gl;
  const double* gr;
  const double* rho_part;  // [slot][nblk3][4]
  int nblk3;
  const double* sig_part;  // [slot][nblk_st][2]
  int nblk_st;
  double tol;
  int maxit;
  int stall_its;           // > 0: a run stops once no shift has converged for this long
  int* escale;             // [S]
  int H;                   // halves per run: 2 (transpose BiCG), 1 (P-symmetric COCG)
  int psym;                // P-symmetric form: the bilinear forms pair r with P_k r
  int nx, ny;
  const double2* phase;    // [nk][2][2][kPhaseN] Bloch phases
  // UNIT results: [item][shift][2] t, [item][shift] iterations and status
  double* res_t;
  int* res_it;
  int* res_st;
};

// Hands queued runs to idle slots in slot order (one thread: the refill of a chunk is
// a few slots, and the order must not depend on the launch).
__global__ void k_ms_assign(const MsArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Queue* q = a.queue;
  int next = q->next;
  for (int s = 0; s < a.S; ++s) {
    Slot& st = a.slots[s];
    st.init = 0;
    if (st.status != SLOT_IDLE || next >= q->nitems) continue;
    const MsItem it = a.items[next];
    Slot ns{};
    ns.status = SLOT_ACTIVE;
    ns.item = next;
    ns.ik = it.ik;
    ns.e = a.e0;
    ns.init = 1;
    ns.j = it.kind == RUN_UNIT
               ? (long long)a.lplanes[it.col / a.nxy] * a.nxy + it.col % a.nxy
               : -1;
    ns.beta = make_double2(0.0, 0.0);
    ns.rho = make_double2(2.0, 0.0);  // <e_j, e_j> in the pairing form; k_ms_rho0 sets the rest
    st = ns;
    MsSlot m{};
    m.alpha = make_double2(0.0, 0.0);
    m.alpha_prev = make_double2(1.0, 0.0);
    m.bnorm = 1.0;
    m.kind = it.kind;
    m.rep = it.rep;
    m.idx = it.idx;
    a.ms[s] = m;
    a.escale[s] = 0;
    ++next;
  }
  q->next = next;
}

// r = b on every half, p = 0, for newly assigned slots.  grid (blocks, S)
template <typename V>
__global__ void __launch_bounds__(256) k_ms_init(const MsArgs a) {
  V* R = reinterpret_cast<V*>(a.R);
  V* P0 = reinterpret_cast<V*>(a.P0);
  const int slot = blockIdx.y;
  const Slot& st = a.slots[slot];
  if (!st.init) return;
  const MsSlot m = a.ms[slot];
  const double2* rl = a.rnd + (((long long)m.rep * 2 + 0) * a.smax + m.idx) * a.np;
  const double2* rr = a.rnd + (((long long)m.rep * 2 + 1) * a.smax + m.idx) * a.np;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (long long)gridDim.x * blockDim.x) {
    double2 b = make_double2(0.0, 0.0);
    const int pl = (int)(i / a.nxy);
    const long long w = i % a.nxy;
    if (m.kind == RUN_UNIT) {
      if (i == st.j) b.x = 1.0;
    } else if (m.kind == RUN_LEFT) {
      const int rk = a.lrank[pl];
      if (rk >= 0) {
        const double s = sqrt(a.gl[pl]);
        const double2 o = rl[(long long)rk * a.nxy + w];
        b = make_double2(s * o.x, s * o.y);
      }
    } else {
      const int rk = a.rrank[pl];
      if (rk >= 0) {
        const double s = sqrt(a.gr[pl]);
        const double2 o = rr[(long long)rk * a.nxy + w];
        b = make_double2(s * o.x, s * o.y);
      }
    }
    for (int h = 0; h < a.H; ++h) {
      const long long off = (long long)slot * a.H * a.n + (long long)h * a.n + i;
      vstore(R, off, b);
      vstore(P0, off, make_double2(0.0, 0.0));
    }
  }
}

// Per-shift vectors and scalars of newly assigned slots.  grid (blocks, ne, S)
__global__ void __launch_bounds__(256) k_ms_init_shift(const MsArgs a) {
  const int slot = blockIdx.z, s = blockIdx.y;
  if (!a.slots[slot].init) return;
  const long long base = ((long long)slot * a.ne + s) * 2 * a.no;
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < 2 * a.no;
       u += (long long)gridDim.x * blockDim.x) {
    a.XS[base + u] = make_double2(0.0, 0.0);
    a.PS[base + u] = make_double2(0.0, 0.0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    MsShift z{};
    z.pi = z.pi_prev = z.pi_next = make_double2(1.0, 0.0);
    const double e = a.energies[s];
    z.active = isfinite(e) ? 1 : 0;
    z.status = isfinite(e) ? kENOCONV : kEINVAL;
    z.conv_it = 0;
    a.sh[(long long)slot * a.ne + s] = z;
  }
}

// rho_0 = 2 b.b (pairing form of the two equal halves; (P_k b)^T b in the P-symmetric
// form) and ||b|| of new random runs.  grid S, 256 threads
template <typename V>
__global__ void __launch_bounds__(256) k_ms_rho0(const MsArgs a) {
  __shared__ double red[3][32];
  const int slot = blockIdx.x;
  Slot& st = a.slots[slot];
  if (!st.init) return;
  MsSlot& m = a.ms[slot];
  if (m.kind == RUN_UNIT) return;
  const int* planes = m.kind == RUN_LEFT ? a.lplanes : a.rplanes;
  const long long np = (long long)(m.kind == RUN_LEFT ? a.nlp : a.nrp) * a.nxy;
  const V* r = reinterpret_cast<const V*>(a.R) + (long long)slot * a.H * a.n;
  const double2* ph = a.phase + (size_t)(st.ik * 2) * 2 * kPhaseN;
  double v[3] = {0.0, 0.0, 0.0};
  for (long long u = threadIdx.x; u < np; u += blockDim.x) {
    const long long pl = (long long)planes[u / a.nxy] * a.nxy;
    const int w = (int)(u % a.nxy);
    const double2 b = vload(r, pl + w);
    double2 o = b;  // the pairing partner of b at this point
    if (a.psym) {
      const int y = w / a.nx, x = w - y * a.nx;
      o = vload(r, pl + (x ? a.nx - x : 0) + (long long)a.nx * (y ? a.ny - y : 0));
      if (x) o = cmul(o, ph[kPhaseW - 1]);
      if (y) o = cmul(o, ph[kPhaseN + kPhaseW - 1]);
    }
    v[0] += o.x * b.x - o.y * b.y;
    v[1] += o.x * b.y + o.y * b.x;
    v[2] += b.x * b.x + b.y * b.y;
  }
  block_sum<3>(v, red);
  if (threadIdx.x == 0) {
    const double f = a.psym ? 1.0 : 2.0;
    st.rho = make_double2(f * v[0], f * v[1]);
    m.bnorm = sqrt(v[2]);
    a.escale[slot] = unit_exponent(m.bnorm);
  }
}

// ---------------------------------------------------------------------------------
// one iteration: coefficients, shifted update, convergence
// ---------------------------------------------------------------------------------

// alpha_n of the seed and pi_{n+1}, alpha_sigma, beta_sigma, 1/pi_n of every active
// shift.  grid S, 256 threads
__global__ void __launch_bounds__(256) k_ms_coef(const MsArgs a) {
  __shared__ double2 s_alpha;
  const int slot = blockIdx.x;
  const Slot& st = a.slots[slot];
  if (st.status != SLOT_ACTIVE) return;
  if (threadIdx.x < 32) {
    const double2 al = slot_alpha(a.sig_part + (size_t)slot * a.nblk_st * 2, a.nblk_st, st.rho);
    if (threadIdx.x == 0) {
      s_alpha = al;
      a.ms[slot].alpha = al;
    }
  }
  __syncthreads();
  const double2 al = s_alpha;
  const double2 bp = st.beta;                 // beta_{n-1}
  const double2 ap = a.ms[slot].alpha_prev;   // alpha_{n-1}
  const double2 c = cdiv(cmul(al, bp), ap);   // alpha_n beta_{n-1} / alpha_{n-1}
  for (int s = threadIdx.x; s < a.ne; s += blockDim.x) {
    MsShift& z = a.sh[(long long)slot * a.ne + s];
    if (!z.active) continue;
    const double sig = a.energies[s] - st.e;
    const double2 t1 = cmul(make_double2(1.0 + al.x * sig, al.y * sig), z.pi);
    const double2 t2 = cmul(c, csub(z.pi, z.pi_prev));
    const double2 pn = cadd(t1, t2);
    if (!(isfinite(pn.x) && isfinite(pn.y)) || (pn.x == 0.0 && pn.y == 0.0)) {
      z.active = 0;
      z.status = kEBREAKDOWN;
      z.conv_it = st.it + 1;
      continue;
    }
    z.pi_next = pn;
    MsCoef co;
    co.alpha_s = cdiv(cmul(al, z.pi), pn);
    co.inv_pi = cdiv(make_double2(1.0, 0.0), z.pi);
    const double2 ratio = cdiv(z.pi_prev, z.pi);
    co.beta_s = cmul(cmul(ratio, ratio), bp);
    co.inv_pi_df = dfc_from_double2(co.inv_pi);
    co.beta_s_df = dfc_from_double2(co.beta_s);
    co.alpha_s_df = dfc_from_double2(co.alpha_s);
    a.coef[(long long)slot * a.ne + s] = co;
  }
}

// p_sigma = r_n / pi_n + beta_sigma p_sigma, x_sigma += alpha_sigma p_sigma on the kept
// planes, every half, active shifts.  grid (ceil(no / 256), ne, S)
__global__ void __launch_bounds__(256) k_ms_shift(const MsArgs a) {
  const int slot = blockIdx.z, s = blockIdx.y;
  if (a.slots[slot].status != SLOT_ACTIVE) return;
  const long long zs = (long long)slot * a.ne + s;
  if (!a.sh[zs].active) return;
  const MsCoef co = a.coef[zs];
  const int kind = a.ms[slot].kind;
  const int* planes = kind == RUN_RIGHT ? a.lplanes : a.rplanes;
  const long long nro = (long long)(kind == RUN_RIGHT ? a.nlp : a.nrp) * a.nxy;
  const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= nro) return;
  const long long pt = (long long)planes[u / a.nxy] * a.nxy + u % a.nxy;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (h >= a.H) break;
    const double2 rv = a.R[(long long)slot * a.H * a.n + (long long)h * a.n + pt];
    const long long off = (zs * 2 + h) * a.no + u;
    double2 pv = a.PS[off];
    pv = cadd(cmul(rv, co.inv_pi), cmul(co.beta_s, pv));
    a.PS[off] = pv;
    a.XS[off] = cadd(a.XS[off], cmul(co.alpha_s, pv));
  }
}

// The same in double-float storage and arithmetic.
__global__ void __launch_bounds__(256) k_ms_shift_df(const MsArgs a) {
  const int slot = blockIdx.z, s = blockIdx.y;
  if (a.slots[slot].status != SLOT_ACTIVE) return;
  const long long zs = (long long)slot * a.ne + s;
  if (!a.sh[zs].active) return;
  const MsCoef& cf = a.coef[zs];
  const dfc inv_pi = dfc_load(cf.inv_pi_df), beta_s = dfc_load(cf.beta_s_df), alpha_s = dfc_load(cf.alpha_s_df);
  const int kind = a.ms[slot].kind;
  const int* planes = kind == RUN_RIGHT ? a.lplanes : a.rplanes;
  const long long nro = (long long)(kind == RUN_RIGHT ? a.nlp : a.nrp) * a.nxy;
  const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= nro) return;
  const long long pt = (long long)planes[u / a.nxy] * a.nxy + u % a.nxy;
  const float4* R = reinterpret_cast<const float4*>(a.R);
  float4* PS = reinterpret_cast<float4*>(a.PS);
  float4* XS = reinterpret_cast<float4*>(a.XS);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (h >= a.H) break;
    const dfc rv = dfc_load(R[(long long)slot * a.H * a.n + (long long)h * a.n + pt]);
    const long long off = (zs * 2 + h) * a.no + u;
    const dfc pv = dfc_add(dfc_mul(rv, inv_pi), dfc_mul(beta_s, dfc_load(PS[off])));
    PS[off] = dfc_store(pv);
    XS[off] = dfc_store(dfc_fma(alpha_s, pv, dfc_load(XS[off])));
  }
}

// Seed residual norms and rho_{n+1}, shift convergence (residual of the shift =
// max(||r||, ||r~||) / |pi_{n+1}|), maxit and breakdown, beta_n.  grid S, 256 threads
__global__ void __launch_bounds__(256) k_ms_scalars(const MsArgs a) {
  __shared__ double s_v[4];
  __shared__ int s_live[8];
  const int slot = blockIdx.x;
  Slot& st = a.slots[slot];
  if (st.status != SLOT_ACTIVE) return;
  if (threadIdx.x < 32) {
    double v[4] = {0, 0, 0, 0};
    const double* rp = a.rho_part + (size_t)slot * a.nblk3 * 4;
    for (int b = threadIdx.x; b < a.nblk3; b += 32)
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] += rp[4 * b + k];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = warp_sum(v[k]);
    if (threadIdx.x == 0)
      for (int k = 0; k < 4; ++k) s_v[k] = v[k];
  }
  __syncthreads();
  const double2 rho_new = make_double2(s_v[0], s_v[1]);
  const double rn = sqrt(fmax(s_v[2], s_v[3]));
  const int it = st.it + 1;
  const double thresh = a.tol * a.ms[slot].bnorm;
  const bool brk = !(isfinite(rho_new.x) && isfinite(rho_new.y)) ||
                   (rho_new.x == 0.0 && rho_new.y == 0.0) || !isfinite(rn);
  int live = 0, fresh = 0;
  for (int s = threadIdx.x; s < a.ne; s += blockDim.x) {
    MsShift& z = a.sh[(long long)slot * a.ne + s];
    if (!z.active) continue;
    z.pi_prev = z.pi;
    z.pi = z.pi_next;
    const double res = rn / hypot(z.pi.x, z.pi.y);
    if (isfinite(res) && res <= thresh) {
      z.active = 0;
      z.status = kOK;
      z.conv_it = it;
      ++fresh;
    } else if (brk || !isfinite(res)) {
      z.active = 0;
      z.status = kEBREAKDOWN;
      z.conv_it = it;
    } else if (it >= a.maxit) {
      z.active = 0;
      z.status = kENOCONV;
      z.conv_it = it;
    } else {
      ++live;
    }
  }
  const int packed = live + (fresh << 16);  // at most 1024 shifts each
  int sum = packed;
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) s_live[threadIdx.x >> 5] = sum;
  __syncthreads();
  // stall rule (double-float runs): no new convergence for stall_its iterations since
  // the last one (3 stall_its before the first) stops the remaining shifts
  __shared__ int s_stop;
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_live[w];
    const int nlive = tot & 0xffff, nfresh = tot >> 16;
    if (nfresh > 0) st.it_best = it;  // iteration of the latest shift convergence
    s_stop = nlive > 0 && a.stall_its > 0 &&
             (st.it_best > 0 ? it - st.it_best > a.stall_its : it > 3 * a.stall_its);
    s_live[0] = s_stop ? 0 : nlive;
  }
  __syncthreads();
  if (s_stop)
    for (int s = threadIdx.x; s < a.ne; s += blockDim.x) {
      MsShift& z = a.sh[(long long)slot * a.ne + s];
      if (!z.active) continue;
      z.active = 0;
      z.status = kENOCONV;
      z.conv_it = it;
    }
  if (threadIdx.x == 0) {
    const int tot = s_live[0];
    st.it = it;
    st.res = rn;
    if (tot == 0) {
      st.status = SLOT_DONE;
      st.result = kOK;
    } else {
      st.beta = cdiv(rho_new, st.rho);
      st.rho = rho_new;
      a.ms[slot].alpha_prev = a.ms[slot].alpha;
      a.escale[slot] = unit_exponent(rn);
    }
  }
}

// UNIT runs that finished: t_j = 4 Gamma_L(j) sum_R Gamma_R |x_sigma|^2 per shift and
// half.  grid (ne, S), 256 threads
template <typename V>
__global__ void __launch_bounds__(256) k_ms_trace(const MsArgs a) {
  __shared__ double red[2][32];
  const int s = blockIdx.x, slot = blockIdx.y;
  const Slot& st = a.slots[slot];
  if (st.status != SLOT_DONE || a.ms[slot].kind != RUN_UNIT) return;
  const long long zs = (long long)slot * a.ne + s;
  const long long nro = (long long)a.nrp * a.nxy;
  double v[2] = {0.0, 0.0};
  for (int h = 0; h < 2; ++h) {
    const V* x = reinterpret_cast<const V*>(a.XS) + (zs * 2 + h) * a.no;
    double acc = 0.0;
    for (long long u = threadIdx.x; u < nro; u += blockDim.x) {
      const double2 xv = vload(x, u);
      acc += a.gr[a.rplanes[u / a.nxy]] * (xv.x * xv.x + xv.y * xv.y);
    }
    v[h] = acc;
  }
  block_sum<2>(v, red);
  if (threadIdx.x == 0) {
    const MsShift z = a.sh[zs];
    const double glj = a.gl[st.j / a.nxy];
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    const long long o = (long long)st.item * a.ne + s;
    a.res_t[2 * o] = z.status == kOK ? 4.0 * glj * v[0] : nan;
    a.res_t[2 * o + 1] = z.status == kOK ? 4.0 * glj * v[1] : nan;
    a.res_it[o] = z.conv_it;
    a.res_st[o] = z.status;
  }
}

// Finished runs release their slots (in slot order) and count as harvested.
__global__ void k_ms_release(const MsArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int h = 0;
  for (int s = 0; s < a.S; ++s) {
    Slot& st = a.slots[s];
    if (st.status != SLOT_DONE) continue;
    st.status = SLOT_IDLE;
    st.item = -1;
    ++h;
  }
  a.queue->harvested += h;
}

// P-symmetric runs iterate the primal half alone.  Their shadow half of the kept planes
// is filled with P_k x: by A(-k) P_k = P_k A(k) (V invariant under the in-plane
// inversion R_{z,pi}, Sec. II.C), P_k x solves A(-k) y = P_k b, so it is the shadow
// solution for the mirrored right-hand side P_k b.  grid (ceil(no / 256), ne, S)
template <typename V>
__global__ void __launch_bounds__(256) k_ms_psym_fill(const MsArgs a) {
  const int slot = blockIdx.z, s = blockIdx.y;
  const long long zs = (long long)slot * a.ne + s;
  const long long nro = (long long)(a.ms[slot].kind == RUN_RIGHT ? a.nlp : a.nrp) * a.nxy;
  const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= nro) return;
  const double2* ph = a.phase + (size_t)(a.slots[slot].ik * 2) * 2 * kPhaseN;
  const long long pl = u / a.nxy;
  const int w = (int)(u - pl * a.nxy);
  const int y = w / a.nx, x = w - y * a.nx;
  V* xs = reinterpret_cast<V*>(a.XS);
  double2 o = vload(xs, zs * 2 * a.no + pl * a.nxy + (x ? a.nx - x : 0) + (long long)a.nx * (y ? a.ny - y : 0));
  if (x) o = cmul(o, ph[kPhaseW - 1]);
  if (y) o = cmul(o, ph[kPhaseN + kPhaseW - 1]);
  vstore(xs, (zs * 2 + 1) * a.no + u, o);
}

// ---------------------------------------------------------------------------------
// two-sided sketch reduction: T(E, +-k) per shift from the LEFT / RIGHT runs
// ---------------------------------------------------------------------------------

struct GnArgs {
  double2* XS;             // [slot][ne][2][no]; the LEFT runs' kept planes are
                           // orthogonalised in place
  const MsShift* sh;
  const int* run_slot;     // [rep][sl + sr]: slots of the LEFT runs, then the RIGHT runs
  const double2* rnd;      // [rep][2][smax][np]
  int smax;
  long long np, no, nxy;
  int ne, sl, sr;
  const int* lplanes;
  const int* rplanes;
  int nlp, nrp;
  const double* gl;
  const double* gr;
  double* T;               // [rep][ne][2] (T(E, k), T(E, -k))
  int* rank;               // [rep][ne][2]
  int* status;             // [rep][ne][2]
  double drop;             // relative norm below which a column of Y adds no direction
  double* miss;            // [rep][ne][2] 4 ||(1 - P) y_last||^2: the energy of M outside the span
                           // of the first s_left - 1 columns of Y (an estimate of what the
                           // sketch misses of T; E ||(1 - P) M omega||^2 = ||(1 - P) M||_F^2)
  int psym;                // P-symmetric runs: the +k rows of W belong to P_k psi
  int nx, ny;
  const Slot* slots;
  const double2* phase;    // [nk][2][2][kPhaseN] Bloch phases
};

constexpr int kGnMaxL = 32, kGnMaxR = 64;

// Block sum of up to 2*kGnChunk doubles per thread into s_out (valid after return).
template <int NV>
__device__ inline void gn_block_sum(double (&v)[NV], double* s_out, double (*red)[32]) {
  block_sum<NV>(v, red);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) s_out[k] = v[k];
  __syncthreads();
}

constexpr int kGnChunk = 8;

// grid (ne, nrep, 2 signs), 256 threads, dynamic shared memory for K and G_b.  V is
// the storage of the kept planes; the LEFT runs' planes are rewritten in place as
// complex FP64 (Y, then Q).
template <typename V>
__global__ void __launch_bounds__(256) k_ms_gn(const GnArgs a) {
  extern __shared__ __align__(16) unsigned char gn_smem[];
  __shared__ double red[2 * kGnChunk][32];
  __shared__ double s_red[2 * kGnChunk];
  __shared__ double2 s_d[kGnMaxL];
  __shared__ int s_keep[kGnMaxL];
  __shared__ int s_status;
  __shared__ double s_nrm0;
  __shared__ double2 s_v[kGnMaxR];
  __shared__ int s_cols[kGnMaxL];
  __shared__ double s_miss;
  const int s = blockIdx.x, rep = blockIdx.y, sign = blockIdx.z;
  const int hY = sign, hW = 1 - sign;  // +k: primal of LEFT, shadow of RIGHT; -k: swapped
  const int sl = a.sl, sr = a.sr;
  double2* K = reinterpret_cast<double2*>(gn_smem);   // [sr][sl]
  double2* Gb = K + kGnMaxR * kGnMaxL;                 // [sr][sr]
  const int* rs = a.run_slot + (long long)rep * (sl + sr);
  const long long o_out = ((long long)rep * a.ne + s) * 2 + sign;
  if (threadIdx.x == 0) {
    int w = kOK;
    for (int c = 0; c < sl + sr; ++c) {
      const int st = a.sh[(long long)rs[c] * a.ne + s].status;
      if (st != kOK && w == kOK) w = st;
    }
    s_status = w;
  }
  __syncthreads();
  if (s_status != kOK) {
    if (threadIdx.x == 0) {
      a.T[o_out] = __longlong_as_double(0x7ff8000000000000LL);
      a.miss[o_out] = __longlong_as_double(0x7ff8000000000000LL);
      a.rank[o_out] = 0;
      a.status[o_out] = s_status;
    }
    return;
  }
  const long long nR = (long long)a.nrp * a.nxy, nL = (long long)a.nlp * a.nxy;
  V* xs = reinterpret_cast<V*>(a.XS);
  auto ycol = [&](int c) {
    return reinterpret_cast<double2*>(xs + (((long long)rs[c] * a.ne + s) * 2 + hY) * a.no);
  };
  auto wcol = [&](int i) -> const V* { return xs + (((long long)rs[sl + i] * a.ne + s) * 2 + hW) * a.no; };
  // Y = Gamma_R^1/2 x on the right-CAP planes, in place as complex FP64
  for (int c = 0; c < sl; ++c) {
    const V* yv = xs + (((long long)rs[c] * a.ne + s) * 2 + hY) * a.no;
    double2* y = ycol(c);
    for (long long u = threadIdx.x; u < nR; u += blockDim.x) {
      const double g = sqrt(a.gr[a.rplanes[u / a.nxy]]);
      const double2 xv = vload(yv, u);
      y[u] = make_double2(g * xv.x, g * xv.y);
    }
  }
  __syncthreads();
  // Q = orth(Y): classical Gram-Schmidt, twice per column; a column whose remaining
  // norm is below drop x its own norm lies in the span already and is skipped
  for (int c = 0; c < sl; ++c) {
    double2* y = ycol(c);
    {
      double v[1] = {0.0};
      for (long long u = threadIdx.x; u < nR; u += blockDim.x) v[0] += y[u].x * y[u].x + y[u].y * y[u].y;
      gn_block_sum<1>(v, s_red, red);
      if (threadIdx.x == 0) s_nrm0 = sqrt(s_red[0]);
      __syncthreads();
    }
    for (int pass = 0; pass < 2; ++pass) {
      for (int j0 = 0; j0 < c; j0 += kGnChunk) {
        double v[2 * kGnChunk];
#pragma unroll
        for (int k = 0; k < 2 * kGnChunk; ++k) v[k] = 0.0;
        for (long long u = threadIdx.x; u < nR; u += blockDim.x) {
          const double2 yv = y[u];
#pragma unroll
          for (int k = 0; k < kGnChunk; ++k) {
            const int j = j0 + k;
            if (j < c && s_keep[j]) {
              const double2 qv = ycol(j)[u];  // <q_j, y> = sum conj(q) y
              v[2 * k] += qv.x * yv.x + qv.y * yv.y;
              v[2 * k + 1] += qv.x * yv.y - qv.y * yv.x;
            }
          }
        }
        gn_block_sum<2 * kGnChunk>(v, s_red, red);
        if (threadIdx.x < kGnChunk && j0 + threadIdx.x < c)
          s_d[j0 + threadIdx.x] = make_double2(s_red[2 * threadIdx.x], s_red[2 * threadIdx.x + 1]);
        __syncthreads();
      }
      for (long long u = threadIdx.x; u < nR; u += blockDim.x) {
        double2 yv = y[u];
        for (int j = 0; j < c; ++j)
          if (s_keep[j]) yv = csub(yv, cmul(s_d[j], ycol(j)[u]));
        y[u] = yv;
      }
      __syncthreads();
    }
    double v[1] = {0.0};
    for (long long u = threadIdx.x; u < nR; u += blockDim.x) v[0] += y[u].x * y[u].x + y[u].y * y[u].y;
    gn_block_sum<1>(v, s_red, red);
    const double nrm = sqrt(s_red[0]);
    const int keep = nrm > a.drop * s_nrm0 && nrm > 0.0;
    if (c == sl - 1 && threadIdx.x == 0) s_miss = 4.0 * nrm * nrm;
    if (keep) {
      const double inv = 1.0 / nrm;
      for (long long u = threadIdx.x; u < nR; u += blockDim.x) y[u] = make_double2(inv * y[u].x, inv * y[u].y);
    }
    if (threadIdx.x == 0) s_keep[c] = keep;
    __syncthreads();
  }
  // K[i][c] = psi_i^T q_c (bilinear) for the kept columns.  With P-symmetric runs the
  // +k rows of W came from P_k x of the RIGHT runs, so they belong to the test vectors
  // P_k psi_i
  const double2* psi = a.rnd + ((long long)rep * 2 + 1) * a.smax * a.np;
  const bool mirror = a.psym && sign == 0;
  const double2* ph = a.phase + (size_t)(a.slots[rs[0]].ik * 2) * 2 * kPhaseN;
  for (int i = 0; i < sr; ++i) {
    const double2* pv = psi + (long long)i * a.np;
    for (int j0 = 0; j0 < sl; j0 += kGnChunk) {
      double v[2 * kGnChunk];
#pragma unroll
      for (int k = 0; k < 2 * kGnChunk; ++k) v[k] = 0.0;
      for (long long u = threadIdx.x; u < nR; u += blockDim.x) {
        double2 p = pv[u];
        if (mirror) {
          const long long pl = u / a.nxy;
          const int w = (int)(u - pl * a.nxy);
          const int y = w / a.nx, x = w - y * a.nx;
          p = pv[pl * a.nxy + (x ? a.nx - x : 0) + (long long)a.nx * (y ? a.ny - y : 0)];
          if (x) p = cmul(p, ph[kPhaseW - 1]);
          if (y) p = cmul(p, ph[kPhaseN + kPhaseW - 1]);
        }
#pragma unroll
        for (int k = 0; k < kGnChunk; ++k) {
          const int j = j0 + k;
          if (j < sl && s_keep[j]) {
            const double2 q = ycol(j)[u];
            v[2 * k] += p.x * q.x - p.y * q.y;
            v[2 * k + 1] += p.x * q.y + p.y * q.x;
          }
        }
      }
      gn_block_sum<2 * kGnChunk>(v, s_red, red);
      if (threadIdx.x < kGnChunk && j0 + threadIdx.x < sl)
        K[i * kGnMaxL + j0 + threadIdx.x] = make_double2(s_red[2 * threadIdx.x], s_red[2 * threadIdx.x + 1]);
      __syncthreads();
    }
  }
  // G_b[i][j] = sum_v w_i(v) conj(w_j(v)), w_i = Gamma_L^1/2 (kept planes of RIGHT run i)
  for (int i = 0; i < sr; ++i) {
    const V* wi = wcol(i);
    for (int j0 = i; j0 < sr; j0 += kGnChunk) {
      double v[2 * kGnChunk];
#pragma unroll
      for (int k = 0; k < 2 * kGnChunk; ++k) v[k] = 0.0;
      for (long long u = threadIdx.x; u < nL; u += blockDim.x) {
        const double g = a.gl[a.lplanes[u / a.nxy]];
        const double2 x = vload(wi, u);
#pragma unroll
        for (int k = 0; k < kGnChunk; ++k) {
          const int j = j0 + k;
          if (j < sr) {
            const double2 w = vload(wcol(j), u);
            v[2 * k] += g * (x.x * w.x + x.y * w.y);
            v[2 * k + 1] += g * (x.y * w.x - x.x * w.y);
          }
        }
      }
      gn_block_sum<2 * kGnChunk>(v, s_red, red);
      if (threadIdx.x < kGnChunk && j0 + threadIdx.x < sr) {
        const int j = j0 + threadIdx.x;
        const double2 g = make_double2(s_red[2 * threadIdx.x], s_red[2 * threadIdx.x + 1]);
        Gb[i * kGnMaxR + j] = g;
        Gb[j * kGnMaxR + i] = make_double2(g.x, -g.y);
      }
      __syncthreads();
    }
  }
  // small dense part (one thread, all in shared memory): Householder QR of K on the
  // kept columns (R_K in place in K), Z = Q_K^H G_b Q_K (in place in G_b), then
  // T = 4 trace(R_K^-1 Z R_K^-H)
  if (threadIdx.x == 0) {
    double2* v = s_v;
    int* cols = s_cols;
    int r = 0;
    for (int c = 0; c < sl; ++c)
      if (s_keep[c]) cols[r++] = c;
    const int m = sr;
    for (int t = 0; t < r; ++t) {
      // reflector H = I - 2 v v^H taking column cols[t] (rows t..m-1) to alpha e_t
      double nx = 0.0;
      for (int i = t; i < m; ++i) {
        const double2 k = K[i * kGnMaxL + cols[t]];
        nx += k.x * k.x + k.y * k.y;
      }
      nx = sqrt(nx);
      const double2 x0 = K[t * kGnMaxL + cols[t]];
      const double ax0 = hypot(x0.x, x0.y);
      const double2 ph = ax0 > 0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
      const double2 alpha = make_double2(-ph.x * nx, -ph.y * nx);  // -e^{i arg x0} ||x||
      for (int i = t; i < m; ++i) v[i] = K[i * kGnMaxL + cols[t]];
      v[t] = csub(v[t], alpha);
      double nv = 0.0;
      for (int i = t; i < m; ++i) nv += v[i].x * v[i].x + v[i].y * v[i].y;
      nv = sqrt(nv);
      if (nv > 0.0)
        for (int i = t; i < m; ++i) v[i] = make_double2(v[i].x / nv, v[i].y / nv);
      else
        for (int i = t; i < m; ++i) v[i] = make_double2(0.0, 0.0);
      for (int tt = t; tt < r; ++tt) {  // K <- H K on the kept columns
        double2 d = make_double2(0.0, 0.0);
        for (int i = t; i < m; ++i) {
          const double2 k = K[i * kGnMaxL + cols[tt]];
          d = cadd(d, make_double2(v[i].x * k.x + v[i].y * k.y, v[i].x * k.y - v[i].y * k.x));
        }
        for (int i = t; i < m; ++i) {
          double2& k = K[i * kGnMaxL + cols[tt]];
          k = csub(k, cmul(make_double2(2.0 * v[i].x, 2.0 * v[i].y), d));
        }
      }
      for (int j = 0; j < m; ++j) {  // G_b <- H G_b: rows t..m-1
        double2 d = make_double2(0.0, 0.0);
        for (int i = t; i < m; ++i) {
          const double2 g = Gb[i * kGnMaxR + j];
          d = cadd(d, make_double2(v[i].x * g.x + v[i].y * g.y, v[i].x * g.y - v[i].y * g.x));
        }
        for (int i = t; i < m; ++i)
          Gb[i * kGnMaxR + j] = csub(Gb[i * kGnMaxR + j], cmul(make_double2(2.0 * v[i].x, 2.0 * v[i].y), d));
      }
      for (int i = 0; i < m; ++i) {  // G_b <- G_b H = G_b - 2 (G_b v) v^H: columns t..m-1
        double2 d = make_double2(0.0, 0.0);
        for (int j = t; j < m; ++j) d = cadd(d, cmul(Gb[i * kGnMaxR + j], v[j]));
        for (int j = t; j < m; ++j)
          Gb[i * kGnMaxR + j] =
              csub(Gb[i * kGnMaxR + j], cmul(make_double2(2.0 * d.x, 2.0 * d.y), make_double2(v[j].x, -v[j].y)));
      }
    }
    // R_K[i][j] = K[i][cols[j]] (i <= j < r).  A1 = R^-1 Z by back substitution, in
    // place over Z = G_b[0:r][0:r]
    bool bad = false;
    for (int i = 0; i < r; ++i) {
      const double2 d = K[i * kGnMaxL + cols[i]];
      if (!(d.x != 0.0 || d.y != 0.0)) bad = true;
    }
    double tr = 0.0;
    if (!bad) {
      for (int j = 0; j < r; ++j)
        for (int i = r - 1; i >= 0; --i) {
          double2 acc = Gb[i * kGnMaxR + j];
          for (int l = i + 1; l < r; ++l) acc = csub(acc, cmul(K[i * kGnMaxL + cols[l]], Gb[l * kGnMaxR + j]));
          Gb[i * kGnMaxR + j] = cdiv(acc, K[i * kGnMaxL + cols[i]]);
        }
      // diagonal of R^-1 A1^H (its real part equals that of M2 = A1 R^-H, its conjugate
      // transpose): column j of A1^H is conj(row j of A1)
      for (int j = 0; j < r; ++j) {
        double2* col = v;
        for (int i = r - 1; i >= 0; --i) {
          const double2 aji = Gb[j * kGnMaxR + i];
          double2 acc = make_double2(aji.x, -aji.y);
          for (int l = i + 1; l < r; ++l) acc = csub(acc, cmul(K[i * kGnMaxL + cols[l]], col[l]));
          col[i] = cdiv(acc, K[i * kGnMaxL + cols[i]]);
        }
        tr += col[j].x;
      }
    }
    a.T[o_out] = bad ? __longlong_as_double(0x7ff8000000000000LL) : 4.0 * tr;
    a.miss[o_out] = s_miss;
    a.rank[o_out] = r;
    a.status[o_out] = bad ? kEBREAKDOWN : kOK;
  }
}

// double -> double-float copies of the operator tables
__global__ void k_real_to_df(const double* x, float2* y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const df d = df_split(x[i]);
    y[i] = make_float2(d.hi, d.lo);
  }
}
__global__ void k_cplx_to_df(const double2* x, float4* y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = dfc_from_double2(x[i]);
}

template <int R, bool ISO>
cudaError_t stencil_df_r(dim3 grid, int threads, size_t smem, cudaStream_t s, const StencilDfArgs& a, bool prepare,
                         int* blocks_per_sm) {
  if (blocks_per_sm)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_stencil_df<R, ISO>, threads, smem);
  if (prepare) {
    // all of the SM's unified memory as shared memory (the z-ring is large)
    cudaError_t e = cudaFuncSetAttribute(k_stencil_df<R, ISO>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_stencil_df<R, ISO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  k_stencil_df<R, ISO><<<grid, threads, smem, s>>>(a);
  return cudaSuccess;
}

template <bool ISO>
cudaError_t stencil_df_iso(int R, dim3 grid, int threads, size_t smem, cudaStream_t s, const StencilDfArgs& a,
                           bool prepare, int* bps) {
  switch (R) {
    case 1: return stencil_df_r<1, ISO>(grid, threads, smem, s, a, prepare, bps);
    case 2: return stencil_df_r<2, ISO>(grid, threads, smem, s, a, prepare, bps);
    case 3: return stencil_df_r<3, ISO>(grid, threads, smem, s, a, prepare, bps);
    case 4: return stencil_df_r<4, ISO>(grid, threads, smem, s, a, prepare, bps);
    case 5: return stencil_df_r<5, ISO>(grid, threads, smem, s, a, prepare, bps);
    case 6: return stencil_df_r<6, ISO>(grid, threads, smem, s, a, prepare, bps);
    default: return cudaErrorInvalidValue;
  }
}

// prepare = true sets the kernel's shared-memory limit; false launches it; with
// blocks_per_sm set, only the kernel's resident blocks per SM at (threads, smem) are
// returned.  iso: the three axes have the same spacing (one coefficient per distance)
cudaError_t stencil_df(int R, bool iso, dim3 grid, int threads, size_t smem, cudaStream_t s,
                       const StencilDfArgs& a, bool prepare, int* blocks_per_sm = nullptr) {
  return iso ? stencil_df_iso<true>(R, grid, threads, smem, s, a, prepare, blocks_per_sm)
             : stencil_df_iso<false>(R, grid, threads, smem, s, a, prepare, blocks_per_sm);
}

// Slabs per run for the double-float stencil when the caller sets no depth: the count
// whose launch of S runs best fills whole waves of resident blocks, each slab paying a
// 2R-plane prologue (about 3.6 planes of stencil time at order 12, measured).
int df_slabs(int S, int nz, int resident) {
  int best = 1;
  double best_cost = 1e300;
  for (int ns = 1; ns <= std::max(1, nz / 8); ++ns) {
    const int D = (nz + ns - 1) / ns;
    const long long blocks = (long long)S * ns;
    const long long waves = (blocks + resident - 1) / resident;
    const double cost = (double)waves * (D + 3.6);  // block-planes along the critical path
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = ns;
    }
  }
  return best;
}

// ---------------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------------

struct DevScope {
  int prev = -1;
  explicit DevScope(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(d);
  }
  ~DevScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int ms_fail(transec_ctx* ctx, int code, const std::string& msg) {
  ctx->err = msg;
  return code;
}

int ms_severity(int code) {
  switch (code) {
    case TRANSEC_OK: return 0;
    case TRANSEC_ENOCONV: return 1;
    case TRANSEC_EBREAKDOWN: return 2;
    case TRANSEC_ETIMEOUT: return 3;
    default: return 4;
  }
}

#define MS_CK(call)                                                                     \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      cudaGetLastError();                                                               \
      return ms_fail(ctx, e_ == cudaErrorMemoryAllocation ? TRANSEC_ENOMEM : TRANSEC_ECUDA, \
                     std::string(#call) + ": " + cudaGetErrorString(e_));               \
    }                                                                                   \
  } while (0)

// (Re)allocate p to hold `need` elements unless its capacity `have` suffices.
template <typename P>
cudaError_t grow(P*& p, size_t have, size_t need) {
  if (have >= need && p) return cudaSuccess;
  cudaFree(p);
  p = nullptr;
  return cudaMalloc(&p, std::max<size_t>(need, 1) * sizeof(P));
}

// One solve of the multi-shift engine: items run to completion (every shift converged
// or stopped), per-shift vectors left in the buffers for the reductions.
// psym: P-symmetric COCG (one half per run; double-float form, the plane in one tile).
int run_sweep(transec_ctx* ctx, const std::vector<MsItem>& items, const std::vector<double>& energies,
              double e0, int S, int nrep, int smax, unsigned long long seed, double** d_res_t,
              int** d_res_it, int** d_res_st, bool psym = false) {
  SweepBufs& B = *ctx->sweep;
  const Geometry& g = ctx->g;
  const bool dfm = ctx->opts.precision == TRANSEC_PREC_DF64;  // double-float kernels
  const int H = psym ? 1 : 2;
  const int ne = (int)energies.size();
  const int nitems = (int)items.size();
  const long long n = g.n, nxy = g.nxy;
  const int nlp = (int)ctx->lplanes.size(), nrp = (int)ctx->rplanes.size();
  const long long no = (long long)std::max(nlp, nrp) * nxy;
  // the double-float stencil's default depth fills whole waves of resident blocks
  // (df_slabs); the FP64 stencil keeps the tile chooser's default
  TileShape ts = choose_tiles(g, H, sizeof(double2), dfm ? kDfThreads : StencilMax<double>::threads,
                              ctx->opts.tile_y, ctx->opts.slab > 0 ? ctx->opts.slab : (dfm ? 64 : 0));
  bool iso = true;
  for (int m = 1; m <= g.R; ++m) iso = iso && g.kx[m] == g.ky[m] && g.kx[m] == g.kz[m];
  const size_t smem_df = stencil_df_smem(g.R, ts.TX, ts.TY, H, ts.threads);
  if (dfm) {
    MS_CK(stencil_df(g.R, iso, dim3(1), 0, smem_df, ctx->s, StencilDfArgs{}, true));
    if (ctx->opts.slab <= 0) {
      int bps = 0, sms = 0;
      MS_CK(stencil_df(g.R, iso, dim3(1), ts.threads, smem_df, ctx->s, StencilDfArgs{}, false, &bps));
      MS_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
      const int ns = df_slabs(S * ts.ntx * ts.nty, g.nz, std::max(1, bps) * std::max(1, sms));
      ts = choose_tiles(g, H, sizeof(double2), kDfThreads, ctx->opts.tile_y, (g.nz + ns - 1) / ns);
    }
  }
  if (psym && (!dfm || ts.ntx != 1 || ts.nty != 1 || ts.TX != g.nx || ts.TY != g.ny))
    return ms_fail(ctx, TRANSEC_EINVAL, "P-symmetric runs need the double-float form and a plane in one tile");
  const int nblk_st = ts.ntx * ts.nty * ts.nslab;
  // blocks per run of the vector update: the double-float update sets up its scalars
  // in FP64 once per thread, so it takes more points per thread (about 8 blocks per SM
  // over all runs)
  const int nblk3 = dfm ? (int)std::max(4LL, std::min((n + 256 * 8 - 1) / (256 * 8), (152LL * 8 + S - 1) / S))
                        : (int)std::min(1024LL, (n + 256 * 8 - 1) / (256 * 8));
  const long long np = no;
  const size_t need_vec = (size_t)S * 2 * n, need_shv = (size_t)S * ne * 2 * no;
  const size_t need_rnd = (size_t)std::max(1, nrep) * 2 * std::max(1, smax) * np;
  MS_CK(grow(B.R, B.cap_vec, need_vec));
  MS_CK(grow(B.P0, B.cap_vec, need_vec));
  MS_CK(grow(B.P1, B.cap_vec, need_vec));
  MS_CK(grow(B.Q, B.cap_vec, need_vec));
  B.cap_vec = std::max(B.cap_vec, need_vec);
  MS_CK(grow(B.XS, B.cap_shv, need_shv));
  MS_CK(grow(B.PS, B.cap_shv, need_shv));
  B.cap_shv = std::max(B.cap_shv, need_shv);
  MS_CK(grow(B.sig_part, B.cap_sig, (size_t)S * nblk_st * 2));
  B.cap_sig = std::max(B.cap_sig, (size_t)S * nblk_st * 2);
  MS_CK(grow(B.rho_part, B.cap_rho, (size_t)S * nblk3 * 4));
  B.cap_rho = std::max(B.cap_rho, (size_t)S * nblk3 * 4);
  MS_CK(grow(B.slots, B.cap_slots, (size_t)S));
  MS_CK(grow(B.ms, B.cap_slots, (size_t)S));
  MS_CK(grow(B.escale, B.cap_slots, (size_t)S));
  B.cap_slots = std::max(B.cap_slots, (size_t)S);
  MS_CK(grow(B.sh, B.cap_shs, (size_t)S * ne));
  MS_CK(grow(B.coef, B.cap_shs, (size_t)S * ne));
  B.cap_shs = std::max(B.cap_shs, (size_t)S * ne);
  MS_CK(grow(B.items, B.cap_items, (size_t)nitems));
  B.cap_items = std::max(B.cap_items, (size_t)nitems);
  MS_CK(grow(B.energies, B.cap_ene, (size_t)ne));
  B.cap_ene = std::max(B.cap_ene, (size_t)ne);
  MS_CK(grow(B.rnd, B.cap_rnd, need_rnd));
  B.cap_rnd = std::max(B.cap_rnd, need_rnd);
  MS_CK(grow(B.lrank, B.cap_nz, (size_t)g.nz));
  MS_CK(grow(B.rrank, B.cap_nz, (size_t)g.nz));
  MS_CK(grow(B.gam_df, B.cap_nz, (size_t)g.nz));
  B.cap_nz = std::max(B.cap_nz, (size_t)g.nz);
  MS_CK(grow(B.v_df, B.cap_n, (size_t)n));
  B.cap_n = std::max(B.cap_n, (size_t)n);
  const size_t nph = (size_t)ctx->nk * 2 * 2 * kPhaseN;
  MS_CK(grow(B.phase_df, B.cap_ph, nph));
  B.cap_ph = std::max(B.cap_ph, nph);
  if (!B.queue) MS_CK(cudaMalloc(&B.queue, sizeof(Queue)));
  B.S = S; B.ne = ne; B.n = n; B.no = no; B.nblk_st = nblk_st; B.nblk3 = nblk3; B.nitems = nitems;
  B.nrnd = nrep;
  cudaStream_t st = ctx->s;
  std::vector<int> lr(g.nz, -1), rr(g.nz, -1);
  for (int i = 0; i < nlp; ++i) lr[ctx->lplanes[i]] = i;
  for (int i = 0; i < nrp; ++i) rr[ctx->rplanes[i]] = i;
  MS_CK(cudaMemcpyAsync(B.lrank, lr.data(), g.nz * sizeof(int), cudaMemcpyHostToDevice, st));
  MS_CK(cudaMemcpyAsync(B.rrank, rr.data(), g.nz * sizeof(int), cudaMemcpyHostToDevice, st));
  if (dfm) {
    k_real_to_df<<<256, 256, 0, st>>>(ctx->d_v, B.v_df, n);
    k_real_to_df<<<1, 256, 0, st>>>(ctx->d_gam, B.gam_df, g.nz);
    k_cplx_to_df<<<1, 256, 0, st>>>(ctx->d_phase, B.phase_df, (long long)nph);
    ctx->launches += 3;
  }
  MS_CK(cudaMemcpyAsync(B.items, items.data(), nitems * sizeof(MsItem), cudaMemcpyHostToDevice, st));
  MS_CK(cudaMemcpyAsync(B.energies, energies.data(), ne * sizeof(double), cudaMemcpyHostToDevice, st));
  Queue q0{};
  q0.nitems = nitems;
  MS_CK(cudaMemcpyAsync(B.queue, &q0, sizeof(Queue), cudaMemcpyHostToDevice, st));
  MS_CK(cudaMemsetAsync(B.slots, 0, (size_t)S * sizeof(Slot), st));
  if (nrep > 0) {
    RandomArgs ra{B.rnd, nrep, smax, np, seed};
    k_ms_random<<<1024, 256, 0, st>>>(ra);
    ctx->launches += 1;
  }
  // results of UNIT runs
  double* res_t = nullptr;
  int *res_it = nullptr, *res_st = nullptr;
  MS_CK(cudaMalloc(&res_t, (size_t)std::max(1, nitems) * ne * 2 * sizeof(double)));
  MS_CK(cudaMalloc(&res_it, (size_t)std::max(1, nitems) * ne * sizeof(int)));
  MS_CK(cudaMalloc(&res_st, (size_t)std::max(1, nitems) * ne * sizeof(int)));
  *d_res_t = res_t;
  *d_res_it = res_it;
  *d_res_st = res_st;

  MsArgs a{};
  a.slots = B.slots; a.ms = B.ms; a.sh = B.sh; a.coef = B.coef; a.queue = B.queue; a.items = B.items;
  a.energies = B.energies; a.e0 = e0; a.S = S; a.ne = ne; a.nk = ctx->nk;
  a.R = B.R; a.P0 = B.P0; a.XS = B.XS; a.PS = B.PS; a.rnd = B.rnd; a.smax = smax; a.np = np;
  a.n = n; a.no = no; a.nxy = nxy; a.lplanes = ctx->d_lplanes; a.rplanes = ctx->d_rplanes;
  a.lrank = B.lrank; a.rrank = B.rrank; a.nlp = nlp; a.nrp = nrp; a.gl = ctx->d_gl; a.gr = ctx->d_gr;
  a.rho_part = B.rho_part; a.nblk3 = nblk3; a.sig_part = B.sig_part; a.nblk_st = nblk_st;
  a.tol = ctx->opts.tol; a.maxit = ctx->opts.maxit; a.escale = B.escale;
  a.stall_its = dfm ? ctx->opts.df_stall_its : 0;
  a.H = H; a.psym = psym ? 1 : 0; a.nx = g.nx; a.ny = g.ny; a.phase = ctx->d_phase;
  a.res_t = res_t; a.res_it = res_it; a.res_st = res_st;

  if (!dfm) MS_CK(prepare_stencil<double>(g.R, ts.smem));
  StencilDfArgs da{};
  da.r = reinterpret_cast<const float4*>(B.R); da.q = reinterpret_cast<float4*>(B.Q); da.part = B.sig_part;
  da.slots = B.slots; da.escale = B.escale; da.phase = B.phase_df; da.v = B.v_df; da.gam = B.gam_df;
  for (int m = 0; m <= kMaxR; ++m) {
    const df x = df_split(g.kx[m]), y = df_split(g.ky[m]), z = df_split(g.kz[m]);
    da.kx[m] = make_float2(x.hi, x.lo);
    da.ky[m] = make_float2(y.hi, y.lo);
    da.kz[m] = make_float2(z.hi, z.lo);
  }
  da.diag_c = g.diag_c; da.nx = g.nx; da.ny = g.ny; da.nz = g.nz; da.nxy = g.nxy; da.n = g.n; da.H = H;
  da.TX = ts.TX; da.TY = ts.TY; da.D = ts.D; da.ntx = ts.ntx; da.conj = 0; da.slot_stride = H * n;
  da.psym = psym ? 1 : 0;
  UpdateDfArgs dua{};
  dua.r = reinterpret_cast<float4*>(B.R); dua.q = reinterpret_cast<const float4*>(B.Q); dua.sig_part = B.sig_part;
  dua.sig_nblk = nblk_st; dua.rho_part = B.rho_part; dua.slots = B.slots; dua.escale = B.escale; dua.n = n;
  dua.slot_stride = 2 * n; dua.H = 2;
  UpdateDfPsymArgs dpa{};
  dpa.r = dua.r; dpa.q = dua.q; dpa.sig_part = B.sig_part; dpa.sig_nblk = nblk_st; dpa.rho_part = B.rho_part;
  dpa.slots = B.slots; dpa.escale = B.escale; dpa.phase = B.phase_df; dpa.nx = g.nx; dpa.ny = g.ny;
  dpa.nxy = nxy; dpa.n = n; dpa.slot_stride = n;
  StencilArgs<double> sa{};
  sa.r = B.R; sa.q = B.Q; sa.part = B.sig_part; sa.slots = B.slots; sa.phase = ctx->d_phase;
  sa.v = ctx->d_v; sa.gam = ctx->d_gam; sa.g = g; sa.H = 2; sa.TX = ts.TX; sa.TY = ts.TY; sa.D = ts.D;
  sa.ntx = ts.ntx; sa.conj = 0; sa.slot_stride = 2 * n; sa.insts = nullptr; sa.tile_idx = 0;
  const dim3 sgrid((unsigned)(ts.ntx * ts.nty), (unsigned)ts.nslab, (unsigned)S);
  UpdateArgs<double> ua{};
  ua.x = nullptr; ua.r = B.R; ua.q = B.Q; ua.sig_part = B.sig_part; ua.sig_nblk = nblk_st;
  ua.rho_part = B.rho_part; ua.slots = B.slots; ua.n = n; ua.slot_stride = 2 * n; ua.H = 2;
  ua.insts = nullptr;
  const dim3 ugrid((unsigned)nblk3, (unsigned)S);
  const dim3 shgrid((unsigned)((no + 255) / 256), (unsigned)ne, (unsigned)S);
  const dim3 igrid((unsigned)std::min<long long>((n + 255) / 256, 1024), (unsigned)S);
  const dim3 isgrid((unsigned)std::min<long long>((2 * no + 255) / 256, 256), (unsigned)ne, (unsigned)S);

  // the queue's refill stage: assignment, vectors, per-shift state, rho_0
  auto refill = [&]() {
    k_ms_assign<<<1, 32, 0, st>>>(a);
    if (dfm) k_ms_init<float4><<<igrid, 256, 0, st>>>(a);
    else k_ms_init<double2><<<igrid, 256, 0, st>>>(a);
    k_ms_init_shift<<<isgrid, 256, 0, st>>>(a);
    if (dfm) k_ms_rho0<float4><<<S, 256, 0, st>>>(a);
    else k_ms_rho0<double2><<<S, 256, 0, st>>>(a);
  };
  refill();
  MS_CK(cudaGetLastError());
  ctx->launches += 4;

  const int C = ctx->opts.chunk;
  const bool prof = ctx->opts.profile != 0;
  if (prof) {
    while ((int)ctx->prof_ev.size() < 4 * C) {
      cudaEvent_t e;
      MS_CK(cudaEventCreate(&e));
      ctx->prof_ev.push_back(e);
    }
  }
  const bool device_loop = !prof && !ctx->opts.host_loop;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle loop{};
  if (device_loop) {
    MS_CK(cudaGraphCreate(&graph, 0));
    cudaError_t eh = cudaGraphConditionalHandleCreate(&loop, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (eh == cudaSuccess) eh = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    if (eh == cudaSuccess)
      eh = cudaStreamBeginCaptureToGraph(st, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal);
    if (eh != cudaSuccess) {
      cudaGraphDestroy(graph);
      cudaGetLastError();
      return ms_fail(ctx, TRANSEC_ECUDA, std::string("device loop set-up: ") + cudaGetErrorString(eh));
    }
  } else {
    MS_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  }
  for (int i = 0; i < C; ++i) {
    sa.p_in = (i % 2 == 0) ? B.P0 : B.P1;
    sa.p_out = (i % 2 == 0) ? B.P1 : B.P0;
    da.p_in = reinterpret_cast<const float4*>(sa.p_in);
    da.p_out = reinterpret_cast<float4*>(sa.p_out);
    if (prof) cudaEventRecordWithFlags(ctx->prof_ev[4 * i + 0], st, cudaEventRecordExternal);
    if (dfm) stencil_df(g.R, iso, sgrid, ts.threads, smem_df, st, da, false);
    else launch_stencil<double>(g.R, sgrid, ts.threads, ts.smem, st, sa);
    if (prof) cudaEventRecordWithFlags(ctx->prof_ev[4 * i + 1], st, cudaEventRecordExternal);
    k_ms_coef<<<S, 256, 0, st>>>(a);
    if (prof) cudaEventRecordWithFlags(ctx->prof_ev[4 * i + 2], st, cudaEventRecordExternal);
    if (dfm) k_ms_shift_df<<<shgrid, 256, 0, st>>>(a);
    else k_ms_shift<<<shgrid, 256, 0, st>>>(a);
    if (prof) cudaEventRecordWithFlags(ctx->prof_ev[4 * i + 3], st, cudaEventRecordExternal);
    ua.p = sa.p_out;
    if (psym) k_update_df_psym<<<ugrid, 256, 0, st>>>(dpa);
    else if (dfm) k_update_df<<<ugrid, 256, 0, st>>>(dua);
    else k_update<double><<<ugrid, 256, 0, st>>>(ua);
    k_ms_scalars<<<S, 256, 0, st>>>(a);
  }
  if (dfm) k_ms_trace<float4><<<dim3((unsigned)ne, (unsigned)S), 256, 0, st>>>(a);
  else k_ms_trace<double2><<<dim3((unsigned)ne, (unsigned)S), 256, 0, st>>>(a);
  k_ms_release<<<1, 32, 0, st>>>(a);
  refill();
  if (device_loop) {
    k_continue<<<1, 1, 0, st>>>(loop, B.queue);
  } else {
    cudaMemcpyAsync(ctx->h_harvest, &B.queue->harvested, sizeof(int), cudaMemcpyDeviceToHost, st);
  }
  {
    cudaGraph_t captured = nullptr;
    cudaError_t e1 = cudaStreamEndCapture(st, &captured);
    if (!device_loop) graph = captured;
    if (e1 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return ms_fail(ctx, TRANSEC_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e1));
    }
  }
  {
    cudaError_t e2 = cudaGraphInstantiate(&exec, graph, 0);
    if (e2 != cudaSuccess) {
      cudaGraphDestroy(graph);
      cudaGetLastError();
      return ms_fail(ctx, TRANSEC_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
    }
  }
  const long long per_chunk = 5LL * C + 6 + (device_loop ? 1 : 0);
  const long long max_chunks =
      ((long long)nitems / std::max(1, S) + 2) * ((long long)ctx->opts.maxit / C + 2) + 16;
  const int per_launch = 4096;
  long long chunks = 0;
  int rcode = TRANSEC_OK;
  *ctx->h_harvest = 0;
  while (true) {
    cudaError_t e3 = cudaSuccess;
    if (device_loop) {
      const int lim = (int)std::min<long long>(chunks + per_launch, 1LL << 30);
      e3 = cudaMemcpyAsync(&B.queue->limit, &lim, sizeof(int), cudaMemcpyHostToDevice, st);
      if (e3 == cudaSuccess) e3 = cudaGraphLaunch(exec, st);
      Queue qh{};
      if (e3 == cudaSuccess) e3 = cudaMemcpyAsync(&qh, B.queue, sizeof(Queue), cudaMemcpyDeviceToHost, st);
      if (e3 == cudaSuccess) e3 = cudaStreamSynchronize(st);
      if (e3 == cudaSuccess) {
        chunks = qh.chunks;
        *ctx->h_harvest = qh.harvested;
      }
    } else {
      e3 = cudaGraphLaunch(exec, st);
      if (e3 == cudaSuccess) e3 = cudaStreamSynchronize(st);
      if (e3 == cudaSuccess) ++chunks;
    }
    if (e3 != cudaSuccess) {
      cudaGetLastError();
      rcode = ms_fail(ctx, TRANSEC_ECUDA, std::string("multi-shift chunk: ") + cudaGetErrorString(e3));
      break;
    }
    if (prof) {
      for (int i = 0; i < C; ++i) {
        float t0 = 0.f, t1 = 0.f;
        if (cudaEventElapsedTime(&t0, ctx->prof_ev[4 * i], ctx->prof_ev[4 * i + 1]) == cudaSuccess) {
          (dfm ? ctx->sweep_stencil_df_ms : ctx->sweep_stencil_ms) += t0;
          (dfm ? ctx->sweep_stencil_df_launches : ctx->sweep_stencil_launches) += 1;
        }
        if (cudaEventElapsedTime(&t1, ctx->prof_ev[4 * i + 2], ctx->prof_ev[4 * i + 3]) == cudaSuccess) {
          (dfm ? ctx->sweep_shift_df_ms : ctx->sweep_shift_ms) += t1;
          (dfm ? ctx->sweep_shift_df_launches : ctx->sweep_shift_launches) += 1;
        }
      }
      cudaGetLastError();
    }
    if (*ctx->h_harvest >= nitems) break;
    if (chunks > max_chunks) {
      rcode = ms_fail(ctx, TRANSEC_ETIMEOUT, "multi-shift solve did not drain its queue within the iteration bound");
      break;
    }
  }
  ctx->launches += chunks * per_chunk;
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  // work counters: seed iterations per run and shifted point updates
  if (rcode == TRANSEC_OK) {
    std::vector<MsShift> hsh((size_t)S * ne);
    std::vector<Slot> hsl(S);
    // the per-run iteration count is the largest stop iteration of its shifts; runs
    // left in slots (the sketch keeps them) are read here, UNIT runs from the results
    if (cudaMemcpy(hsh.data(), B.sh, hsh.size() * sizeof(MsShift), cudaMemcpyDeviceToHost) == cudaSuccess) {
      for (int s2 = 0; s2 < S; ++s2) {
        int mx = 0;
        for (int e = 0; e < ne; ++e) {
          mx = std::max(mx, hsh[(size_t)s2 * ne + e].conv_it);
          ctx->sweep_shift_points += (long long)hsh[(size_t)s2 * ne + e].conv_it * H * (long long)std::max(nlp, nrp) * nxy;
        }
        ctx->sweep_iters += mx;
      }
    }
    cudaGetLastError();
  }
  return rcode;
}

}  // namespace

namespace {

// Results of one multi-shift call, row-major [item or k group][energy].
struct SweepOut {
  std::vector<double> t, tm, miss;
  std::vector<int> it, st, rank;
};

// Runs in flight for UNIT items: enough point-halves to fill the GPU, bounded by memory.
long long unit_slots(transec_ctx* ctx, int ne, int nitems) {
  const long long n = ctx->g.n;
  const long long no = (long long)std::max(ctx->lplanes.size(), ctx->rplanes.size()) * ctx->g.nxy;
  const size_t per_slot = (size_t)4 * 2 * n * 16 + (size_t)2 * ne * 2 * no * 16;
  long long S = ctx->opts.slots > 0 ? ctx->opts.slots : std::max(1LL, (24LL << 20) / (2 * n));
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) S = std::min<long long>(S, std::max<long long>(1, fr / 2 / per_slot));
  return std::max(1LL, std::min<long long>(S, nitems));
}

double seed_energy(const std::vector<double>& es) {
  std::vector<double> sorted = es;
  std::sort(sorted.begin(), sorted.end());
  return sorted[sorted.size() / 2];
}

// Unit columns (k index, left-CAP column) at the energies es, in the context's
// precision.  Outputs [item][energy].
int columns_solve(transec_ctx* ctx, const std::vector<double>& es, const std::vector<int>& ik,
                  const std::vector<long long>& cols, SweepOut& out) {
  const int ne = (int)es.size(), nitems = (int)ik.size();
  std::vector<MsItem> items(nitems);
  for (int i = 0; i < nitems; ++i) items[i] = MsItem{ik[i], RUN_UNIT, 0, 0, cols[i]};
  if (!ctx->sweep) ctx->sweep = new SweepBufs();
  double* rt = nullptr;
  int *rit = nullptr, *rst = nullptr;
  const int S = (int)unit_slots(ctx, ne, nitems);
  int rc = run_sweep(ctx, items, es, seed_energy(es), S, 0, 0, 0ULL, &rt, &rit, &rst);
  if (rc == TRANSEC_OK) {
    const size_t m = (size_t)nitems * ne;
    std::vector<double> t(2 * m);
    out.it.assign(m, 0);
    out.st.assign(m, 0);
    cudaError_t e = cudaMemcpy(t.data(), rt, t.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out.it.data(), rit, m * sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out.st.data(), rst, m * sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      cudaGetLastError();
      rc = ms_fail(ctx, TRANSEC_ECUDA, std::string("multi-shift results: ") + cudaGetErrorString(e));
    } else {
      out.t.resize(m);
      out.tm.resize(m);
      for (size_t u = 0; u < m; ++u) {
        out.t[u] = t[2 * u];
        out.tm[u] = t[2 * u + 1];
      }
    }
  }
  cudaFree(rt);
  cudaFree(rit);
  cudaFree(rst);
  return rc;
}

// Full trace T(E, k), T(E, -k) of the k groups ik by the two-sided sketch, in the
// context's precision (psym: P-symmetric COCG runs).  Outputs [group][energy].
int sketch_solve(transec_ctx* ctx, const std::vector<double>& es, const std::vector<int>& ik, int s_left,
                 int s_right, unsigned long long seed, SweepOut& out, bool psym = false) {
  const int ne = (int)es.size(), nrep = (int)ik.size();
  const int per = s_left + s_right;
  std::vector<MsItem> items;
  std::vector<int> run_slot((size_t)nrep * per);
  for (int r = 0; r < nrep; ++r) {
    for (int i = 0; i < s_left; ++i) {
      run_slot[(size_t)r * per + i] = (int)items.size();
      items.push_back(MsItem{ik[r], RUN_LEFT, r, i, 0});
    }
    for (int i = 0; i < s_right; ++i) {
      run_slot[(size_t)r * per + s_left + i] = (int)items.size();
      items.push_back(MsItem{ik[r], RUN_RIGHT, r, i, 0});
    }
  }
  // every run keeps its slot (and its kept planes) until the reduction: S = runs
  const int S = (int)items.size();
  if (!ctx->sweep) ctx->sweep = new SweepBufs();
  double* rt = nullptr;
  int *rit = nullptr, *rst = nullptr;
  int rc = run_sweep(ctx, items, es, seed_energy(es), S, nrep, std::max(s_left, s_right), seed, &rt, &rit, &rst,
                     psym);
  cudaFree(rt);
  cudaFree(rit);
  cudaFree(rst);
  if (rc != TRANSEC_OK) return rc;
  SweepBufs& B = *ctx->sweep;
  int *d_rs = nullptr, *d_rank = nullptr, *d_st = nullptr;
  double *d_T = nullptr, *d_miss = nullptr;
  const size_t nout = (size_t)nrep * ne * 2;
  cudaError_t e = cudaMalloc(&d_rs, run_slot.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&d_T, nout * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_miss, nout * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_rank, nout * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&d_st, nout * sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_rs, run_slot.data(), run_slot.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->s);
  const size_t smem = (size_t)(kGnMaxR * kGnMaxL + kGnMaxR * kGnMaxR) * sizeof(double2);
  const bool dfm = ctx->opts.precision == TRANSEC_PREC_DF64;
  if (e == cudaSuccess)
    e = dfm ? cudaFuncSetAttribute(k_ms_gn<float4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
            : cudaFuncSetAttribute(k_ms_gn<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaEvent_t g0 = nullptr, g1 = nullptr;
  const bool prof = ctx->opts.profile != 0;
  if (e == cudaSuccess && prof) {
    cudaEventCreate(&g0);
    cudaEventCreate(&g1);
    cudaEventRecord(g0, ctx->s);
  }
  if (e == cudaSuccess && psym) {
    MsArgs fa{};
    fa.slots = B.slots; fa.ms = B.ms; fa.XS = B.XS; fa.ne = ne; fa.no = B.no; fa.nxy = ctx->g.nxy;
    fa.nlp = (int)ctx->lplanes.size(); fa.nrp = (int)ctx->rplanes.size(); fa.nx = ctx->g.nx; fa.ny = ctx->g.ny;
    fa.phase = ctx->d_phase;
    const dim3 fgrid((unsigned)((B.no + 255) / 256), (unsigned)ne, (unsigned)S);
    k_ms_psym_fill<float4><<<fgrid, 256, 0, ctx->s>>>(fa);
    ctx->launches += 1;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    GnArgs ga{};
    ga.XS = B.XS; ga.sh = B.sh; ga.run_slot = d_rs; ga.rnd = B.rnd; ga.smax = std::max(s_left, s_right);
    ga.np = B.no; ga.no = B.no; ga.nxy = ctx->g.nxy; ga.ne = ne; ga.sl = s_left; ga.sr = s_right;
    ga.lplanes = ctx->d_lplanes; ga.rplanes = ctx->d_rplanes; ga.nlp = (int)ctx->lplanes.size();
    ga.nrp = (int)ctx->rplanes.size(); ga.gl = ctx->d_gl; ga.gr = ctx->d_gr; ga.T = d_T; ga.rank = d_rank;
    ga.status = d_st; ga.drop = 1e-13; ga.miss = d_miss;
    ga.psym = psym ? 1 : 0; ga.nx = ctx->g.nx; ga.ny = ctx->g.ny; ga.slots = B.slots; ga.phase = ctx->d_phase;
    if (dfm) k_ms_gn<float4><<<dim3((unsigned)ne, (unsigned)nrep, 2), 256, smem, ctx->s>>>(ga);
    else k_ms_gn<double2><<<dim3((unsigned)ne, (unsigned)nrep, 2), 256, smem, ctx->s>>>(ga);
    ctx->launches += 1;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && prof) cudaEventRecord(g1, ctx->s);
  std::vector<double> T(nout), miss(nout);
  std::vector<int> rk(nout), stt(nout);
  if (e == cudaSuccess) e = cudaMemcpyAsync(T.data(), d_T, nout * sizeof(double), cudaMemcpyDeviceToHost, ctx->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(miss.data(), d_miss, nout * sizeof(double), cudaMemcpyDeviceToHost, ctx->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rk.data(), d_rank, nout * sizeof(int), cudaMemcpyDeviceToHost, ctx->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(stt.data(), d_st, nout * sizeof(int), cudaMemcpyDeviceToHost, ctx->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->s);
  if (e == cudaSuccess && prof) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g0, g1) == cudaSuccess) ctx->sweep_reduce_ms += ms;
  }
  if (g0) cudaEventDestroy(g0);
  if (g1) cudaEventDestroy(g1);
  // seed iterations per group: the longest run of the group
  std::vector<MsShift> hsh((size_t)S * ne);
  if (e == cudaSuccess) e = cudaMemcpy(hsh.data(), B.sh, hsh.size() * sizeof(MsShift), cudaMemcpyDeviceToHost);
  cudaFree(d_rs);
  cudaFree(d_T);
  cudaFree(d_miss);
  cudaFree(d_rank);
  cudaFree(d_st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ms_fail(ctx, TRANSEC_ECUDA, std::string("sketch reduction: ") + cudaGetErrorString(e));
  }
  const size_t m = (size_t)nrep * ne;
  out.t.resize(m);
  out.tm.resize(m);
  out.miss.resize(m);
  out.rank.resize(m);
  out.st.resize(m);
  out.it.resize(m);
  for (int r = 0; r < nrep; ++r)
    for (int s = 0; s < ne; ++s) {
      const size_t o = ((size_t)r * ne + s) * 2;
      const size_t u = (size_t)r * ne + s;
      out.t[u] = T[o];
      out.tm[u] = T[o + 1];
      out.miss[u] = std::max(miss[o], miss[o + 1]);
      out.rank[u] = std::min(rk[o], rk[o + 1]);
      out.st[u] = ms_severity(stt[o]) >= ms_severity(stt[o + 1]) ? stt[o] : stt[o + 1];
      int mx = 0;
      for (int c = 0; c < per; ++c) mx = std::max(mx, hsh[(size_t)run_slot[(size_t)r * per + c] * ne + s].conv_it);
      out.it[u] = mx;
    }
  return TRANSEC_OK;
}

bool redo_status(int st) { return st == TRANSEC_ENOCONV || st == TRANSEC_EBREAKDOWN; }

// Energies (as indices into es) and rows (items or k groups) of a [row][energy] status
// table that failed; empty when none did.
void failed_parts(const std::vector<int>& st, int nrows, int ne, std::vector<int>& rows, std::vector<int>& cols) {
  rows.clear();
  cols.clear();
  std::vector<char> ce(ne, 0);
  for (int r = 0; r < nrows; ++r) {
    bool any = false;
    for (int s = 0; s < ne; ++s)
      if (redo_status(st[(size_t)r * ne + s])) {
        any = true;
        ce[s] = 1;
      }
    if (any) rows.push_back(r);
  }
  for (int s = 0; s < ne; ++s)
    if (ce[s]) cols.push_back(s);
}

// Runs f with the context's precision set to FP64, restoring it afterwards.
template <typename F>
int in_fp64(transec_ctx* ctx, F f) {
  const int saved = ctx->opts.precision;
  ctx->opts.precision = TRANSEC_PREC_FP64;
  const int rc = f();
  ctx->opts.precision = saved;
  return rc;
}

}  // namespace

extern "C" {

int transec_shifted_columns(transec_ctx* ctx, int ne, const double* energies, int nitems, const int* ik,
                            const int64_t* cols, double* t_out, double* t_minus_out, int* iters_out,
                            int* status_out) {
  if (!ctx) return TRANSEC_EINVAL;
  if (!ctx->have_v || !ctx->have_abc || !ctx->have_k)
    return ms_fail(ctx, TRANSEC_ESTATE, "potential, absorbing boundary and k-mesh must be set");
  if (ne < 1 || ne > 1024 || nitems < 0 || !energies || (nitems > 0 && (!ik || !cols || !t_out)))
    return ms_fail(ctx, TRANSEC_EINVAL, "bad multi-shift arguments (1 <= ne <= 1024)");
  if (nitems == 0) return TRANSEC_OK;
  const long long nrhs = (long long)ctx->lplanes.size() * ctx->g.nxy;
  for (int e = 0; e < ne; ++e)
    if (!std::isfinite(energies[e])) return ms_fail(ctx, TRANSEC_EINVAL, "non-finite energy");
  for (int i = 0; i < nitems; ++i) {
    if (ik[i] < 0 || ik[i] >= ctx->nk) return ms_fail(ctx, TRANSEC_EINVAL, "k index out of range");
    if (cols[i] < 0 || cols[i] >= nrhs) return ms_fail(ctx, TRANSEC_EINVAL, "column out of range");
  }
  if (ctx->rplanes.empty()) return ms_fail(ctx, TRANSEC_EINVAL, "right absorbing profile is zero everywhere");
  DevScope ds(ctx->device);
  MS_CK(cudaStreamSynchronize(ctx->user));
  const std::vector<double> es(energies, energies + ne);
  const std::vector<int> hik(ik, ik + nitems);
  const std::vector<long long> hc(cols, cols + nitems);
  SweepOut out;
  int rc = columns_solve(ctx, es, hik, hc, out);
  if (rc != TRANSEC_OK) return rc;
  // double-float results that did not converge: the failed items again in FP64 at the
  // energies that failed for any of them
  std::vector<int> rows, ecols;
  if (ctx->opts.precision == TRANSEC_PREC_DF64) failed_parts(out.st, nitems, ne, rows, ecols);
  if (!rows.empty()) {
    std::vector<double> e2;
    std::vector<int> k2;
    std::vector<long long> c2;
    for (int s : ecols) e2.push_back(es[s]);
    for (int r : rows) {
      k2.push_back(hik[r]);
      c2.push_back(hc[r]);
    }
    SweepOut o2;
    rc = in_fp64(ctx, [&] { return columns_solve(ctx, e2, k2, c2, o2); });
    if (rc != TRANSEC_OK) return rc;
    for (size_t a = 0; a < rows.size(); ++a)
      for (size_t b = 0; b < ecols.size(); ++b) {
        const size_t u = (size_t)rows[a] * ne + ecols[b], v = a * ecols.size() + b;
        if (!redo_status(out.st[u])) continue;
        out.t[u] = o2.t[v];
        out.tm[u] = o2.tm[v];
        out.st[u] = o2.st[v];
        out.it[u] += o2.it[v];
        ctx->sweep_fp64_redone += 1;
      }
  }
  int worst = TRANSEC_OK;
  for (size_t u = 0; u < (size_t)nitems * ne; ++u) {
    t_out[u] = out.t[u];
    if (t_minus_out) t_minus_out[u] = out.tm[u];
    if (iters_out) iters_out[u] = out.it[u];
    if (status_out) status_out[u] = out.st[u];
    if (ms_severity(out.st[u]) > ms_severity(worst)) worst = out.st[u];
  }
  if (worst != TRANSEC_OK) ctx->err = std::string("some columns failed: ") + transec_status_string(worst);
  return worst;
}

int transec_transmission_sketch(transec_ctx* ctx, int ne, const double* energies, int nrep, const int* ik,
                                int s_left, int s_right, unsigned long long seed, double* T_out,
                                double* T_minus_out, int* rank_out, int* status_out, int* iters_out,
                                double* miss_out) {
  if (!ctx) return TRANSEC_EINVAL;
  if (!ctx->have_v || !ctx->have_abc || !ctx->have_k)
    return ms_fail(ctx, TRANSEC_ESTATE, "potential, absorbing boundary and k-mesh must be set");
  if (ne < 1 || ne > 1024 || nrep < 0 || !energies || (nrep > 0 && (!ik || !T_out)))
    return ms_fail(ctx, TRANSEC_EINVAL, "bad sketch arguments (1 <= ne <= 1024)");
  if (s_left < 1 || s_left > kGnMaxL || s_right < s_left || s_right > kGnMaxR)
    return ms_fail(ctx, TRANSEC_EINVAL, "sketch sizes must satisfy 1 <= s_left <= 32, s_left <= s_right <= 64");
  if (nrep == 0) return TRANSEC_OK;
  for (int e = 0; e < ne; ++e)
    if (!std::isfinite(energies[e])) return ms_fail(ctx, TRANSEC_EINVAL, "non-finite energy");
  for (int r = 0; r < nrep; ++r)
    if (ik[r] < 0 || ik[r] >= ctx->nk) return ms_fail(ctx, TRANSEC_EINVAL, "k index out of range");
  if (ctx->rplanes.empty()) return ms_fail(ctx, TRANSEC_EINVAL, "right absorbing profile is zero everywhere");
  const bool psym = ctx->opts.psym != 0;
  if (psym) {
    if (ctx->opts.precision != TRANSEC_PREC_DF64)
      return ms_fail(ctx, TRANSEC_EINVAL, "P-symmetric runs are built in the double-float form (precision 2)");
    if (!(ctx->v_inversion_gap <= kPsymTol))
      return ms_fail(ctx, TRANSEC_EINVAL, "the potential is not invariant under the in-plane inversion about grid "
                                          "point (0, 0)");
  }
  DevScope ds(ctx->device);
  MS_CK(cudaStreamSynchronize(ctx->user));
  const std::vector<double> es(energies, energies + ne);
  const std::vector<int> hik(ik, ik + nrep);
  SweepOut out;
  int rc = sketch_solve(ctx, es, hik, s_left, s_right, seed, out, psym);
  if (rc != TRANSEC_OK) return rc;
  // double-float results that did not converge: the failed k groups again with FP64
  // runs at the energies that failed for any of them (a fresh random draw)
  std::vector<int> rows, ecols;
  if (ctx->opts.precision == TRANSEC_PREC_DF64) failed_parts(out.st, nrep, ne, rows, ecols);
  if (!rows.empty()) {
    std::vector<double> e2;
    std::vector<int> k2;
    for (int s : ecols) e2.push_back(es[s]);
    for (int r : rows) k2.push_back(hik[r]);
    SweepOut o2;
    rc = in_fp64(ctx, [&] { return sketch_solve(ctx, e2, k2, s_left, s_right, seed ^ 0x5DEECE66DULL, o2); });
    if (rc != TRANSEC_OK) return rc;
    for (size_t a = 0; a < rows.size(); ++a)
      for (size_t b = 0; b < ecols.size(); ++b) {
        const size_t u = (size_t)rows[a] * ne + ecols[b], v = a * ecols.size() + b;
        if (!redo_status(out.st[u])) continue;
        out.t[u] = o2.t[v];
        out.tm[u] = o2.tm[v];
        out.miss[u] = o2.miss[v];
        out.rank[u] = o2.rank[v];
        out.st[u] = o2.st[v];
        out.it[u] += o2.it[v];
        ctx->sweep_fp64_redone += 1;
      }
  }
  // the a-posteriori checks acting: results whose independent +-k estimates disagree by
  // more than the guard, or whose sketch may miss more than the guard of T (the energy
  // of M outside the span of all but the last LEFT column), are computed again with a
  // sketch of twice the sizes (for P-symmetric runs only the second check applies)
  const double guard = ctx->opts.sketch_guard;
  for (int round = 0; guard > 0 && round < 3; ++round) {
    std::vector<int> st2((size_t)nrep * ne, TRANSEC_OK);
    bool any = false;
    for (size_t u = 0; u < st2.size(); ++u)
      if (out.st[u] == TRANSEC_OK &&
          (!(out.miss[u] <= guard) || (!psym && !(std::fabs(out.t[u] - out.tm[u]) <= guard)))) {
        st2[u] = TRANSEC_ENOCONV;  // marks the result for failed_parts
        any = true;
      }
    if (!any || (s_left >= kGnMaxL && s_right >= kGnMaxR)) break;
    s_left = std::min(2 * s_left, kGnMaxL);
    s_right = std::max(s_left, std::min(2 * s_right, kGnMaxR));
    failed_parts(st2, nrep, ne, rows, ecols);
    std::vector<double> e3;
    std::vector<int> k3;
    for (int s : ecols) e3.push_back(es[s]);
    for (int r : rows) k3.push_back(hik[r]);
    SweepOut o3;
    rc = sketch_solve(ctx, e3, k3, s_left, s_right, splitmix64(seed + 0x9E37ULL * (round + 1)), o3, psym);
    if (rc != TRANSEC_OK) return rc;
    for (size_t a = 0; a < rows.size(); ++a)
      for (size_t b = 0; b < ecols.size(); ++b) {
        const size_t u = (size_t)rows[a] * ne + ecols[b], v = a * ecols.size() + b;
        if (st2[u] == TRANSEC_OK) continue;
        out.it[u] += o3.it[v];
        if (o3.st[v] != TRANSEC_OK) continue;  // keep the smaller sketch's estimate
        out.t[u] = o3.t[v];
        out.tm[u] = o3.tm[v];
        out.miss[u] = o3.miss[v];
        out.rank[u] = o3.rank[v];
        ctx->sweep_guard_redone += 1;
      }
  }
  int worst = TRANSEC_OK;
  for (size_t u = 0; u < (size_t)nrep * ne; ++u) {
    T_out[u] = out.t[u];
    if (T_minus_out) T_minus_out[u] = out.tm[u];
    if (rank_out) rank_out[u] = out.rank[u];
    if (status_out) status_out[u] = out.st[u];
    if (iters_out) iters_out[u] = out.it[u];
    if (miss_out) miss_out[u] = out.miss[u];
    if (ms_severity(out.st[u]) > ms_severity(worst)) worst = out.st[u];
  }
  if (worst != TRANSEC_OK) ctx->err = std::string("some (E, k) failed: ") + transec_status_string(worst);
  return worst;
}

}  // extern "C"
