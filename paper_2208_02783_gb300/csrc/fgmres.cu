// Flexible GMRES(m) with the U-Net as right preconditioner, and the trainer that fits the
// network to one operator family A(E, k) = E - H_k + i Gamma.
//
// FGMRES, for one column: A x = e_j.  Arnoldi step i applies the preconditioner to the
// basis vector v_i (z_i = M(v_i), with M the network on every `net_every`-th step and
// the identity on the others, or the identity throughout when no network is given), the
// FP64 stencil to z_i (w = A z_i), and orthogonalises w against v_0..v_i by classical
// Gram-Schmidt applied twice; the small least-squares problem is solved with Givens
// rotations on the host.  After m steps x += Z y and the cycle restarts from the true
// residual.  M changes nothing about A, so an accepted x meets ||e_j - A x|| <= tol in
// FP64 whatever the network does.  A column whose residual has not halved over the last
// 10 cycles, that reaches maxit applications, or whose Hessenberg matrix turns singular
// (a zero preconditioned direction) is handed to the plain FP64 Krylov engine.
//
// Training pairs (r, e) with r = A e, at a random energy of the window and a random k of
// the mesh, from one of two sources:
//   0: e is a seeded random complex field (normal values smoothed by 0..8 passes of a
//      [1 2 1]/4 filter per axis, so that its spectrum ranges from white to smooth);
//   1: e = x* - x_i for the iterates x_i of a transpose-BiCG solve of one random
//      left-CAP column (x* its converged solution; x_0 = 0 gives e = x*, r = e_j): the
//      residuals a Krylov solver hands to the preconditioner.
// The network sees (s_r Re r, s_r Im r, V - E, Gamma) and is fitted to s_e e under the
// relative L2 loss, with s_r, s_e scaling r and e to unit RMS: FGMRES needs only the
// direction of z_i.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <random>
#include <string>
#include <vector>

#include "engine.cuh"

namespace transec {
template <typename T>
cudaError_t prepare_stencil(int R, size_t smem);
}

using namespace transec;

namespace {

using cplx = std::complex<double>;

#define FG_GS(i, n) \
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// partial dots sum conj(V_j) w (Hermitian, conj = 1) or sum V_j w (bilinear, conj = 0);
// grid (blocks, count), 256 threads
__global__ void __launch_bounds__(256) k_fg_dots(const double2* V, const double2* w, long long n, int conj,
                                                 double* part) {
  const int j = blockIdx.y;
  const double2* v = V + (long long)j * n;
  const double sg = conj ? -1.0 : 1.0;
  double sr = 0.0, si = 0.0;
  FG_GS(i, n) {
    const double2 a = v[i], b = w[i];
    sr += a.x * b.x - sg * a.y * b.y;
    si += a.x * b.y + sg * a.y * b.x;
  }
  __shared__ double red[2][8];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    si += __shfl_down_sync(0xffffffffu, si, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { red[0][wid] = sr; red[1][wid] = si; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int k = 0; k < 8; ++k) { a += red[0][k]; b += red[1][k]; }
    part[((long long)j * gridDim.x + blockIdx.x) * 2] = a;
    part[((long long)j * gridDim.x + blockIdx.x) * 2 + 1] = b;
  }
}

// w += sum_j c_j V_j
__global__ void k_fg_axpy(double2* w, const double2* V, const double2* c, int count, long long n) {
  FG_GS(i, n) {
    double2 acc = w[i];
    for (int j = 0; j < count; ++j) {
      const double2 v = V[(long long)j * n + i], cj = c[j];
      acc.x += cj.x * v.x - cj.y * v.y;
      acc.y += cj.x * v.y + cj.y * v.x;
    }
    w[i] = acc;
  }
}

// p = r + beta p
__global__ void k_fg_xpby(double2* p, const double2* r, double2 beta, long long n) {
  FG_GS(i, n) {
    const double2 a = p[i];
    p[i] = make_double2(r[i].x + beta.x * a.x - beta.y * a.y, r[i].y + beta.x * a.y + beta.y * a.x);
  }
}

// d = a - b
__global__ void k_fg_sub(double2* d, const double2* a, const double2* b, long long n) {
  FG_GS(i, n) d[i] = make_double2(a[i].x - b[i].x, a[i].y - b[i].y);
}

__global__ void k_fg_unit(double2* v, long long j, long long n) {
  FG_GS(i, n) v[i] = make_double2(i == j ? 1.0 : 0.0, 0.0);
}

__global__ void k_fg_scale(double2* out, const double2* w, double s, long long n) {
  FG_GS(i, n) out[i] = make_double2(w[i].x * s, w[i].y * s);
}

// r = e_j - q (in place allowed)
__global__ void k_fg_residual(double2* r, const double2* q, long long j, long long n) {
  FG_GS(i, n) r[i] = make_double2((i == j ? 1.0 : 0.0) - q[i].x, -q[i].y);
}

// network input per voxel: (s Re v, s Im v, V - E, Gamma)
__global__ void k_fg_input(const double2* v, double s, const double* pot, double e, const double* gam,
                           long long nxy, float* in, long long n) {
  FG_GS(i, n) {
    in[4 * i + 0] = (float)(v[i].x * s);
    in[4 * i + 1] = (float)(v[i].y * s);
    in[4 * i + 2] = (float)(pot[i] - e);
    in[4 * i + 3] = (float)gam[i / nxy];
  }
}

__global__ void k_fg_output(const float* o, double2* z, long long n) {
  FG_GS(i, n) z[i] = make_double2(o[2 * i], o[2 * i + 1]);
}

__global__ void k_fg_target(const double2* x, double s, float* t, long long n) {
  FG_GS(i, n) {
    t[2 * i] = (float)(x[i].x * s);
    t[2 * i + 1] = (float)(x[i].y * s);
  }
}

// splitmix64 finaliser (Steele, Lea and Flood, 2014) as a counter-based generator
__device__ inline unsigned long long fg_mix(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// x[i] = two independent standard normals (Box-Muller) from the counter (key, i)
__global__ void k_fg_noise(double2* x, unsigned long long key, long long n) {
  FG_GS(i, n) {
    const unsigned long long a = fg_mix(key ^ fg_mix(2 * (unsigned long long)i));
    const unsigned long long b = fg_mix(key ^ fg_mix(2 * (unsigned long long)i + 1));
    const double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740992.0);  // (0, 1]
    const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);          // [0, 1)
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    x[i] = make_double2(rad * cs, rad * sn);
  }
}

// one [1 2 1]/4 pass along axis (0 = x, 1 = y: periodic; 2 = z: zero outside)
__global__ void k_fg_smooth(const double2* in, double2* out, int axis, int nx, int ny, int nz, long long n) {
  FG_GS(i, n) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
    long long lo, hi;
    bool has_lo = true, has_hi = true;
    if (axis == 0) {
      lo = i - x + (x + nx - 1) % nx;
      hi = i - x + (x + 1) % nx;
    } else if (axis == 1) {
      lo = i + (long long)(((y + ny - 1) % ny) - y) * nx;
      hi = i + (long long)(((y + 1) % ny) - y) * nx;
    } else {
      lo = i - (long long)nx * ny;
      hi = i + (long long)nx * ny;
      has_lo = z > 0;
      has_hi = z + 1 < nz;
    }
    const double2 a = in[i];
    double2 r = make_double2(0.5 * a.x, 0.5 * a.y);
    if (has_lo) { r.x += 0.25 * in[lo].x; r.y += 0.25 * in[lo].y; }
    if (has_hi) { r.x += 0.25 * in[hi].x; r.y += 0.25 * in[hi].y; }
    out[i] = r;
  }
}

struct DBuf {
  void* p = nullptr;
  ~DBuf() { if (p) cudaFree(p); }
};

// work arrays of one FGMRES or training call
struct Fg {
  transec_ctx* ctx = nullptr;
  long long n = 0;
  int nb = 152;
  unsigned eg = 0;  // grid of the elementwise kernels
  double2 *V = nullptr, *Z = nullptr, *w = nullptr, *x = nullptr, *pscr = nullptr, *coef = nullptr;
  double* part = nullptr;
  float *in = nullptr, *out = nullptr;
  Slot* slot = nullptr;
  double* spart = nullptr;
  TileShape ts{};
  DBuf b[14];
  cudaError_t e = cudaSuccess;
  void* alloc(int k, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(&b[k].p, bytes);
    return e == cudaSuccess ? b[k].p : nullptr;
  }
};

int fg_fail(transec_ctx* ctx, int code, const std::string& msg) {
  ctx->err = msg;
  return code;
}

int fg_cuda(transec_ctx* ctx, cudaError_t e, const char* what) {
  cudaGetLastError();
  return fg_fail(ctx, e == cudaErrorMemoryAllocation ? TRANSEC_ENOMEM : TRANSEC_ECUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

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

// buffers for restart length m
cudaError_t fg_setup(Fg& f, transec_ctx* ctx, int m) {
  f.ctx = ctx;
  f.n = ctx->g.n;
  f.eg = (unsigned)std::min<long long>((f.n + 255) / 256, 152LL * 16);
  f.ts = choose_tiles(ctx->g, 1, sizeof(double2), StencilMax<double>::threads, ctx->opts.tile_y, ctx->opts.slab);
  const size_t vb = (size_t)f.n * sizeof(double2);
  f.V = (double2*)f.alloc(0, (size_t)(m + 1) * vb);
  f.Z = (double2*)f.alloc(1, (size_t)m * vb);
  f.w = (double2*)f.alloc(2, vb);
  f.x = (double2*)f.alloc(3, vb);
  f.pscr = (double2*)f.alloc(4, vb);
  f.coef = (double2*)f.alloc(5, (size_t)(m + 1) * sizeof(double2));
  f.part = (double*)f.alloc(6, (size_t)(m + 1) * f.nb * 2 * sizeof(double));
  f.in = (float*)f.alloc(7, (size_t)f.n * 4 * sizeof(float));
  f.out = (float*)f.alloc(8, (size_t)f.n * 2 * sizeof(float));
  f.slot = (Slot*)f.alloc(9, sizeof(Slot));
  f.spart = (double*)f.alloc(10, (size_t)f.ts.ntx * f.ts.nty * f.ts.nslab * 2 * sizeof(double));
  f.alloc(11, sizeof(long long));
  f.alloc(12, sizeof(double));
  if (f.e == cudaSuccess) f.e = prepare_stencil<double>(ctx->g.R, f.ts.smem);
  return f.e;
}

// q = A(E, k) v for one FP64 vector (the stencil in argument mode with beta = 0)
cudaError_t apply_A(Fg& f, double e, int ik, const double2* v, double2* q, int transpose = 0) {
  transec_ctx* ctx = f.ctx;
  Slot hs{};
  hs.status = SLOT_ACTIVE;
  hs.ik = ik;
  hs.e = e;
  hs.beta = make_double2(0.0, 0.0);
  cudaError_t err = cudaMemcpyAsync(f.slot, &hs, sizeof(Slot), cudaMemcpyHostToDevice, ctx->s);
  if (err != cudaSuccess) return err;
  StencilArgs<double> sa{};
  sa.r = v; sa.p_in = v; sa.p_out = f.pscr; sa.q = q; sa.part = f.spart; sa.slots = f.slot;
  sa.phase = ctx->d_phase; sa.v = ctx->d_v; sa.gam = ctx->d_gam; sa.g = ctx->g; sa.H = 1;
  sa.TX = f.ts.TX; sa.TY = f.ts.TY; sa.D = f.ts.D; sa.ntx = f.ts.ntx; sa.conj = transpose; sa.slot_stride = f.n;
  launch_stencil<double>(ctx->g.R, dim3(f.ts.ntx * f.ts.nty, f.ts.nslab, 1), f.ts.threads, f.ts.smem,
                         ctx->s, sa);
  ctx->launches += 1;
  ctx->point_applies += f.n;
  return cudaGetLastError();
}

// h[j] = <V_j, w> for j < count (partial sums on the device, final sum on the host in a
// fixed order)
cudaError_t dots(Fg& f, const double2* V, int count, const double2* w, std::vector<cplx>& h, int conj = 1) {
  k_fg_dots<<<dim3(f.nb, count), 256, 0, f.ctx->s>>>(V, w, f.n, conj, f.part);
  f.ctx->launches += 1;
  std::vector<double> hp((size_t)count * f.nb * 2);
  cudaError_t e = cudaMemcpyAsync(hp.data(), f.part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                  f.ctx->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(f.ctx->s);
  h.assign(count, cplx(0, 0));
  for (int j = 0; j < count; ++j)
    for (int b = 0; b < f.nb; ++b)
      h[j] += cplx(hp[((size_t)j * f.nb + b) * 2], hp[((size_t)j * f.nb + b) * 2 + 1]);
  return e;
}

double norm2(Fg& f, const double2* w, cudaError_t& e) {
  std::vector<cplx> h;
  e = dots(f, w, 1, w, h);
  return std::sqrt(std::max(0.0, h[0].real()));
}

// w += sum_j c_j V_j
cudaError_t axpy(Fg& f, double2* w, const double2* V, const std::vector<cplx>& c) {
  std::vector<double2> hc(c.size());
  for (size_t j = 0; j < c.size(); ++j) hc[j] = make_double2(c[j].real(), c[j].imag());
  cudaError_t e = cudaMemcpyAsync(f.coef, hc.data(), hc.size() * sizeof(double2), cudaMemcpyHostToDevice,
                                  f.ctx->s);
  if (e != cudaSuccess) return e;
  k_fg_axpy<<<f.eg, 256, 0, f.ctx->s>>>(w, V, f.coef, (int)c.size(), f.n);
  f.ctx->launches += 1;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(f.ctx->s);  // coef is reused by the next call
  return e;
}

// z = M(v): the network on (s v, V - E, Gamma) with s = sqrt(n) (v has unit norm), or a copy
int precondition(Fg& f, transec_unet* net, double E, const double2* v, double2* z) {
  transec_ctx* ctx = f.ctx;
  if (!net) {
    cudaError_t e = cudaMemcpyAsync(z, v, (size_t)f.n * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->s);
    return e == cudaSuccess ? TRANSEC_OK : fg_cuda(ctx, e, "preconditioner copy");
  }
  k_fg_input<<<f.eg, 256, 0, ctx->s>>>(v, std::sqrt((double)f.n), ctx->d_v, E, ctx->d_gam, ctx->g.nxy, f.in,
                                       f.n);
  ctx->launches += 1;
  cudaError_t e = cudaStreamSynchronize(ctx->s);
  if (e != cudaSuccess) return fg_cuda(ctx, e, "preconditioner input");
  const int rc = transec_unet_forward(net, f.in, f.out, 1);
  if (rc != TRANSEC_OK) return fg_fail(ctx, rc, std::string("network: ") + transec_unet_last_error(net));
  k_fg_output<<<f.eg, 256, 0, ctx->s>>>(f.out, z, f.n);
  ctx->launches += 1;
  return TRANSEC_OK;
}

int check_net(transec_ctx* ctx, const transec_unet* net) {
  if (!net) return TRANSEC_OK;
  int nx = 0, ny = 0, nz = 0;
  transec_unet_dims(net, &nx, &ny, &nz);
  if (nx != ctx->g.nx || ny != ctx->g.ny || nz != ctx->g.nz)
    return fg_fail(ctx, TRANSEC_EINVAL, "network volume differs from the grid");
  return TRANSEC_OK;
}

// one column by FGMRES(m): OK (solution in f.x), ENOCONV (stalled or maxit reached),
// EBREAKDOWN, or a CUDA / network error
int fgmres_column(Fg& f, transec_unet* net, int every, double E, int k, long long j, int m, int maxit,
                  int& applies) {
  transec_ctx* ctx = f.ctx;
  const double tol = ctx->opts.tol;
  cudaError_t e = cudaMemsetAsync(f.x, 0, (size_t)f.n * sizeof(double2), ctx->s);
  if (e != cudaSuccess) return fg_cuda(ctx, e, "fgmres");
  std::vector<double> cycle_beta;
  std::vector<cplx> H((size_t)(m + 1) * m), g(m + 1), cs(m), sn(m), h, hh, y;
  while (true) {
    // true residual r = e_j - A x; v_0 = r / beta
    e = apply_A(f, E, k, f.x, f.w);
    if (e != cudaSuccess) return fg_cuda(ctx, e, "fgmres apply");
    k_fg_residual<<<f.eg, 256, 0, ctx->s>>>(f.w, f.w, j, f.n);
    ctx->launches += 1;
    const double beta = norm2(f, f.w, e);
    if (e != cudaSuccess) return fg_cuda(ctx, e, "fgmres norm");
    if (!std::isfinite(beta)) return fg_fail(ctx, TRANSEC_EBREAKDOWN, "fgmres: non-finite residual");
    if (beta <= tol) return TRANSEC_OK;
    cycle_beta.push_back(beta);
    const size_t c = cycle_beta.size();
    if (applies >= maxit || (c > 10 && beta > 0.5 * cycle_beta[c - 11])) return TRANSEC_ENOCONV;
    k_fg_scale<<<f.eg, 256, 0, ctx->s>>>(f.V, f.w, 1.0 / beta, f.n);
    ctx->launches += 1;
    std::fill(H.begin(), H.end(), cplx(0, 0));
    std::fill(g.begin(), g.end(), cplx(0, 0));
    g[0] = beta;
    int i = 0;
    while (i < m && applies < maxit) {
      double2* vi = f.V + (long long)i * f.n;
      double2* zi = f.Z + (long long)i * f.n;
      int rc = precondition(f, i % every == 0 ? net : nullptr, E, vi, zi);
      if (rc != TRANSEC_OK) return rc;
      e = apply_A(f, E, k, zi, f.w);
      if (e != cudaSuccess) return fg_cuda(ctx, e, "fgmres apply");
      ++applies;
      h.assign(i + 1, cplx(0, 0));
      for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
        e = dots(f, f.V, i + 1, f.w, hh);
        if (e != cudaSuccess) return fg_cuda(ctx, e, "fgmres dots");
        for (int q = 0; q <= i; ++q) { h[q] += hh[q]; hh[q] = -hh[q]; }
        e = axpy(f, f.w, f.V, hh);
        if (e != cudaSuccess) return fg_cuda(ctx, e, "fgmres axpy");
      }
      const double hn = norm2(f, f.w, e);
      if (e != cudaSuccess) return fg_cuda(ctx, e, "fgmres norm");
      for (int q = 0; q <= i; ++q) H[(size_t)q * m + i] = h[q];
      if (hn > 0) {
        k_fg_scale<<<f.eg, 256, 0, ctx->s>>>(f.V + (long long)(i + 1) * f.n, f.w, 1.0 / hn, f.n);
        ctx->launches += 1;
      }
      // the earlier rotations, then the one that zeroes the subdiagonal entry hn
      for (int q = 0; q < i; ++q) {
        const cplx a = H[(size_t)q * m + i], b = H[(size_t)(q + 1) * m + i];
        H[(size_t)q * m + i] = std::conj(cs[q]) * a + std::conj(sn[q]) * b;
        H[(size_t)(q + 1) * m + i] = -sn[q] * a + cs[q] * b;
      }
      const cplx a = H[(size_t)i * m + i];
      const double den = std::sqrt(std::norm(a) + hn * hn);
      cs[i] = den > 0 ? a / den : cplx(1, 0);
      sn[i] = den > 0 ? cplx(hn / den, 0) : cplx(0, 0);
      H[(size_t)i * m + i] = den;
      g[i + 1] = -sn[i] * g[i];
      g[i] = std::conj(cs[i]) * g[i];
      ++i;
      if (std::abs(g[i]) <= 0.5 * tol || hn == 0) break;
    }
    // y = R^-1 g, x += Z y
    y.assign(i, cplx(0, 0));
    for (int q = i - 1; q >= 0; --q) {
      cplx s = g[q];
      for (int c2 = q + 1; c2 < i; ++c2) s -= H[(size_t)q * m + c2] * y[c2];
      const cplx d = H[(size_t)q * m + q];
      if (std::abs(d) == 0) return fg_fail(ctx, TRANSEC_EBREAKDOWN, "fgmres: singular Hessenberg");
      y[q] = s / d;
    }
    if (i > 0) {
      e = axpy(f, f.x, f.Z, y);
      if (e != cudaSuccess) return fg_cuda(ctx, e, "fgmres update");
    }
  }
}

}  // namespace

extern "C" int transec_fgmres_columns(transec_ctx* ctx, transec_unet* net, int net_every, int nitems,
                                      const double* energies,
                                      const int* ik, const int64_t* cols, int restart, int maxit,
                                      double* t_out, int* iters_out, int* status_out, int* fallback_out) {
  if (!ctx) return TRANSEC_EINVAL;
  if (!ctx->have_v || !ctx->have_abc || !ctx->have_k)
    return fg_fail(ctx, TRANSEC_ESTATE, "potential, absorbing boundary and k-mesh must be set");
  if (nitems < 0 || restart < 1 || restart > 100 || maxit < 1 || net_every < 1)
    return fg_fail(ctx, TRANSEC_EINVAL, "bad fgmres arguments");
  if (nitems == 0) return TRANSEC_OK;
  if (!energies || !ik || !cols || !t_out) return fg_fail(ctx, TRANSEC_EINVAL, "NULL argument");
  int rc = check_net(ctx, net);
  if (rc) return rc;
  DevScope ds(ctx->device);
  cudaStreamSynchronize(ctx->user);
  Fg f;
  if (fg_setup(f, ctx, restart) != cudaSuccess) return fg_cuda(ctx, f.e, "fgmres set-up");
  const long long nrhs = (long long)ctx->lplanes.size() * ctx->g.nxy;
  int worst = TRANSEC_OK;
  for (int it = 0; it < nitems; ++it) {
    const double E = energies[it];
    const int k = ik[it];
    const long long col = cols[it];
    int status = TRANSEC_OK, applies = 0;
    bool fell = false;
    double t = std::nan("");
    if (k < 0 || k >= ctx->nk || col < 0 || col >= nrhs || !std::isfinite(E)) {
      status = TRANSEC_EINVAL;
    } else {
      const long long j = (long long)ctx->lplanes[col / ctx->g.nxy] * ctx->g.nxy + col % ctx->g.nxy;
      status = fgmres_column(f, net, net_every, E, k, j, restart, maxit, applies);
      if (status == TRANSEC_OK) {
        // t_j = 4 Gamma_L(j) sum_i Gamma_R(i) |x_i|^2 from the FP64 solution
        VecTraceArgs va{};
        va.x = f.x; va.cols = (const long long*)f.b[11].p; va.lplanes = ctx->d_lplanes;
        va.rplanes = ctx->d_rplanes; va.nlp = (int)ctx->lplanes.size(); va.nrp = (int)ctx->rplanes.size();
        va.gl = ctx->d_gl; va.gr = ctx->d_gr; va.t_out = (double*)f.b[12].p; va.nxy = ctx->g.nxy; va.n = f.n;
        const long long c64 = col;
        cudaError_t e = cudaMemcpyAsync(f.b[11].p, &c64, sizeof(long long), cudaMemcpyHostToDevice, ctx->s);
        k_vec_trace<<<1, 256, 0, ctx->s>>>(va);
        ctx->launches += 1;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&t, f.b[12].p, sizeof(double), cudaMemcpyDeviceToHost, ctx->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->s);
        if (e != cudaSuccess) return fg_cuda(ctx, e, "fgmres trace");
      } else if (status == TRANSEC_ENOCONV || status == TRANSEC_EBREAKDOWN) {
        // fallback (no progress, maxit, or a degenerate preconditioned direction): the
        // plain FP64 Krylov engine solves the column
        fell = true;
        int itp = 0, stp = 0;
        const int prec = ctx->opts.precision;
        ctx->opts.precision = TRANSEC_PREC_FP64;
        const int64_t c64 = col;
        const int r2 = transec_column_contributions(ctx, 1, &E, &k, &c64, &t, nullptr, &itp, &stp, 0);
        ctx->opts.precision = prec;
        if (r2 != TRANSEC_OK && r2 != TRANSEC_ENOCONV && r2 != TRANSEC_EBREAKDOWN) return r2;
        status = stp;
        applies += itp;
      } else {
        return status;  // a CUDA or network failure: the context's message says which
      }
    }
    if (status != TRANSEC_OK) t = std::nan("");
    t_out[it] = t;
    if (iters_out) iters_out[it] = applies;
    if (status_out) status_out[it] = status;
    if (fallback_out) fallback_out[it] = fell ? 1 : 0;
    if (status != TRANSEC_OK && (worst == TRANSEC_OK || status < worst)) worst = status;
  }
  if (worst != TRANSEC_OK) ctx->err = "some columns failed (see status_out)";
  return worst;
}

namespace {

// Transpose BiCG for A x = e_j (shadow system A^T x~ = e_j, bilinear forms; COCG when A
// is complex symmetric), keeping every `every`-th iterate in `bank` (at most K; when the
// bank fills, every other one is dropped and the spacing doubles).  On convergence the
// solution is left in f.x and the iterates stored are counted in `stored`.
int bicg_bank(Fg& f, double E, int k, long long j, double2* bank, int K, int& stored) {
  transec_ctx* ctx = f.ctx;
  const long long n = f.n;
  double2 *r = f.V, *rt = f.V + n, *p = f.V + 2 * n, *pt = f.V + 3 * n, *q = f.V + 4 * n, *qt = f.V + 5 * n;
  k_fg_unit<<<f.eg, 256, 0, ctx->s>>>(r, j, n);
  k_fg_unit<<<f.eg, 256, 0, ctx->s>>>(rt, j, n);
  k_fg_unit<<<f.eg, 256, 0, ctx->s>>>(p, j, n);
  k_fg_unit<<<f.eg, 256, 0, ctx->s>>>(pt, j, n);
  ctx->launches += 4;
  cudaError_t e = cudaMemsetAsync(f.x, 0, (size_t)n * sizeof(double2), ctx->s);
  if (e != cudaSuccess) return fg_cuda(ctx, e, "training solve");
  e = cudaMemsetAsync(bank, 0, (size_t)n * sizeof(double2), ctx->s);  // x_0 = 0: e_0 = x*
  if (e != cudaSuccess) return fg_cuda(ctx, e, "training bank");
  cplx rho(1.0, 0.0);
  int every = 2;
  stored = 1;
  std::vector<cplx> h;
  for (int it = 0; it < ctx->opts.maxit; ++it) {
    e = apply_A(f, E, k, p, q, 0);
    if (e == cudaSuccess) e = apply_A(f, E, k, pt, qt, 1);
    if (e == cudaSuccess) e = dots(f, pt, 1, q, h, 0);
    if (e != cudaSuccess) return fg_cuda(ctx, e, "training solve");
    if (std::abs(h[0]) == 0) return TRANSEC_EBREAKDOWN;
    const cplx alpha = rho / h[0];
    if ((e = axpy(f, f.x, p, {alpha})) != cudaSuccess || (e = axpy(f, r, q, {-alpha})) != cudaSuccess ||
        (e = axpy(f, rt, qt, {-alpha})) != cudaSuccess)
      return fg_cuda(ctx, e, "training solve");
    if (it % every == 0) {
      if (stored == K) {  // keep every other iterate and double the spacing
        for (int q2 = 1; q2 < K / 2; ++q2)
          e = cudaMemcpyAsync(bank + (long long)q2 * n, bank + (long long)(2 * q2) * n, (size_t)n * sizeof(double2),
                              cudaMemcpyDeviceToDevice, ctx->s);
        stored = K / 2;
        every *= 2;
      }
      if (it % every == 0) {
        e = cudaMemcpyAsync(bank + (long long)stored * n, f.x, (size_t)n * sizeof(double2),
                            cudaMemcpyDeviceToDevice, ctx->s);
        ++stored;
      }
      if (e != cudaSuccess) return fg_cuda(ctx, e, "training bank");
    }
    const double rn = norm2(f, r, e);
    if (e != cudaSuccess) return fg_cuda(ctx, e, "training solve");
    if (!std::isfinite(rn)) return TRANSEC_EBREAKDOWN;
    if (rn <= ctx->opts.tol) return TRANSEC_OK;
    if ((e = dots(f, rt, 1, r, h, 0)) != cudaSuccess) return fg_cuda(ctx, e, "training solve");
    if (std::abs(rho) == 0) return TRANSEC_EBREAKDOWN;
    const cplx beta = h[0] / rho;
    rho = h[0];
    k_fg_xpby<<<f.eg, 256, 0, ctx->s>>>(p, r, make_double2(beta.real(), beta.imag()), n);
    k_fg_xpby<<<f.eg, 256, 0, ctx->s>>>(pt, rt, make_double2(beta.real(), beta.imag()), n);
    ctx->launches += 2;
  }
  return TRANSEC_ENOCONV;
}

// one Adam step on the pair (r, e): input (s_r r, V - E, Gamma), target s_e e, both scaled
// to unit RMS
int train_pair(Fg& f, transec_unet* net, double E, const double2* r, const double2* e_vec, float* target,
               float lr, float* loss) {
  transec_ctx* ctx = f.ctx;
  cudaError_t e = cudaSuccess;
  const double rn = norm2(f, r, e);
  if (e != cudaSuccess) return fg_cuda(ctx, e, "training norm");
  const double en = norm2(f, e_vec, e);
  if (e != cudaSuccess) return fg_cuda(ctx, e, "training norm");
  if (!(rn > 0) || !(en > 0) || !std::isfinite(rn) || !std::isfinite(en)) return TRANSEC_EBREAKDOWN;
  const double sq = std::sqrt((double)f.n);
  k_fg_input<<<f.eg, 256, 0, ctx->s>>>(r, sq / rn, ctx->d_v, E, ctx->d_gam, ctx->g.nxy, f.in, f.n);
  k_fg_target<<<f.eg, 256, 0, ctx->s>>>(e_vec, sq / en, target, f.n);
  ctx->launches += 2;
  e = cudaStreamSynchronize(ctx->s);
  if (e != cudaSuccess) return fg_cuda(ctx, e, "training pair");
  const int rc = transec_unet_train_step(net, f.in, target, lr, loss, nullptr, 1);
  if (rc != TRANSEC_OK) return fg_fail(ctx, rc, std::string("network: ") + transec_unet_last_error(net));
  return TRANSEC_OK;
}

}  // namespace

extern "C" int transec_unet_train_operator(transec_ctx* ctx, transec_unet* net, int source, int steps,
                                           double e_lo, double e_hi, float lr, unsigned long long seed,
                                           float* loss_out) {
  if (!ctx) return TRANSEC_EINVAL;
  if (!net) return fg_fail(ctx, TRANSEC_EINVAL, "NULL network");
  if (!ctx->have_v || !ctx->have_abc || !ctx->have_k)
    return fg_fail(ctx, TRANSEC_ESTATE, "potential, absorbing boundary and k-mesh must be set");
  if ((source != 0 && source != 1) || steps < 0 || !std::isfinite(e_lo) || !std::isfinite(e_hi) ||
      e_hi < e_lo || !(lr >= 0))
    return fg_fail(ctx, TRANSEC_EINVAL, "bad training arguments");
  int rc = check_net(ctx, net);
  if (rc) return rc;
  if (steps == 0) return TRANSEC_OK;
  DevScope ds(ctx->device);
  cudaStreamSynchronize(ctx->user);
  Fg f;
  if (fg_setup(f, ctx, 6) != cudaSuccess) return fg_cuda(ctx, f.e, "training set-up");
  const int K = 48;
  DBuf bank;
  if (source == 1) {
    const cudaError_t e = cudaMalloc(&bank.p, (size_t)K * f.n * sizeof(double2));
    if (e != cudaSuccess) return fg_cuda(ctx, e, "training bank");
  }
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> ue(e_lo, e_hi);
  const long long nrhs = (long long)ctx->lplanes.size() * ctx->g.nxy;
  float* target = (float*)(f.V + 6 * f.n);  // [n][2] floats in the last basis vector
  double2* ev = f.Z;                         // the error vector of a pair
  double2* xb = f.Z + f.n;                   // smoothing ping-pong
  int st = 0, failures = 0;
  while (st < steps) {
    const double E = ue(rng);
    const int k = (int)(rng() % (unsigned long long)ctx->nk);
    float loss = 0.f;
    if (source == 0) {
      // random field x, r = A x
      const int passes[6] = {0, 1, 2, 3, 5, 8};
      const int np = passes[rng() % 6];
      double2* xa = ev;
      double2* xo = xb;
      k_fg_noise<<<f.eg, 256, 0, ctx->s>>>(xa, rng(), f.n);
      for (int p = 0; p < np; ++p)
        for (int axis = 0; axis < 3; ++axis) {
          k_fg_smooth<<<f.eg, 256, 0, ctx->s>>>(xa, xo, axis, ctx->g.nx, ctx->g.ny, ctx->g.nz, f.n);
          std::swap(xa, xo);
        }
      ctx->launches += 1 + 3 * np;
      cudaError_t e = apply_A(f, E, k, xa, f.w);
      if (e != cudaSuccess) return fg_cuda(ctx, e, "training apply");
      rc = train_pair(f, net, E, f.w, xa, target, lr, &loss);
      if (rc == TRANSEC_EBREAKDOWN) return fg_fail(ctx, rc, "training: zero pair");
      if (rc) return rc;
      if (loss_out) loss_out[st] = loss;
      ++st;
    } else {
      // Krylov iterates of one column: e_i = x* - x_i, r_i = A e_i
      const long long col = (long long)(rng() % (unsigned long long)nrhs);
      const long long j = (long long)ctx->lplanes[col / ctx->g.nxy] * ctx->g.nxy + col % ctx->g.nxy;
      int stored = 0;
      rc = bicg_bank(f, E, k, j, (double2*)bank.p, K, stored);
      if (rc == TRANSEC_ENOCONV || rc == TRANSEC_EBREAKDOWN) {
        if (++failures > 16) return fg_fail(ctx, rc, "training: the column solves do not converge");
        continue;
      }
      if (rc) return rc;
      std::vector<int> order(stored);
      for (int q = 0; q < stored; ++q) order[q] = q;
      std::shuffle(order.begin(), order.end(), rng);
      for (int q = 0; q < stored && st < steps; ++q) {
        k_fg_sub<<<f.eg, 256, 0, ctx->s>>>(ev, f.x, (double2*)bank.p + (long long)order[q] * f.n, f.n);
        ctx->launches += 1;
        cudaError_t e = apply_A(f, E, k, ev, f.w);
        if (e != cudaSuccess) return fg_cuda(ctx, e, "training apply");
        rc = train_pair(f, net, E, f.w, ev, target, lr, &loss);
        if (rc == TRANSEC_EBREAKDOWN) continue;  // an iterate equal to the solution
        if (rc) return rc;
        if (loss_out) loss_out[st] = loss;
        ++st;
      }
    }
  }
  return TRANSEC_OK;
}
