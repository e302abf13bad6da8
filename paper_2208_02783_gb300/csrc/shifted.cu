// Multi-shift transpose BiCG: one Krylov run for a left-CAP column at many energies.
//
// A(E, k) = A(E0, k) + (E - E0) 1, so the Krylov spaces of all energies coincide with
// the seed's (E0).  The seed runs the transpose BiCG of the plain engine (A x = e_j with
// the shadow system A^T y = e_j, bilinear forms; A^T = A(E, -k), Sec. II.B).  For a shift
// sigma = E - E0 the residuals stay collinear with the seed's, r_sigma = r / pi_sigma,
// with the scalar pi_sigma following from the seed's alpha, beta by the three-term
// recurrence
//   pi_{n+1} = (1 + alpha_n sigma) pi_n + (alpha_n beta_{n-1} / alpha_{n-1}) (pi_n - pi_{n-1}),
//   alpha_sigma = alpha_n pi_n / pi_{n+1},   beta_sigma = (pi_n / pi_{n+1})^2 beta_n,
// and x_sigma += alpha_sigma p_sigma, p_sigma = r / pi_{n+1} + beta_sigma p_sigma (the same
// for the shadow y_sigma with the seed's shadow residual).  The trace t_j reads x only on
// the Gamma_R planes, so the per-shift x and p are kept on those planes alone.  A shift
// is converged when max(||r||, ||r~||) / |pi_sigma| <= tol; its vectors and pi then stop
// changing.
//
// This is a host-driven single-column form (one seed in flight, host sums of the
// partial dot products each iteration) that states the method on the GPU; it is not
// part of the slot engine.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
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

#define SH_GS(i, n) \
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// partial bilinear (conj = 0) or Hermitian (conj = 1) dots of two vectors; 256 threads
__global__ void __launch_bounds__(256) k_sh_dot(const double2* a, const double2* b, long long n, int conj,
                                                double* part) {
  const double sg = conj ? -1.0 : 1.0;
  double sr = 0.0, si = 0.0;
  SH_GS(i, n) {
    const double2 u = a[i], v = b[i];
    sr += u.x * v.x - sg * u.y * v.y;
    si += u.x * v.y + sg * u.y * v.x;
  }
  __shared__ double red[2][8];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    si += __shfl_down_sync(0xffffffffu, si, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sr;
    red[1][threadIdx.x >> 5] = si;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0, y = 0;
    for (int w = 0; w < 8; ++w) { x += red[0][w]; y += red[1][w]; }
    part[2 * blockIdx.x] = x;
    part[2 * blockIdx.x + 1] = y;
  }
}

__global__ void k_sh_unit(double2* v, long long j, long long n) {
  SH_GS(i, n) v[i] = make_double2(i == j ? 1.0 : 0.0, 0.0);
}

// v += c w
__global__ void k_sh_axpy(double2* v, const double2* w, double2 c, long long n) {
  SH_GS(i, n) {
    const double2 a = w[i];
    v[i].x += c.x * a.x - c.y * a.y;
    v[i].y += c.x * a.y + c.y * a.x;
  }
}

// p = r + beta p
__global__ void k_sh_xpby(double2* p, const double2* r, double2 beta, long long n) {
  SH_GS(i, n) {
    const double2 a = p[i];
    p[i] = make_double2(r[i].x + beta.x * a.x - beta.y * a.y, r[i].y + beta.x * a.y + beta.y * a.x);
  }
}

// grid index of the u-th point of the Gamma_R planes
__device__ inline long long sh_point(long long u, const int* rplanes, long long nxy) {
  return (long long)rplanes[u / nxy] * nxy + u % nxy;
}

// per-shift x_s += alpha_s p_s (both halves) for active shifts; sx/sp are [2][ns][nr]
__global__ void k_sh_update_x(double2* sx, const double2* sp, const double2* alpha_s, const int* active, int ns,
                              long long nr) {
  const long long total = 2LL * ns * nr;
  SH_GS(u, total) {
    const int s = (int)((u / nr) % ns);
    if (!active[s]) continue;
    const double2 a = alpha_s[s], pv = sp[u];
    sx[u].x += a.x * pv.x - a.y * pv.y;
    sx[u].y += a.x * pv.y + a.y * pv.x;
  }
}

// per-shift p_s = r / pi_s + beta_s p_s on the Gamma_R planes (half 0 from r, half 1
// from the shadow residual rs) for active shifts
__global__ void k_sh_update_p(double2* sp, const double2* r, const double2* rs, const double2* inv_pi,
                              const double2* beta_s, const int* active, int ns, long long nr,
                              const int* rplanes, long long nxy) {
  const long long total = 2LL * ns * nr;
  SH_GS(u, total) {
    const long long w = u % nr;
    const int s = (int)((u / nr) % ns);
    const int h = (int)(u / ((long long)ns * nr));
    if (!active[s]) continue;
    const double2 rv = (h == 0 ? r : rs)[sh_point(w, rplanes, nxy)];
    const double2 ip = inv_pi[s], b = beta_s[s], pv = sp[u];
    sp[u] = make_double2(rv.x * ip.x - rv.y * ip.y + b.x * pv.x - b.y * pv.y,
                         rv.x * ip.y + rv.y * ip.x + b.x * pv.y + b.y * pv.x);
  }
}

// copy the Gamma_R planes of v into every shift's slice of half h: sp[h][s][w] = v[point(w)]
__global__ void k_sh_gather(double2* sp, const double2* v, int h, int ns, long long nr, const int* rplanes,
                            long long nxy) {
  const long long total = (long long)ns * nr;
  SH_GS(u, total) sp[(long long)h * ns * nr + u] = v[sh_point(u % nr, rplanes, nxy)];
}

// t[h][s] = 4 gl * sum_w Gamma_R(point(w)) |sx[h][s][w]|^2; grid (blocks, 2 ns), 256 threads
__global__ void __launch_bounds__(256) k_sh_trace(const double2* sx, long long nr, const int* rplanes,
                                                  long long nxy, const double* gr, double* part) {
  const long long base = (long long)blockIdx.y * nr;
  double acc = 0.0;
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nr; w += (long long)gridDim.x * blockDim.x) {
    const double2 v = sx[base + w];
    acc += gr[rplanes[w / nxy]] * (v.x * v.x + v.y * v.y);
  }
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0;
    for (int w = 0; w < 8; ++w) x += red[w];
    part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = x;
  }
}

struct ShBuf {
  void* p = nullptr;
  ~ShBuf() { if (p) cudaFree(p); }
};

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

// Ranking of per-energy statuses for the call's return value (the same order as the
// other solve entry points: not converged < breakdown < timeout < anything else).
int shifted_severity(int code) {
  switch (code) {
    case TRANSEC_OK: return 0;
    case TRANSEC_ENOCONV: return 1;
    case TRANSEC_EBREAKDOWN: return 2;
    case TRANSEC_ETIMEOUT: return 3;
    default: return 4;
  }
}

int sh_fail(transec_ctx* ctx, int code, const std::string& msg) {
  ctx->err = msg;
  return code;
}

}  // namespace

extern "C" int transec_shifted_column(transec_ctx* ctx, int ne, const double* energies, int ik, int64_t col,
                                      double* t_out, double* t_minus_out, int* iters_out, int* status_out) {
  if (!ctx) return TRANSEC_EINVAL;
  if (!ctx->have_v || !ctx->have_abc || !ctx->have_k)
    return sh_fail(ctx, TRANSEC_ESTATE, "potential, absorbing boundary and k-mesh must be set");
  if (ne < 1 || ne > 4096 || !energies || !t_out || ik < 0 || ik >= ctx->nk)
    return sh_fail(ctx, TRANSEC_EINVAL, "bad shifted-column arguments");
  const long long nxy = ctx->g.nxy;
  const long long nrhs = (long long)ctx->lplanes.size() * nxy;
  if (col < 0 || col >= nrhs) return sh_fail(ctx, TRANSEC_EINVAL, "column out of range");
  for (int s = 0; s < ne; ++s)
    if (!std::isfinite(energies[s])) return sh_fail(ctx, TRANSEC_EINVAL, "non-finite energy");
  DevScope ds(ctx->device);
  cudaStreamSynchronize(ctx->user);
  cudaStream_t st = ctx->s;
  const long long n = ctx->g.n;
  const long long nr = (long long)ctx->rplanes.size() * nxy;
  const long long j = (long long)ctx->lplanes[col / nxy] * nxy + col % nxy;
  // seed: the middle energy of the sorted list
  std::vector<double> es(energies, energies + ne);
  std::vector<int> order(ne);
  for (int s = 0; s < ne; ++s) order[s] = s;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return es[a] < es[b]; });
  const double e0 = es[order[ne / 2]];
  std::vector<double> sig(ne);
  for (int s = 0; s < ne; ++s) sig[s] = es[s] - e0;

  const int nb = 152;
  const unsigned eg = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16);
  const TileShape ts = choose_tiles(ctx->g, 1, sizeof(double2), StencilMax<double>::threads, ctx->opts.tile_y,
                                    ctx->opts.slab);
  ShBuf bv, bsx, bsp, bpart, bslot, bspart, bscal, bact, bpscr;
  cudaError_t e = cudaSuccess;
  auto M = [&](ShBuf& b, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(&b.p, bytes);
    return b.p;
  };
  double2* V = (double2*)M(bv, (size_t)6 * n * sizeof(double2));  // r, rs, p, ps, q, qs
  double2* sx = (double2*)M(bsx, (size_t)2 * ne * std::max(1LL, nr) * sizeof(double2));
  double2* sp = (double2*)M(bsp, (size_t)2 * ne * std::max(1LL, nr) * sizeof(double2));
  double* part = (double*)M(bpart, (size_t)std::max(2 * nb, 2 * ne * nb) * sizeof(double));
  Slot* slot = (Slot*)M(bslot, sizeof(Slot));
  double* spart = (double*)M(bspart, (size_t)ts.ntx * ts.nty * ts.nslab * 2 * sizeof(double));
  double2* scal = (double2*)M(bscal, (size_t)3 * ne * sizeof(double2));  // alpha_s, beta_s, 1/pi
  int* act = (int*)M(bact, (size_t)ne * sizeof(int));
  double2* pscr = (double2*)M(bpscr, (size_t)n * sizeof(double2));
  if (e == cudaSuccess) e = prepare_stencil<double>(ctx->g.R, ts.smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return sh_fail(ctx, e == cudaErrorMemoryAllocation ? TRANSEC_ENOMEM : TRANSEC_ECUDA,
                   std::string("shifted set-up: ") + cudaGetErrorString(e));
  }
  double2 *r = V, *rs = V + n, *p = V + 2 * n, *ps = V + 3 * n, *q = V + 4 * n, *qs = V + 5 * n;
  double2* alpha_d = scal;
  double2* beta_d = scal + ne;
  double2* invpi_d = scal + 2 * ne;

  auto apply = [&](const double2* v, double2* out, int transpose) -> cudaError_t {
    Slot hs{};
    hs.status = SLOT_ACTIVE;
    hs.ik = ik;
    hs.e = e0;
    hs.beta = make_double2(0.0, 0.0);
    cudaError_t err = cudaMemcpyAsync(slot, &hs, sizeof(Slot), cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess) return err;
    StencilArgs<double> sa{};
    sa.r = v; sa.p_in = v; sa.p_out = pscr; sa.q = out; sa.part = spart; sa.slots = slot;
    sa.phase = ctx->d_phase; sa.v = ctx->d_v; sa.gam = ctx->d_gam; sa.g = ctx->g; sa.H = 1;
    sa.TX = ts.TX; sa.TY = ts.TY; sa.D = ts.D; sa.ntx = ts.ntx; sa.conj = transpose; sa.slot_stride = n;
    launch_stencil<double>(ctx->g.R, dim3(ts.ntx * ts.nty, ts.nslab, 1), ts.threads, ts.smem, st, sa);
    ctx->launches += 1;
    ctx->point_applies += n;
    return cudaGetLastError();
  };
  std::vector<double> hp(2 * nb);
  auto dot = [&](const double2* a, const double2* b, int conj, cplx& out) -> cudaError_t {
    k_sh_dot<<<nb, 256, 0, st>>>(a, b, n, conj, part);
    ctx->launches += 1;
    cudaError_t err = cudaMemcpyAsync(hp.data(), part, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    out = cplx(0, 0);
    for (int b2 = 0; b2 < nb; ++b2) out += cplx(hp[2 * b2], hp[2 * b2 + 1]);
    return err;
  };

  // start: x = 0, r = rs = p = ps = e_j; per-shift p on the Gamma_R planes = e_j there
  k_sh_unit<<<eg, 256, 0, st>>>(r, j, n);
  k_sh_unit<<<eg, 256, 0, st>>>(rs, j, n);
  k_sh_unit<<<eg, 256, 0, st>>>(p, j, n);
  k_sh_unit<<<eg, 256, 0, st>>>(ps, j, n);
  ctx->launches += 4;
  if (nr > 0) {
    e = cudaMemsetAsync(sx, 0, (size_t)2 * ne * nr * sizeof(double2), st);
    const unsigned sg = (unsigned)std::min<long long>((ne * nr + 255) / 256, 152LL * 16);
    k_sh_gather<<<sg, 256, 0, st>>>(sp, r, 0, ne, nr, ctx->d_rplanes, nxy);
    k_sh_gather<<<sg, 256, 0, st>>>(sp, rs, 1, ne, nr, ctx->d_rplanes, nxy);
    ctx->launches += 2;
  }
  std::vector<cplx> pi(ne, cplx(1, 0)), pi_prev(ne, cplx(1, 0)), pi_next(ne);
  std::vector<int> active(ne, 1), its(ne, 0), status(ne, TRANSEC_ENOCONV);
  std::vector<double2> h_alpha(ne), h_beta(ne), h_invpi(ne);
  cplx rho(1, 0), alpha_prev(1, 0), beta_prev(0, 0);
  const double tol = ctx->opts.tol;
  const unsigned shg = (unsigned)std::min<long long>((2LL * ne * std::max(1LL, nr) + 255) / 256, 152LL * 16);
  int n_it = 0;
  int live = ne;
  for (int it = 1; it <= ctx->opts.maxit && live > 0 && e == cudaSuccess; ++it) {
    n_it = it;
    if ((e = apply(p, q, 0)) != cudaSuccess || (e = apply(ps, qs, 1)) != cudaSuccess) break;
    cplx sq;
    if ((e = dot(ps, q, 0, sq)) != cudaSuccess) break;
    if (std::abs(sq) == 0 || !std::isfinite(std::abs(sq))) {
      for (int s = 0; s < ne; ++s)
        if (active[s]) status[s] = TRANSEC_EBREAKDOWN;
      break;
    }
    const cplx alpha = rho / sq;
    for (int s = 0; s < ne; ++s) {
      if (!active[s]) { h_alpha[s] = make_double2(0, 0); continue; }
      pi_next[s] = (1.0 + alpha * sig[s]) * pi[s] + (alpha * beta_prev / alpha_prev) * (pi[s] - pi_prev[s]);
      const cplx as = alpha * pi[s] / pi_next[s];
      h_alpha[s] = make_double2(as.real(), as.imag());
    }
    e = cudaMemcpyAsync(alpha_d, h_alpha.data(), ne * sizeof(double2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(act, active.data(), ne * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) break;
    if (nr > 0) {
      k_sh_update_x<<<shg, 256, 0, st>>>(sx, sp, alpha_d, act, ne, nr);
      ctx->launches += 1;
    }
    k_sh_axpy<<<eg, 256, 0, st>>>(r, q, make_double2(-alpha.real(), -alpha.imag()), n);
    k_sh_axpy<<<eg, 256, 0, st>>>(rs, qs, make_double2(-alpha.real(), -alpha.imag()), n);
    ctx->launches += 2;
    cplx rr, rrs;
    if ((e = dot(r, r, 1, rr)) != cudaSuccess || (e = dot(rs, rs, 1, rrs)) != cudaSuccess) break;
    const double rn = std::sqrt(std::max(std::max(rr.real(), rrs.real()), 0.0));
    for (int s = 0; s < ne; ++s) {
      if (!active[s]) continue;
      const double res = rn / std::abs(pi_next[s]);
      if (!std::isfinite(res)) {
        active[s] = 0;
        status[s] = TRANSEC_EBREAKDOWN;
        its[s] = it;
        --live;
      } else if (res <= tol) {
        active[s] = 0;
        status[s] = TRANSEC_OK;
        its[s] = it;
        --live;
      }
    }
    if (live == 0) break;
    cplx rho_new;
    if ((e = dot(rs, r, 0, rho_new)) != cudaSuccess) break;
    // BiCG breaks down when the new bilinear form <r~, r> vanishes (or is not finite)
    // while the residuals are not yet small: beta = rho_new / rho would then be zero
    // and every later alpha with it
    if (std::abs(rho_new) == 0 || !std::isfinite(std::abs(rho_new))) {
      for (int s = 0; s < ne; ++s)
        if (active[s]) status[s] = TRANSEC_EBREAKDOWN;
      break;
    }
    const cplx beta = rho_new / rho;
    for (int s = 0; s < ne; ++s) {
      if (!active[s]) continue;
      const cplx ratio = pi[s] / pi_next[s];
      const cplx bs = ratio * ratio * beta;
      const cplx ip = 1.0 / pi_next[s];
      h_beta[s] = make_double2(bs.real(), bs.imag());
      h_invpi[s] = make_double2(ip.real(), ip.imag());
    }
    e = cudaMemcpyAsync(beta_d, h_beta.data(), ne * sizeof(double2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(invpi_d, h_invpi.data(), ne * sizeof(double2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(act, active.data(), ne * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) break;
    if (nr > 0) {
      k_sh_update_p<<<shg, 256, 0, st>>>(sp, r, rs, invpi_d, beta_d, act, ne, nr, ctx->d_rplanes, nxy);
      ctx->launches += 1;
    }
    k_sh_xpby<<<eg, 256, 0, st>>>(p, r, make_double2(beta.real(), beta.imag()), n);
    k_sh_xpby<<<eg, 256, 0, st>>>(ps, rs, make_double2(beta.real(), beta.imag()), n);
    ctx->launches += 2;
    // the host arrays above are read by the copies: finish them before the next update
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
    rho = rho_new;
    alpha_prev = alpha;
    beta_prev = beta;
    for (int s = 0; s < ne; ++s)
      if (active[s]) {
        pi_prev[s] = pi[s];
        pi[s] = pi_next[s];
      }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return sh_fail(ctx, TRANSEC_ECUDA, std::string("shifted iteration: ") + cudaGetErrorString(e));
  }
  // traces of every shift and half on the Gamma_R planes
  std::vector<double> tp((size_t)2 * ne * nb, 0.0);
  if (nr > 0) {
    k_sh_trace<<<dim3(nb, 2 * ne), 256, 0, st>>>(sx, nr, ctx->d_rplanes, nxy, ctx->d_gr, part);
    ctx->launches += 1;
    e = cudaMemcpyAsync(tp.data(), part, tp.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return sh_fail(ctx, TRANSEC_ECUDA, std::string("shifted trace: ") + cudaGetErrorString(e));
  }
  const double glj = ctx->gl[ctx->lplanes[col / nxy]];
  int worst = TRANSEC_OK;
  for (int s = 0; s < ne; ++s) {
    double a = 0, b = 0;
    for (int b2 = 0; b2 < nb; ++b2) {
      a += tp[(size_t)s * nb + b2];
      b += tp[(size_t)(ne + s) * nb + b2];
    }
    const bool ok = status[s] == TRANSEC_OK;
    t_out[s] = ok ? 4.0 * glj * a : std::nan("");
    if (t_minus_out) t_minus_out[s] = ok ? 4.0 * glj * b : std::nan("");
    if (iters_out) iters_out[s] = ok ? its[s] : n_it;
    if (status_out) status_out[s] = status[s];
    if (!ok && shifted_severity(status[s]) > shifted_severity(worst)) worst = status[s];
  }
  if (worst != TRANSEC_OK) ctx->err = "some energies failed (see status_out)";
  return worst;
}
