// The paper's eigen route, its per-energy stage: T(E, k) from a partial eigensolution
// of B(k) = H_k - i Gamma (Sec. II.A, Eqs. transmission-eigenbasis, Gamma-tilde and
// G-diag; the biorthogonal +-k basis of Sec. II.B; truncation to a fraction of the
// eigenpairs, Sec. II.D).
//
// With right eigenvectors V, left eigenvectors W (W^T B = diag(lambda) W^T, W^T V = 1)
// and g_n(E) = 1/(E - lambda_n), G(E) = V diag(g) W^T, and the library's trace
// T = 4 Tr[Gamma_L G^dagger Gamma_R G] becomes
//
//   T(E) = 4 sum_{m,n} conj(g_m) g_n Rt[m, n] Lt[n, m],
//   Rt = V^H Gamma_R V,   Lt = W^T Gamma_L conj(W) = conj(W^H Gamma_L W).
//
// Both transformed CAPs are Gram matrices of the eigenvectors' rows on the CAP
// supports (Gamma is zero elsewhere), and since W^H Gamma_L W is Hermitian,
// Rt[m, n] Lt[n, m] = Gv[m, n] Gw[m, n] with Gv = V^H Gamma_R V, Gw = W^H Gamma_L W.
// So the stage is: two weighted Gram matrices (k_eig_gram, once per k), their
// element-wise product X, and for every energy the quadratic form
// T(E) = 4 Re[g(E)^H X g(E)] (k_eig_sum, X read once per block of energies).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "engine.cuh"

namespace {

__device__ inline double2 zmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ inline double2 zcmul(double2 a, double2 b) {  // conj(a) b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

constexpr int kGT = 16;  // Gram tile

// out[m][n] (= or *=) sum_i w_i conj(A[i][m]) A[i][n], A row-major [rows][p].  The
// matrix is Hermitian: only the tiles on and above the diagonal are computed, and each
// writes its mirror image conj(.) as well.  grid (ceil(p/16), ceil(p/16)), block 16 x 16
__global__ void __launch_bounds__(kGT * kGT) k_eig_gram(const double2* A, const double* wgt, long long rows, int p,
                                                      double2* out, int multiply) {
  __shared__ double2 sa[kGT][kGT + 1], sb[kGT][kGT + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (blockIdx.y > blockIdx.x) return;  // below the diagonal: written by the mirror tile
  const int m0 = blockIdx.y * kGT, n0 = blockIdx.x * kGT;
  double2 acc = make_double2(0.0, 0.0);
  for (long long i0 = 0; i0 < rows; i0 += kGT) {
    const long long i = i0 + ty;
    const bool ri = i < rows;
    const double w = ri ? wgt[i] : 0.0;
    sa[ty][tx] = (ri && m0 + tx < p) ? A[i * p + m0 + tx] : make_double2(0.0, 0.0);
    const double2 bv = (ri && n0 + tx < p) ? A[i * p + n0 + tx] : make_double2(0.0, 0.0);
    sb[ty][tx] = make_double2(w * bv.x, w * bv.y);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kGT; ++k) {  // acc += conj(a) b as four fused multiply-adds
      const double2 a = sa[k][ty], b = sb[k][tx];
      acc.x = fma(a.x, b.x, acc.x);
      acc.x = fma(a.y, b.y, acc.x);
      acc.y = fma(a.x, b.y, acc.y);
      acc.y = fma(-a.y, b.x, acc.y);
    }
    __syncthreads();
  }
  const int m = m0 + ty, n = n0 + tx;
  if (m < p && n < p) {
    out[(long long)m * p + n] = multiply ? zmul(out[(long long)m * p + n], acc) : acc;
    if (blockIdx.y != blockIdx.x) {  // the mirror element of an off-diagonal tile
      const double2 c = make_double2(acc.x, -acc.y);
      out[(long long)n * p + m] = multiply ? zmul(out[(long long)n * p + m], c) : c;
    }
  }
}

constexpr int kEB = 8;  // energies per block at most

// T[e] = 4 Re sum_m conj(g_m) sum_n X[m][n] g_n, g_n = 1/(E_e - lambda_n), for eb
// energies per block; one warp per row m at a time, lanes over n (coalesced), sums in a
// fixed order.  grid ceil(ne/eb), 256 threads, dynamic shared memory eb p 16 bytes
__global__ void __launch_bounds__(256) k_eig_sum(const double2* X, const double2* lam, int p, const double* E,
                                                 int ne, int eb, double* T) {
  extern __shared__ double2 gsh[];  // [eb][p]
  __shared__ double red[8][kEB];
  const int e0 = blockIdx.x * eb;
  const int nb = min(eb, ne - e0);
  for (int idx = threadIdx.x; idx < nb * p; idx += blockDim.x) {
    const int j = idx / p, n = idx - j * p;
    const double2 d = make_double2(E[e0 + j] - lam[n].x, -lam[n].y);
    const double s = 1.0 / (d.x * d.x + d.y * d.y);
    gsh[idx] = make_double2(d.x * s, -d.y * s);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double acc[kEB];
#pragma unroll
  for (int j = 0; j < kEB; ++j) acc[j] = 0.0;
  for (int m = warp; m < p; m += nw) {
    double2 y[kEB];
#pragma unroll
    for (int j = 0; j < kEB; ++j) y[j] = make_double2(0.0, 0.0);
    for (int n = lane; n < p; n += 32) {
      const double2 x = X[(long long)m * p + n];
#pragma unroll
      for (int j = 0; j < kEB; ++j)
        if (j < nb) {  // y += x g as four fused multiply-adds
          const double2 g = gsh[j * p + n];
          y[j].x = fma(x.x, g.x, y[j].x);
          y[j].x = fma(-x.y, g.y, y[j].x);
          y[j].y = fma(x.x, g.y, y[j].y);
          y[j].y = fma(x.y, g.x, y[j].y);
        }
    }
#pragma unroll
    for (int j = 0; j < kEB; ++j) {
      for (int o = 16; o > 0; o >>= 1) {
        y[j].x += __shfl_down_sync(0xffffffffu, y[j].x, o);
        y[j].y += __shfl_down_sync(0xffffffffu, y[j].y, o);
      }
      if (j < nb) acc[j] += zcmul(gsh[j * p + m], y[j]).x;  // lane 0 holds the row sum
    }
  }
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < kEB; ++j) red[warp][j] = acc[j];
  __syncthreads();
  if (threadIdx.x < nb) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w][threadIdx.x];
    T[e0 + threadIdx.x] = 4.0 * s;
  }
}

}  // namespace

extern "C" {

int transec_eigen_transmission(transec_ctx* ctx, int p, const double* lambda, const double* v_right,
                               const double* w_left, int ne, const double* energies, double* T_out) {
  if (!ctx) return TRANSEC_EINVAL;
  if (!ctx->have_abc) {
    ctx->err = "absorbing boundary not set";
    return TRANSEC_ESTATE;
  }
  if (p < 1 || p > 10240 || ne < 0 || !lambda || !v_right || !w_left || (ne > 0 && (!energies || !T_out))) {
    ctx->err = "bad eigen-route arguments (1 <= p <= 10240)";
    return TRANSEC_EINVAL;
  }
  if (ne == 0) return TRANSEC_OK;
  const long long nxy = ctx->g.nxy;
  const long long nr = (long long)ctx->rplanes.size() * nxy, nl = (long long)ctx->lplanes.size() * nxy;
  // per-row CAP weights in support order (planes ascending, xy within a plane)
  std::vector<double> wr(nr), wl(nl);
  for (size_t a = 0; a < ctx->rplanes.size(); ++a)
    for (long long u = 0; u < nxy; ++u) wr[a * nxy + u] = ctx->gr[ctx->rplanes[a]];
  for (size_t a = 0; a < ctx->lplanes.size(); ++a)
    for (long long u = 0; u < nxy; ++u) wl[a * nxy + u] = ctx->gl[ctx->lplanes[a]];
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  cudaSetDevice(ctx->device);
  double2 *dv = nullptr, *dw = nullptr, *dx = nullptr, *dl = nullptr;
  double *dwr = nullptr, *dwl = nullptr, *de = nullptr, *dt = nullptr;
  int rc = TRANSEC_OK;
  auto ck = [&](cudaError_t e) {
    if (rc == TRANSEC_OK && e != cudaSuccess) {
      rc = e == cudaErrorMemoryAllocation ? TRANSEC_ENOMEM : TRANSEC_ECUDA;
      ctx->err = std::string("eigen route: ") + cudaGetErrorString(e);
    }
  };
  const cudaStream_t s = ctx->s;
  ck(cudaMalloc(&dv, (size_t)nr * p * sizeof(double2)));
  ck(cudaMalloc(&dw, (size_t)nl * p * sizeof(double2)));
  ck(cudaMalloc(&dx, (size_t)p * p * sizeof(double2)));
  ck(cudaMalloc(&dl, (size_t)p * sizeof(double2)));
  ck(cudaMalloc(&dwr, (size_t)nr * sizeof(double)));
  ck(cudaMalloc(&dwl, (size_t)nl * sizeof(double)));
  ck(cudaMalloc(&de, (size_t)ne * sizeof(double)));
  ck(cudaMalloc(&dt, (size_t)ne * sizeof(double)));
  if (rc == TRANSEC_OK) {
    ck(cudaStreamSynchronize(ctx->user));
    ck(cudaMemcpyAsync(dv, v_right, (size_t)nr * p * sizeof(double2), cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(dw, w_left, (size_t)nl * p * sizeof(double2), cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(dl, lambda, (size_t)p * sizeof(double2), cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(dwr, wr.data(), (size_t)nr * sizeof(double), cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(dwl, wl.data(), (size_t)nl * sizeof(double), cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(de, energies, (size_t)ne * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  if (rc == TRANSEC_OK) {
    const dim3 gg((unsigned)((p + kGT - 1) / kGT), (unsigned)((p + kGT - 1) / kGT));
    const bool prof = ctx->opts.profile != 0;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    if (prof)
      for (auto& e : ev) ck(cudaEventCreate(&e));
    if (prof && rc == TRANSEC_OK) cudaEventRecord(ev[0], s);
    k_eig_gram<<<gg, dim3(kGT, kGT), 0, s>>>(dv, dwr, nr, p, dx, 0);  // Gv = V^H Gamma_R V
    k_eig_gram<<<gg, dim3(kGT, kGT), 0, s>>>(dw, dwl, nl, p, dx, 1);  // X = Gv o (W^H Gamma_L W)
    if (prof && rc == TRANSEC_OK) cudaEventRecord(ev[1], s);
    // energies per block: as many as 160 KB of shared memory holds for g, up to 8
    const int eb = (int)std::max<long long>(1, std::min<long long>(kEB, (160LL * 1024) / (16LL * p)));
    const size_t smem = (size_t)eb * p * sizeof(double2);
    ck(cudaFuncSetAttribute(k_eig_sum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (rc == TRANSEC_OK) k_eig_sum<<<(unsigned)((ne + eb - 1) / eb), 256, smem, s>>>(dx, dl, p, de, ne, eb, dt);
    if (prof && rc == TRANSEC_OK) cudaEventRecord(ev[2], s);
    ctx->launches += 3;
    ck(cudaGetLastError());
    ck(cudaMemcpyAsync(T_out, dt, (size_t)ne * sizeof(double), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    if (prof && rc == TRANSEC_OK) {
      float a = 0.f, b = 0.f;
      if (cudaEventElapsedTime(&a, ev[0], ev[1]) == cudaSuccess) ctx->eig_gram_ms += a;
      if (cudaEventElapsedTime(&b, ev[1], ev[2]) == cudaSuccess) ctx->eig_sum_ms += b;
    }
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  }
  cudaFree(dv); cudaFree(dw); cudaFree(dx); cudaFree(dl); cudaFree(dwr); cudaFree(dwl); cudaFree(de); cudaFree(dt);
  cudaGetLastError();
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}

int transec_eigen_stats(const transec_ctx* ctx, double* gram_ms, double* sum_ms) {
  if (!ctx) return TRANSEC_EINVAL;
  if (gram_ms) *gram_ms = ctx->eig_gram_ms;
  if (sum_ms) *sum_ms = ctx->eig_sum_ms;
  return TRANSEC_OK;
}

}  // extern "C"
