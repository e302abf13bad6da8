// The learned preconditioner's network on the GPU: parameters, activations, forward,
// backward, Adam, and the C ABI (transec_unet_*).  See unet.cuh for the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/transec.h"
#include "unet.cuh"
#include "unet_tc.cuh"

using namespace transec::unet;

namespace {

struct Layer {
  int cin, cout, cin_p, cout_p, relu;
  long long w_off, b_off;  // offsets in the flat padded parameter buffer
};

// execution order and sizes (the NumPy reference oracle/unet.py uses the same table)
const int kL = 11;
const int kCin[kL] = {4, 16, 16, 32, 32, 64, 96, 32, 48, 16, 16};
const int kCout[kL] = {16, 16, 32, 32, 64, 64, 32, 32, 16, 16, 2};
const int kRelu[kL] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 0};
enum { E1A, E1B, E2A, E2B, E3A, E3B, D2A, D2B, D1A, D1B, OUT };

int pad16(int c) { return (c + 15) / 16 * 16; }

}  // namespace

struct transec_unet {
  int device = 0;
  int nx = 0, ny = 0, nz = 0;
  long long n0 = 0, n1 = 0, n2 = 0;
  Layer L[kL];
  long long np_pad = 0, nw_pad = 0;
  float* p = nullptr;   // FP32 master parameters (padded layout)
  float* g = nullptr;   // gradients
  float* m = nullptr;   // Adam moments
  float* v = nullptr;
  bf16* wbf = nullptr;  // BF16 weights (first nw_pad entries of the padded layout)
  bf16* wt = nullptr;   // transposed, tap-flipped BF16 weights for the data gradient
  long long step = 0;
  // activations and their gradients (BF16, channels last)
  bf16 *x0 = nullptr, *e1a = nullptr, *a1 = nullptr, *p1 = nullptr, *e2a = nullptr, *a2 = nullptr;
  bf16 *p2 = nullptr, *e3a = nullptr, *a3 = nullptr, *u3 = nullptr, *cat2 = nullptr, *d2a = nullptr;
  bf16 *d2 = nullptr, *u2 = nullptr, *cat1 = nullptr, *d1a = nullptr, *d1 = nullptr;
  float* out = nullptr;  // [n0][16]
  bf16 *gA = nullptr, *gB = nullptr, *gC = nullptr, *gSkip1 = nullptr, *gSkip2 = nullptr;
  double* sums = nullptr;
  double* lpart = nullptr;  // per-block loss partial sums [256][2]
  float* wpart = nullptr;   // per-chunk weight-gradient partial sums
  float* bpart = nullptr;   // per-block bias-gradient partial sums
  float* in_buf = nullptr;
  cudaStream_t s = nullptr;
  int sms = 0;            // SMs of the device
  int path = 0;           // 0: tensor-core (tcgen05) convolutions where the plane fits; 1: mma.sync only
  int* d_err = nullptr;   // set by a tcgen05 convolution whose wait timed out
  std::string err;
};

namespace {

int ufail(transec_unet* u, int code, const std::string& msg) {
  if (u) u->err = msg;
  return code;
}

#define UCK(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      cudaGetLastError();                                                                 \
      return ufail(u, e_ == cudaErrorMemoryAllocation ? TRANSEC_ENOMEM : TRANSEC_ECUDA,   \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    }                                                                                     \
  } while (0)

struct Dev {
  int prev = -1;
  explicit Dev(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(d);
  }
  ~Dev() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

unsigned grid_for(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 65535LL * 8); }

void conv(transec_unet* u, int l, const bf16* x, bf16* y, float* yf, long long nvox, int nx, int ny,
          int nz, bool data_grad, bf16* dx) {
  const Layer& L = u->L[l];
  ConvArgs a{};
  if (!data_grad) {
    a.x = x; a.w = u->wbf + L.w_off; a.b = u->p + L.b_off; a.y = y; a.yf = yf;
    a.cin = L.cin_p; a.cout = L.cout_p; a.relu = L.relu;
  } else {  // dx = conv(dy, flipped transposed weights): roles of cin and cout swap
    a.x = x; a.w = u->wt + L.w_off; a.b = nullptr; a.y = dx; a.yf = nullptr;
    a.cin = L.cout_p; a.cout = L.cin_p; a.relu = 0;
  }
  a.nx = nx; a.ny = ny; a.nz = nz; a.nvox = nvox;
  const ConvTcPlan p = u->path == 0 ? conv_tc_plan(nx, ny, nz, a.cin, a.cout, u->sms) : ConvTcPlan{};
  if (p.ok) {
    ConvTcArgs ta{};
    ta.x = a.x; ta.w = a.w; ta.b = a.b; ta.y = a.y; ta.yf = a.yf; ta.err = u->d_err;
    ta.cin = a.cin; ta.cout = a.cout; ta.nx = nx; ta.ny = ny; ta.nz = nz; ta.relu = a.relu;
    ta.bz = p.bz; ta.kc = p.kc; ta.mt = p.mt; ta.tcols = p.tcols; ta.npos = p.npos;
    k_conv_tc<<<(unsigned)((nz + p.bz - 1) / p.bz), 128, p.smem, u->s>>>(ta);
    return;
  }
  const size_t smem = conv_smem_bytes(a.cin);
  const unsigned bricks = (unsigned)(((nx + kBX - 1) / kBX) * ((ny + kBY - 1) / kBY) * ((nz + kBZ - 1) / kBZ));
  k_conv<<<dim3(bricks, (unsigned)(a.cout / 16)), 128, smem, u->s>>>(a);
}

// ETIMEOUT (and the flag cleared) when a tensor-core convolution gave up waiting
int check_tc_error(transec_unet* u) {
  int h = 0;
  UCK(cudaMemcpy(&h, u->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (!h) return TRANSEC_OK;
  UCK(cudaMemset(u->d_err, 0, sizeof(int)));
  return ufail(u, TRANSEC_ETIMEOUT, "a tensor-core convolution timed out waiting for its MMAs");
}

int wgrad_chunk(long long nvox) {
  const long long c = (nvox + 1023) / 1024;
  return (int)std::max<long long>(512, (c + 15) / 16 * 16);
}

const int kBiasBlocks = 120;

void wgrad(transec_unet* u, int l, const bf16* x, const bf16* dy, long long nvox, int nx, int ny, int nz) {
  const Layer& L = u->L[l];
  WgradArgs a{};
  a.x = x; a.dy = dy; a.part = u->wpart; a.cin = L.cin_p; a.cout = L.cout_p;
  a.nx = nx; a.ny = ny; a.nz = nz; a.nvox = nvox; a.chunk = wgrad_chunk(nvox);
  const unsigned nchunks = (unsigned)((nvox + a.chunk - 1) / a.chunk);
  const long long nw = 27LL * L.cout_p * L.cin_p;
  k_wgrad<<<dim3(27, nchunks), 128, 0, u->s>>>(a);
  k_wgrad_reduce<<<grid_for(nw), 256, 0, u->s>>>(u->wpart, u->g + L.w_off, nw, (int)nchunks);
  k_bias_grad<<<kBiasBlocks, 256, 0, u->s>>>(dy, u->bpart, L.cout_p, nvox);
  k_bias_reduce<<<1, 128, 0, u->s>>>(u->bpart, u->g + L.b_off, L.cout_p, kBiasBlocks);
}

__global__ void k_to_bf16(const float* p, bf16* q, long long n) {
  GRID_STRIDE(i, n) q[i] = __float2bfloat16(p[i]);
}

void flip_all(transec_unet* u) {
  for (int l = 0; l < kL; ++l) {
    const Layer& L = u->L[l];
    k_wflip<<<grid_for(27LL * L.cout_p * L.cin_p), 256, 0, u->s>>>(u->wbf + L.w_off, u->wt + L.w_off,
                                                                    L.cout_p, L.cin_p);
  }
}

int forward(transec_unet* u) {
  const int nx = u->nx, ny = u->ny, nz = u->nz;
  const int x1 = nx / 2, y1 = ny / 2, z1 = nz / 2, x2 = nx / 4, y2 = ny / 4, z2 = nz / 4;
  conv(u, E1A, u->x0, u->e1a, nullptr, u->n0, nx, ny, nz, false, nullptr);
  conv(u, E1B, u->e1a, u->a1, nullptr, u->n0, nx, ny, nz, false, nullptr);
  k_pool<<<grid_for(u->n1 * 16), 256, 0, u->s>>>(u->a1, u->p1, 16, nx, ny, nz);
  conv(u, E2A, u->p1, u->e2a, nullptr, u->n1, x1, y1, z1, false, nullptr);
  conv(u, E2B, u->e2a, u->a2, nullptr, u->n1, x1, y1, z1, false, nullptr);
  k_pool<<<grid_for(u->n2 * 32), 256, 0, u->s>>>(u->a2, u->p2, 32, x1, y1, z1);
  conv(u, E3A, u->p2, u->e3a, nullptr, u->n2, x2, y2, z2, false, nullptr);
  conv(u, E3B, u->e3a, u->a3, nullptr, u->n2, x2, y2, z2, false, nullptr);
  k_upsample<<<grid_for(u->n1 * 64), 256, 0, u->s>>>(u->a3, u->u3, 64, x1, y1, u->n1);
  k_concat<<<grid_for(u->n1 * 96), 256, 0, u->s>>>(u->u3, 64, u->a2, 32, u->cat2, u->n1);
  conv(u, D2A, u->cat2, u->d2a, nullptr, u->n1, x1, y1, z1, false, nullptr);
  conv(u, D2B, u->d2a, u->d2, nullptr, u->n1, x1, y1, z1, false, nullptr);
  k_upsample<<<grid_for(u->n0 * 32), 256, 0, u->s>>>(u->d2, u->u2, 32, nx, ny, u->n0);
  k_concat<<<grid_for(u->n0 * 48), 256, 0, u->s>>>(u->u2, 32, u->a1, 16, u->cat1, u->n0);
  conv(u, D1A, u->cat1, u->d1a, nullptr, u->n0, nx, ny, nz, false, nullptr);
  conv(u, D1B, u->d1a, u->d1, nullptr, u->n0, nx, ny, nz, false, nullptr);
  conv(u, OUT, u->d1, nullptr, u->out, u->n0, nx, ny, nz, false, nullptr);
  UCK(cudaGetLastError());
  return TRANSEC_OK;
}

// backward from the BF16 output gradient in gA ([n0][16]); parameter gradients in g
int backward(transec_unet* u) {
  const int nx = u->nx, ny = u->ny, nz = u->nz;
  const int x1 = nx / 2, y1 = ny / 2, z1 = nz / 2, x2 = nx / 4, y2 = ny / 4, z2 = nz / 4;
  UCK(cudaMemsetAsync(u->g, 0, u->np_pad * sizeof(float), u->s));
  auto layer = [&](int l, const bf16* in, const bf16* out, bf16* dy, bf16* dx, long long nv, int ax, int ay,
                   int az) {
    const Layer& L = u->L[l];
    if (L.relu) k_relu_bwd<<<grid_for(nv * L.cout_p), 256, 0, u->s>>>(dy, out, nv * L.cout_p);
    wgrad(u, l, in, dy, nv, ax, ay, az);
    if (dx) conv(u, l, dy, nullptr, nullptr, nv, ax, ay, az, true, dx);
  };
  // gA: d out (n0 x 16) -> gB: d d1 (n0 x 16)
  layer(OUT, u->d1, nullptr, u->gA, u->gB, u->n0, nx, ny, nz);
  layer(D1B, u->d1a, u->d1, u->gB, u->gA, u->n0, nx, ny, nz);            // gA: d d1a
  layer(D1A, u->cat1, u->d1a, u->gA, u->gC, u->n0, nx, ny, nz);          // gC: d cat1 (48)
  k_split<<<grid_for(u->n0 * 48), 256, 0, u->s>>>(u->gC, 32, u->gB, 16, u->gSkip1, u->n0);  // gB: d u2
  k_upsample_bwd<<<grid_for(u->n1 * 32), 256, 0, u->s>>>(u->gB, u->gA, 32, nx, ny, nz);      // gA: d d2
  layer(D2B, u->d2a, u->d2, u->gA, u->gB, u->n1, x1, y1, z1);            // gB: d d2a
  layer(D2A, u->cat2, u->d2a, u->gB, u->gC, u->n1, x1, y1, z1);          // gC: d cat2 (96)
  k_split<<<grid_for(u->n1 * 96), 256, 0, u->s>>>(u->gC, 64, u->gA, 32, u->gSkip2, u->n1);  // gA: d u3
  k_upsample_bwd<<<grid_for(u->n2 * 64), 256, 0, u->s>>>(u->gA, u->gB, 64, x1, y1, z1);      // gB: d a3
  layer(E3B, u->e3a, u->a3, u->gB, u->gA, u->n2, x2, y2, z2);            // gA: d e3a
  layer(E3A, u->p2, u->e3a, u->gA, u->gB, u->n2, x2, y2, z2);            // gB: d p2
  k_pool_bwd<<<grid_for(u->n1 * 32), 256, 0, u->s>>>(u->gB, u->gSkip2, u->gA, 32, x1, y1, u->n1);  // d a2
  layer(E2B, u->e2a, u->a2, u->gA, u->gB, u->n1, x1, y1, z1);            // gB: d e2a
  layer(E2A, u->p1, u->e2a, u->gB, u->gA, u->n1, x1, y1, z1);            // gA: d p1
  k_pool_bwd<<<grid_for(u->n0 * 16), 256, 0, u->s>>>(u->gA, u->gSkip1, u->gB, 16, nx, ny, u->n0);  // d a1
  layer(E1B, u->e1a, u->a1, u->gB, u->gA, u->n0, nx, ny, nz);            // gA: d e1a
  layer(E1A, u->x0, u->e1a, u->gA, nullptr, u->n0, nx, ny, nz);
  UCK(cudaGetLastError());
  return TRANSEC_OK;
}

}  // namespace

extern "C" {

int transec_unet_create(transec_unet** out, int device, int nx, int ny, int nz, unsigned long long seed) {
  if (!out) return TRANSEC_EINVAL;
  *out = nullptr;
  if (nx < 4 || ny < 4 || nz < 4 || nx % 4 || ny % 4 || nz % 4) return TRANSEC_EINVAL;
  transec_unet* u = new transec_unet();
  Dev dg(device);
  u->device = device;
  u->nx = nx; u->ny = ny; u->nz = nz;
  u->n0 = (long long)nx * ny * nz;
  u->n1 = u->n0 / 8;
  u->n2 = u->n1 / 8;
  long long off = 0;
  for (int l = 0; l < kL; ++l) {
    Layer& L = u->L[l];
    L.cin = kCin[l]; L.cout = kCout[l]; L.cin_p = pad16(kCin[l]); L.cout_p = pad16(kCout[l]);
    L.relu = kRelu[l];
    L.w_off = off;
    off += 27LL * L.cin_p * L.cout_p;
  }
  u->nw_pad = off;
  for (int l = 0; l < kL; ++l) {
    u->L[l].b_off = off;
    off += u->L[l].cout_p;
  }
  u->np_pad = off;
  int rc = TRANSEC_OK;
  auto bf = [&](bf16** p, long long n) {
    if (rc == TRANSEC_OK && cudaMalloc(p, n * sizeof(bf16)) != cudaSuccess) rc = TRANSEC_ENOMEM;
  };
  auto fl = [&](float** p, long long n) {
    if (rc == TRANSEC_OK && cudaMalloc(p, n * sizeof(float)) != cudaSuccess) rc = TRANSEC_ENOMEM;
  };
  fl(&u->p, u->np_pad); fl(&u->g, u->np_pad); fl(&u->m, u->np_pad); fl(&u->v, u->np_pad);
  bf(&u->wbf, u->nw_pad); bf(&u->wt, u->nw_pad);
  bf(&u->x0, u->n0 * 16); bf(&u->e1a, u->n0 * 16); bf(&u->a1, u->n0 * 16);
  bf(&u->p1, u->n1 * 16); bf(&u->e2a, u->n1 * 32); bf(&u->a2, u->n1 * 32);
  bf(&u->p2, u->n2 * 32); bf(&u->e3a, u->n2 * 64); bf(&u->a3, u->n2 * 64);
  bf(&u->u3, u->n1 * 64); bf(&u->cat2, u->n1 * 96); bf(&u->d2a, u->n1 * 32); bf(&u->d2, u->n1 * 32);
  bf(&u->u2, u->n0 * 32); bf(&u->cat1, u->n0 * 48); bf(&u->d1a, u->n0 * 16); bf(&u->d1, u->n0 * 16);
  fl(&u->out, u->n0 * 16);
  bf(&u->gA, u->n0 * 48); bf(&u->gB, u->n0 * 48); bf(&u->gC, u->n0 * 48);
  bf(&u->gSkip1, u->n0 * 16); bf(&u->gSkip2, u->n1 * 32);
  fl(&u->in_buf, u->n0 * 4);
  if (rc == TRANSEC_OK && cudaMalloc(&u->sums, 2 * sizeof(double)) != cudaSuccess) rc = TRANSEC_ENOMEM;
  if (rc == TRANSEC_OK && cudaMalloc(&u->lpart, 512 * sizeof(double)) != cudaSuccess) rc = TRANSEC_ENOMEM;
  if (rc == TRANSEC_OK && cudaMalloc(&u->d_err, sizeof(int)) != cudaSuccess) rc = TRANSEC_ENOMEM;
  if (rc == TRANSEC_OK && cudaMemset(u->d_err, 0, sizeof(int)) != cudaSuccess) rc = TRANSEC_ECUDA;
  if (rc == TRANSEC_OK && cudaDeviceGetAttribute(&u->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    rc = TRANSEC_ECUDA;
  if (rc == TRANSEC_OK &&
      cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax) != cudaSuccess)
    rc = TRANSEC_ECUDA;
  {
    // the largest [chunks][27][cout][cin] slice set over the layers (level of each layer
    // from the execution order: e1*, d1*, out at full size; e2*, d2* at 1/8; e3* at 1/64)
    const int level[kL] = {0, 0, 1, 1, 2, 2, 1, 1, 0, 0, 0};
    long long wp = 0;
    for (int l = 0; l < kL; ++l) {
      const long long nv = level[l] == 0 ? u->n0 : level[l] == 1 ? u->n1 : u->n2;
      const long long ch = (nv + wgrad_chunk(nv) - 1) / wgrad_chunk(nv);
      wp = std::max(wp, ch * 27LL * u->L[l].cout_p * u->L[l].cin_p);
    }
    fl(&u->wpart, wp);
    fl(&u->bpart, (long long)kBiasBlocks * 96);
  }
  if (rc == TRANSEC_OK && cudaStreamCreateWithFlags(&u->s, cudaStreamNonBlocking) != cudaSuccess) rc = TRANSEC_ECUDA;
  // the widest convolution input has 96 channels
  if (rc == TRANSEC_OK &&
      cudaFuncSetAttribute(k_conv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem_bytes(96)) !=
          cudaSuccess)
    rc = TRANSEC_ECUDA;
  if (rc != TRANSEC_OK) {
    cudaGetLastError();
    transec_unet_destroy(u);
    return rc;
  }
  // He initialisation (padded entries zero), zero biases and moments
  std::vector<float> hp(u->np_pad, 0.f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < kL; ++l) {
    const Layer& L = u->L[l];
    std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / (27.0 * L.cin)));
    for (int t = 0; t < 27; ++t)
      for (int o = 0; o < L.cout; ++o)
        for (int i = 0; i < L.cin; ++i)
          hp[L.w_off + ((long long)t * L.cout_p + o) * L.cin_p + i] = (float)nd(rng);
  }
  rc = transec_unet_set_params(u, nullptr);
  if (rc == TRANSEC_OK) {
    if (cudaMemcpy(u->p, hp.data(), u->np_pad * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      rc = TRANSEC_ECUDA;
    k_to_bf16<<<grid_for(u->nw_pad), 256, 0, u->s>>>(u->p, u->wbf, u->nw_pad);
    flip_all(u);
    if (cudaStreamSynchronize(u->s) != cudaSuccess) rc = TRANSEC_ECUDA;
  }
  if (rc != TRANSEC_OK) {
    cudaGetLastError();
    transec_unet_destroy(u);
    return rc;
  }
  *out = u;
  return TRANSEC_OK;
}

int transec_unet_n_params(const transec_unet* u, long long* n) {
  if (!u || !n) return TRANSEC_EINVAL;
  long long c = 0;
  for (int l = 0; l < kL; ++l) c += 27LL * u->L[l].cin * u->L[l].cout + u->L[l].cout;
  *n = c;
  return TRANSEC_OK;
}

// flat host layout: per layer w (27, cout, cin) then b (cout), true sizes.
// NULL resets the optimiser state only.
int transec_unet_set_params(transec_unet* u, const float* params) {
  if (!u) return TRANSEC_EINVAL;
  Dev dg(u->device);
  UCK(cudaMemsetAsync(u->m, 0, u->np_pad * sizeof(float), u->s));
  UCK(cudaMemsetAsync(u->v, 0, u->np_pad * sizeof(float), u->s));
  u->step = 0;
  if (params) {
    std::vector<float> hp(u->np_pad, 0.f);
    long long q = 0;
    for (int l = 0; l < kL; ++l) {
      const Layer& L = u->L[l];
      for (int t = 0; t < 27; ++t)
        for (int o = 0; o < L.cout; ++o)
          for (int i = 0; i < L.cin; ++i) hp[L.w_off + ((long long)t * L.cout_p + o) * L.cin_p + i] = params[q++];
      for (int o = 0; o < L.cout; ++o) hp[L.b_off + o] = params[q++];
    }
    UCK(cudaMemcpyAsync(u->p, hp.data(), u->np_pad * sizeof(float), cudaMemcpyHostToDevice, u->s));
    k_to_bf16<<<grid_for(u->nw_pad), 256, 0, u->s>>>(u->p, u->wbf, u->nw_pad);
    flip_all(u);
  }
  UCK(cudaStreamSynchronize(u->s));
  return TRANSEC_OK;
}

int transec_unet_zero_output(transec_unet* u) {
  if (!u) return TRANSEC_EINVAL;
  Dev dg(u->device);
  const Layer& L = u->L[OUT];
  UCK(cudaMemsetAsync(u->p + L.w_off, 0, 27LL * L.cout_p * L.cin_p * sizeof(float), u->s));
  UCK(cudaMemsetAsync(u->m, 0, u->np_pad * sizeof(float), u->s));
  UCK(cudaMemsetAsync(u->v, 0, u->np_pad * sizeof(float), u->s));
  u->step = 0;
  k_to_bf16<<<grid_for(u->nw_pad), 256, 0, u->s>>>(u->p, u->wbf, u->nw_pad);
  flip_all(u);
  UCK(cudaGetLastError());
  UCK(cudaStreamSynchronize(u->s));
  return TRANSEC_OK;
}

static int get_flat(transec_unet* u, const float* src, float* params) {
  std::vector<float> hp(u->np_pad);
  UCK(cudaMemcpyAsync(hp.data(), src, u->np_pad * sizeof(float), cudaMemcpyDeviceToHost, u->s));
  UCK(cudaStreamSynchronize(u->s));
  long long q = 0;
  for (int l = 0; l < kL; ++l) {
    const Layer& L = u->L[l];
    for (int t = 0; t < 27; ++t)
      for (int o = 0; o < L.cout; ++o)
        for (int i = 0; i < L.cin; ++i) params[q++] = hp[L.w_off + ((long long)t * L.cout_p + o) * L.cin_p + i];
    for (int o = 0; o < L.cout; ++o) params[q++] = hp[L.b_off + o];
  }
  return TRANSEC_OK;
}

int transec_unet_get_params(transec_unet* u, float* params) {
  if (!u || !params) return TRANSEC_EINVAL;
  Dev dg(u->device);
  return get_flat(u, u->p, params);
}

int transec_unet_forward(transec_unet* u, const float* in, float* out, int on_device) {
  if (!u || !in || !out) return TRANSEC_EINVAL;
  Dev dg(u->device);
  const float* din = in;
  if (!on_device) {
    UCK(cudaMemcpyAsync(u->in_buf, in, u->n0 * 4 * sizeof(float), cudaMemcpyHostToDevice, u->s));
    din = u->in_buf;
  }
  k_input<<<grid_for(u->n0 * 16), 256, 0, u->s>>>(din, u->x0, u->n0);
  int rc = forward(u);
  if (rc) return rc;
  // channels 0, 1 of the padded FP32 output
  UCK(cudaMemcpy2DAsync(out, 2 * sizeof(float), u->out, 16 * sizeof(float), 2 * sizeof(float), u->n0,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, u->s));
  UCK(cudaStreamSynchronize(u->s));
  return check_tc_error(u);
}

// one step: forward on `in`, relative loss against `target` ([n0][2]), backward; with
// lr > 0 an Adam update follows.  grads (may be NULL) receives the parameter
// gradients (host, flat layout); loss (may be NULL) the loss before the update.
int transec_unet_train_step(transec_unet* u, const float* in, const float* target, float lr, float* loss,
                            float* grads, int on_device) {
  if (!u || !in || !target) return TRANSEC_EINVAL;
  Dev dg(u->device);
  const float* din = in;
  const float* dt = target;
  float* tbuf = nullptr;
  if (!on_device) {
    UCK(cudaMemcpyAsync(u->in_buf, in, u->n0 * 4 * sizeof(float), cudaMemcpyHostToDevice, u->s));
    din = u->in_buf;
    UCK(cudaMalloc(&tbuf, u->n0 * 2 * sizeof(float)));
    UCK(cudaMemcpyAsync(tbuf, target, u->n0 * 2 * sizeof(float), cudaMemcpyHostToDevice, u->s));
    dt = tbuf;
  }
  k_input<<<grid_for(u->n0 * 16), 256, 0, u->s>>>(din, u->x0, u->n0);
  int rc = forward(u);
  if (rc == TRANSEC_OK) {
    k_loss_sums<<<256, 256, 0, u->s>>>(u->out, dt, u->n0, u->lpart);
    k_loss_final<<<1, 32, 0, u->s>>>(u->lpart, 256, u->sums);
    k_loss_grad<<<grid_for(u->n0 * 16), 256, 0, u->s>>>(u->out, dt, u->sums, u->gA, u->n0);
    rc = backward(u);
  }
  if (rc == TRANSEC_OK && loss) {
    double hs[2];
    if (cudaMemcpyAsync(hs, u->sums, sizeof(hs), cudaMemcpyDeviceToHost, u->s) != cudaSuccess ||
        cudaStreamSynchronize(u->s) != cudaSuccess)
      rc = TRANSEC_ECUDA;
    else
      *loss = (float)(hs[0] / hs[1]);
  }
  if (rc == TRANSEC_OK && grads) rc = get_flat(u, u->g, grads);
  if (rc == TRANSEC_OK && lr > 0) {
    u->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)u->step), c2 = 1.f - std::pow(b2, (float)u->step);
    k_adam<<<grid_for(u->np_pad), 256, 0, u->s>>>(u->p, u->g, u->m, u->v, nullptr, u->np_pad, lr, b1, b2,
                                                  1e-8f, c1, c2);
    k_to_bf16<<<grid_for(u->nw_pad), 256, 0, u->s>>>(u->p, u->wbf, u->nw_pad);
    flip_all(u);
  }
  if (tbuf) cudaFree(tbuf);
  if (rc == TRANSEC_OK && cudaStreamSynchronize(u->s) != cudaSuccess) rc = TRANSEC_ECUDA;
  if (rc != TRANSEC_OK) cudaGetLastError();
  if (rc == TRANSEC_OK) rc = check_tc_error(u);
  return rc;
}

int transec_unet_conv3d(int device, int nx, int ny, int nz, int cin, int cout, const uint16_t* x,
                        const uint16_t* w, const float* b, float* y, int path) {
  if (nx < 1 || ny < 1 || nz < 1 || cin < 16 || cout < 16 || cin % 16 || cout % 16 || cout > 256 || !x || !w ||
      !y || path < 0 || path > 1)
    return TRANSEC_EINVAL;
  Dev dg(device);
  const long long nv = (long long)nx * ny * nz;
  bf16 *dx = nullptr, *dw = nullptr;
  float *db = nullptr, *dy = nullptr;
  int* de = nullptr;
  int rc = TRANSEC_OK;
  auto ck = [&](cudaError_t e) {
    if (rc == TRANSEC_OK && e != cudaSuccess) rc = e == cudaErrorMemoryAllocation ? TRANSEC_ENOMEM : TRANSEC_ECUDA;
  };
  ck(cudaMalloc(&dx, nv * cin * sizeof(bf16)));
  ck(cudaMalloc(&dw, 27LL * cout * cin * sizeof(bf16)));
  ck(cudaMalloc(&dy, nv * cout * sizeof(float)));
  ck(cudaMalloc(&de, sizeof(int)));
  if (b) ck(cudaMalloc(&db, cout * sizeof(float)));
  ck(cudaMemcpy(dx, x, nv * cin * sizeof(bf16), cudaMemcpyHostToDevice));
  ck(cudaMemcpy(dw, w, 27LL * cout * cin * sizeof(bf16), cudaMemcpyHostToDevice));
  if (b) ck(cudaMemcpy(db, b, cout * sizeof(float), cudaMemcpyHostToDevice));
  ck(cudaMemset(de, 0, sizeof(int)));
  int sms = 0;
  ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  if (rc == TRANSEC_OK) {
    const ConvTcPlan p = path == 0 ? conv_tc_plan(nx, ny, nz, cin, cout, sms) : ConvTcPlan{};
    if (p.ok) {
      ck(cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax));
      ConvTcArgs ta{};
      ta.x = dx; ta.w = dw; ta.b = db; ta.y = nullptr; ta.yf = dy; ta.err = de;
      ta.cin = cin; ta.cout = cout; ta.nx = nx; ta.ny = ny; ta.nz = nz; ta.relu = 0;
      ta.bz = p.bz; ta.kc = p.kc; ta.mt = p.mt; ta.tcols = p.tcols; ta.npos = p.npos;
      if (rc == TRANSEC_OK) k_conv_tc<<<(unsigned)((nz + p.bz - 1) / p.bz), 128, p.smem>>>(ta);
    } else {
      ck(cudaFuncSetAttribute(k_conv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem_bytes(cin)));
      ConvArgs a{};
      a.x = dx; a.w = dw; a.b = db; a.y = nullptr; a.yf = dy;
      a.cin = cin; a.cout = cout; a.nx = nx; a.ny = ny; a.nz = nz; a.relu = 0; a.nvox = nv;
      const unsigned bricks = (unsigned)(((nx + kBX - 1) / kBX) * ((ny + kBY - 1) / kBY) * ((nz + kBZ - 1) / kBZ));
      if (rc == TRANSEC_OK) k_conv<<<dim3(bricks, (unsigned)(cout / 16)), 128, conv_smem_bytes(cin)>>>(a);
    }
    ck(cudaGetLastError());
    ck(cudaDeviceSynchronize());
  }
  int herr = 0;
  ck(cudaMemcpy(y, dy, nv * cout * sizeof(float), cudaMemcpyDeviceToHost));
  ck(cudaMemcpy(&herr, de, sizeof(int), cudaMemcpyDeviceToHost));
  if (rc == TRANSEC_OK && herr) rc = TRANSEC_ETIMEOUT;
  cudaFree(dx); cudaFree(dw); cudaFree(db); cudaFree(dy); cudaFree(de);
  cudaGetLastError();
  return rc;
}

int transec_unet_set_path(transec_unet* u, int path) {
  if (!u || path < 0 || path > 1) return TRANSEC_EINVAL;
  u->path = path;
  return TRANSEC_OK;
}

int transec_unet_dims(const transec_unet* u, int* nx, int* ny, int* nz) {
  if (!u) return TRANSEC_EINVAL;
  if (nx) *nx = u->nx;
  if (ny) *ny = u->ny;
  if (nz) *nz = u->nz;
  return TRANSEC_OK;
}

const char* transec_unet_last_error(const transec_unet* u) { return u ? u->err.c_str() : ""; }

void transec_unet_destroy(transec_unet* u) {
  if (!u) return;
  Dev dg(u->device);
  if (u->s) cudaStreamSynchronize(u->s);
  for (void* q : {(void*)u->p, (void*)u->g, (void*)u->m, (void*)u->v, (void*)u->wbf, (void*)u->wt,
                  (void*)u->x0, (void*)u->e1a, (void*)u->a1, (void*)u->p1, (void*)u->e2a, (void*)u->a2,
                  (void*)u->p2, (void*)u->e3a, (void*)u->a3, (void*)u->u3, (void*)u->cat2, (void*)u->d2a,
                  (void*)u->d2, (void*)u->u2, (void*)u->cat1, (void*)u->d1a, (void*)u->d1, (void*)u->out,
                  (void*)u->gA, (void*)u->gB, (void*)u->gC, (void*)u->gSkip1, (void*)u->gSkip2,
                  (void*)u->sums, (void*)u->lpart, (void*)u->wpart, (void*)u->bpart, (void*)u->in_buf,
                  (void*)u->d_err})
    if (q) cudaFree(q);
  if (u->s) cudaStreamDestroy(u->s);
  cudaGetLastError();
  delete u;
}

}  // extern "C"
