// Kernels of the learned preconditioner: a 3-level 3D U-Net (16/32/64 channels,
// 3x3x3 convolutions, ReLU, 2x2x2 average pooling, nearest 2x upsampling, skip
// concatenation) trained and applied on the GPU.
//
// Activations are channels-last BF16 arrays [voxel][C], voxel = x + nx*(y + ny*z), C a
// multiple of 16.  The convolutions are implicit GEMMs on the BF16 tensor cores
// (mma.sync m16n8k16, FP32 accumulation):
//   forward / data gradient: rows = voxels, columns = output channels, K = 27 taps x
//                            input channels; the data gradient is the same product
//                            with transposed, tap-flipped weights;
//   weight gradient:         rows = output channels, columns = input channels,
//                            K = voxels of a chunk, one tap per block, FP32 atomics.
// Weights are [27][Cout][Cin] (tap t = (dz+1)*9 + (dy+1)*3 + (dx+1)); zero outside the
// volume.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace transec {
namespace unet {

using bf16 = __nv_bfloat16;

__device__ inline uint32_t ld_pair(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ inline uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ inline void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// neighbour voxel of v at tap t, or -1 outside the volume
__device__ inline long long neighbour(long long v, int t, int nx, int ny, int nz) {
  if (v < 0) return -1;
  const int x = (int)(v % nx);
  const long long r = v / nx;
  const int y = (int)(r % ny);
  const int z = (int)(r / ny);
  const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
  const int xx = x + dx, yy = y + dy, zz = z + dz;
  if (xx < 0 || xx >= nx || yy < 0 || yy >= ny || zz < 0 || zz >= nz) return -1;
  return (long long)xx + (long long)nx * (yy + (long long)ny * zz);
}

struct ConvArgs {
  const bf16* x;   // [nvox][cin]
  const bf16* w;   // [27][cout][cin]
  const float* b;  // [cout] or NULL
  bf16* y;         // [nvox][cout] BF16 output (or NULL)
  float* yf;       // [nvox][cout] FP32 output (or NULL)
  int cin, cout, nx, ny, nz, relu;
  long long nvox;
};

// 4 warps x 16 voxels per block; NT = cout / 8 column tiles per warp.
template <int NT>
__global__ void __launch_bounds__(128) k_conv(const ConvArgs a) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const long long v0 = (long long)blockIdx.x * 64 + warp * 16;
  const long long r0 = v0 + g, r1 = v0 + g + 8;
  const long long q0 = r0 < a.nvox ? r0 : -1, q1 = r1 < a.nvox ? r1 : -1;
  float acc[NT][4];
#pragma unroll
  for (int n = 0; n < NT; ++n)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[n][k] = 0.f;
  const int kchunks = a.cin / 16;
  for (int tap = 0; tap < 27; ++tap) {
    const long long n0 = neighbour(q0, tap, a.nx, a.ny, a.nz);
    const long long n1 = neighbour(q1, tap, a.nx, a.ny, a.nz);
    const bf16* x0 = a.x + (n0 >= 0 ? n0 : 0) * a.cin;
    const bf16* x1 = a.x + (n1 >= 0 ? n1 : 0) * a.cin;
    const bf16* wt = a.w + (long long)tap * a.cout * a.cin;
    for (int kc = 0; kc < kchunks; ++kc) {
      const int k0 = kc * 16 + 2 * t;
      const uint32_t a0 = n0 >= 0 ? ld_pair(x0 + k0) : 0u;
      const uint32_t a1 = n1 >= 0 ? ld_pair(x1 + k0) : 0u;
      const uint32_t a2 = n0 >= 0 ? ld_pair(x0 + k0 + 8) : 0u;
      const uint32_t a3 = n1 >= 0 ? ld_pair(x1 + k0 + 8) : 0u;
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        const bf16* wr = wt + (long long)(n * 8 + g) * a.cin + k0;
        mma_bf16(acc[n], a0, a1, a2, a3, ld_pair(wr), ld_pair(wr + 8));
      }
    }
  }
#pragma unroll
  for (int n = 0; n < NT; ++n) {
    const int c = n * 8 + 2 * t;
    const float b0 = a.b ? a.b[c] : 0.f, b1 = a.b ? a.b[c + 1] : 0.f;
    float v[4] = {acc[n][0] + b0, acc[n][1] + b1, acc[n][2] + b0, acc[n][3] + b1};
    if (a.relu)
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = fmaxf(v[k], 0.f);
    if (r0 < a.nvox) {
      if (a.y) *reinterpret_cast<__nv_bfloat162*>(a.y + r0 * a.cout + c) = __floats2bfloat162_rn(v[0], v[1]);
      if (a.yf) { a.yf[r0 * a.cout + c] = v[0]; a.yf[r0 * a.cout + c + 1] = v[1]; }
    }
    if (r1 < a.nvox) {
      if (a.y) *reinterpret_cast<__nv_bfloat162*>(a.y + r1 * a.cout + c) = __floats2bfloat162_rn(v[2], v[3]);
      if (a.yf) { a.yf[r1 * a.cout + c] = v[2]; a.yf[r1 * a.cout + c + 1] = v[3]; }
    }
  }
}

struct WgradArgs {
  const bf16* x;   // [nvox][cin]  layer input
  const bf16* dy;  // [nvox][cout] gradient of the layer output (after the ReLU mask)
  float* dw;       // [27][cout][cin] accumulated with atomics
  int cin, cout, nx, ny, nz, chunk;
  long long nvox;
};

// grid (27 taps, voxel chunks); warp w takes row tile mt = w % MT and every
// (4/MT)-th column tile; MT = cout/16 in {1, 2, 4}, up to 12 column tiles per warp.
__global__ void __launch_bounds__(128) k_wgrad(const WgradArgs a) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int tap = blockIdx.x;
  const int MT = a.cout / 16, NTT = a.cin / 8;
  const int mt = warp % MT, nstride = 4 / MT, nfirst = warp / MT;
  float acc[12][4];
#pragma unroll
  for (int j = 0; j < 12; ++j)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[j][k] = 0.f;
  const long long vb = (long long)blockIdx.y * a.chunk;
  const bf16 zero = __float2bfloat16(0.f);
  for (int ks = 0; ks < a.chunk; ks += 16) {
    long long vk[4], nb[4];
    const int koff[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      vk[u] = vb + ks + koff[u];
      const bool in = vk[u] < a.nvox && vk[u] < vb + a.chunk;
      if (!in) vk[u] = -1;
      nb[u] = neighbour(vk[u], tap, a.nx, a.ny, a.nz);
    }
    const int co0 = mt * 16 + g, co1 = co0 + 8;
    auto dyv = [&](int u, int co) { return vk[u] >= 0 ? a.dy[vk[u] * a.cout + co] : zero; };
    const uint32_t a0 = pack2(dyv(0, co0), dyv(1, co0));
    const uint32_t a1 = pack2(dyv(0, co1), dyv(1, co1));
    const uint32_t a2 = pack2(dyv(2, co0), dyv(3, co0));
    const uint32_t a3 = pack2(dyv(2, co1), dyv(3, co1));
    int j = 0;
    for (int nt = nfirst; nt < NTT; nt += nstride, ++j) {
      const int ci = nt * 8 + g;
      auto xv = [&](int u) { return nb[u] >= 0 ? a.x[nb[u] * a.cin + ci] : zero; };
      const uint32_t b0 = pack2(xv(0), xv(1));
      const uint32_t b1 = pack2(xv(2), xv(3));
#pragma unroll
      for (int jj = 0; jj < 12; ++jj)
        if (jj == j) mma_bf16(acc[jj], a0, a1, a2, a3, b0, b1);
    }
  }
  int j = 0;
  for (int nt = nfirst; nt < NTT; nt += nstride, ++j) {
    const int co0 = mt * 16 + g, ci0 = nt * 8 + 2 * t;
    float* base = a.dw + (long long)tap * a.cout * a.cin;
#pragma unroll
    for (int jj = 0; jj < 12; ++jj) {
      if (jj != j) continue;
      atomicAdd(base + (long long)co0 * a.cin + ci0, acc[jj][0]);
      atomicAdd(base + (long long)co0 * a.cin + ci0 + 1, acc[jj][1]);
      atomicAdd(base + (long long)(co0 + 8) * a.cin + ci0, acc[jj][2]);
      atomicAdd(base + (long long)(co0 + 8) * a.cin + ci0 + 1, acc[jj][3]);
    }
  }
}

// ---------------------------------------------------------------------------------
// element-wise and reshaping kernels (SIMT)
// ---------------------------------------------------------------------------------

#define GRID_STRIDE(i, n) \
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// voxel of the coarse grid that holds fine voxel v (fine dims nx, ny)
__device__ inline long long parent(long long v, int nx, int ny) {
  const int x = (int)(v % nx);
  const long long r = v / nx;
  const int y = (int)(r % ny);
  const int z = (int)(r / ny);
  return (long long)(x / 2) + (long long)(nx / 2) * (y / 2 + (long long)(ny / 2) * (z / 2));
}

// 2x2x2 average pooling: coarse [nvox/8][C] from fine [nvox][C] (fine dims nx, ny, nz)
static __global__ void k_pool(const bf16* src, bf16* y, int C, int nx, int ny, int nz) {
  const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
  const long long n = (long long)cx * cy * cz * C;
  GRID_STRIDE(i, n) {
    const int c = (int)(i % C);
    const long long v = i / C;
    const int x = (int)(v % cx), y0 = (int)((v / cx) % cy), z = (int)(v / ((long long)cx * cy));
    float s = 0.f;
    for (int d = 0; d < 8; ++d) {
      const long long f = (long long)(2 * x + (d & 1)) +
                          (long long)nx * ((2 * y0 + ((d >> 1) & 1)) + (long long)ny * (2 * z + (d >> 2)));
      s += __bfloat162float(src[f * C + c]);
    }
    y[i] = __float2bfloat16(s * 0.125f);
  }
}

// gradient of pooling (+ an optional skip gradient of the fine tensor): fine dx
static __global__ void k_pool_bwd(const bf16* dy, const bf16* add, bf16* dx, int C, int nx, int ny,
                                  long long nvox) {
  GRID_STRIDE(i, nvox * C) {
    const int c = (int)(i % C);
    const long long v = i / C;
    float s = 0.125f * __bfloat162float(dy[parent(v, nx, ny) * C + c]);
    if (add) s += __bfloat162float(add[i]);
    dx[i] = __float2bfloat16(s);
  }
}

// nearest 2x upsampling: fine [nvox][C] from coarse
static __global__ void k_upsample(const bf16* x, bf16* y, int C, int nx, int ny, long long nvox) {
  GRID_STRIDE(i, nvox * C) {
    const int c = (int)(i % C);
    y[i] = x[parent(i / C, nx, ny) * C + c];
  }
}

// gradient of upsampling: coarse dx = sum of its 8 fine children (fine dims nx, ny, nz)
static __global__ void k_upsample_bwd(const bf16* dy, bf16* dx, int C, int nx, int ny, int nz) {
  const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
  const long long n = (long long)cx * cy * cz * C;
  GRID_STRIDE(i, n) {
    const int c = (int)(i % C);
    const long long v = i / C;
    const int x = (int)(v % cx), y0 = (int)((v / cx) % cy), z = (int)(v / ((long long)cx * cy));
    float s = 0.f;
    for (int d = 0; d < 8; ++d) {
      const long long f = (long long)(2 * x + (d & 1)) +
                          (long long)nx * ((2 * y0 + ((d >> 1) & 1)) + (long long)ny * (2 * z + (d >> 2)));
      s += __bfloat162float(dy[f * C + c]);
    }
    dx[i] = __float2bfloat16(s);
  }
}

// channel concatenation y = [a | b] and its split
static __global__ void k_concat(const bf16* a, int ca, const bf16* b, int cb, bf16* y, long long nvox) {
  const int C = ca + cb;
  GRID_STRIDE(i, nvox * C) {
    const int c = (int)(i % C);
    const long long v = i / C;
    y[i] = c < ca ? a[v * ca + c] : b[v * cb + (c - ca)];
  }
}
static __global__ void k_split(const bf16* y, int ca, bf16* a, int cb, bf16* b, long long nvox) {
  const int C = ca + cb;
  GRID_STRIDE(i, nvox * C) {
    const int c = (int)(i % C);
    const long long v = i / C;
    if (c < ca) a[v * ca + c] = y[i];
    else b[v * cb + (c - ca)] = y[i];
  }
}

// ReLU gradient mask, in place: dy = y > 0 ? dy : 0
static __global__ void k_relu_bwd(bf16* dy, const bf16* y, long long n) {
  GRID_STRIDE(i, n) {
    if (!(__bfloat162float(y[i]) > 0.f)) dy[i] = __float2bfloat16(0.f);
  }
}

// bias gradient db[c] += sum_v dy[v][c]
static __global__ void k_bias_grad(const bf16* dy, float* db, int C, long long nvox) {
  __shared__ float s[64];
  for (int c = threadIdx.x; c < C; c += blockDim.x) s[c] = 0.f;
  __syncthreads();
  GRID_STRIDE(i, nvox * C) atomicAdd(&s[i % C], __bfloat162float(dy[i]));
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&db[c], s[c]);
}

// transposed, tap-flipped weights for the data gradient: wt[26-t][i][o] = w[t][o][i]
static __global__ void k_wflip(const bf16* w, bf16* wt, int cout, int cin) {
  GRID_STRIDE(u, 27LL * cout * cin) {
    const int i = (int)(u % cin);
    const int o = (int)((u / cin) % cout);
    const int t = (int)(u / ((long long)cin * cout));
    wt[((long long)(26 - t) * cin + i) * cout + o] = w[u];
  }
}

// FP32 [nvox][4] network input -> BF16 [nvox][16] (channels 4..15 zero)
static __global__ void k_input(const float* in, bf16* x, long long nvox) {
  GRID_STRIDE(i, nvox * 16) {
    const int c = (int)(i % 16);
    x[i] = __float2bfloat16(c < 4 ? in[(i / 16) * 4 + c] : 0.f);
  }
}

// relative loss sums: s[0] += sum |y - t|^2, s[1] += sum |t|^2 (y: [nvox][16] FP32,
// channels 0, 1 used; t: [nvox][2])
static __global__ void k_loss_sums(const float* y, const float* t, long long nvox, double* s) {
  double a = 0.0, b = 0.0;
  GRID_STRIDE(v, nvox) {
    for (int c = 0; c < 2; ++c) {
      const double d = (double)y[v * 16 + c] - t[v * 2 + c];
      a += d * d;
      b += (double)t[v * 2 + c] * t[v * 2 + c];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&s[0], a);
    atomicAdd(&s[1], b);
  }
}

// dL/dy = 2 (y - t) / sum |t|^2 on channels 0, 1 (zero elsewhere), BF16
static __global__ void k_loss_grad(const float* y, const float* t, const double* s, bf16* dy, long long nvox) {
  const float scale = (float)(2.0 / s[1]);
  GRID_STRIDE(i, nvox * 16) {
    const int c = (int)(i % 16);
    const long long v = i / 16;
    dy[i] = __float2bfloat16(c < 2 ? scale * (y[i] - t[v * 2 + c]) : 0.f);
  }
}

// Adam on FP32 master parameters; refreshes the BF16 copy of the weights
static __global__ void k_adam(float* p, const float* g, float* m, float* v, bf16* pbf, long long n,
                              float lr, float b1, float b2, float eps, float c1, float c2) {
  GRID_STRIDE(i, n) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (pbf) pbf[i] = __float2bfloat16(pi);
  }
}

}  // namespace unet
}  // namespace transec
