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
//                            K = voxels of a chunk, one tap per block; per-chunk
//                            partial sums added in chunk order (deterministic).
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

// Forward / data-gradient convolution over bricks of 4 x 4 x 8 voxels (x fastest).
// Block = 4 warps; blockIdx.x picks the brick, blockIdx.y a group of 16 output
// channels.  The block stages (a) the group's weights for all 27 taps,
// [27][16][cin + 8], and (b) the brick's input with a one-voxel halo, [6*6*10][cin + 8]
// with zeros outside the volume, in shared memory (16-byte row pads).  An m-tile is one
// z-plane of the brick (16 voxels), so for every tap the A fragment of a thread is a
// fixed offset from its row in the staged tile: no index arithmetic or bounds checks
// in the inner loop.  Warp w computes z-planes 2w and 2w + 1 against both 8-channel
// n-tiles (one B fragment feeds two tensor-core products).  Dynamic shared memory:
// conv_smem_bytes(cin).
constexpr int kBX = 4, kBY = 4, kBZ = 8;                   // brick
constexpr int kHX = kBX + 2, kHY = kBY + 2, kHZ = kBZ + 2;  // with halo
constexpr int kHV = kHX * kHY * kHZ;
__host__ __device__ constexpr int conv_ldw(int cin) { return cin + 8; }
__host__ __device__ constexpr size_t conv_smem_bytes(int cin) {
  return ((size_t)27 * 16 + kHV) * conv_ldw(cin) * 2;
}

__global__ void __launch_bounds__(128) k_conv(const ConvArgs a) {
  extern __shared__ __align__(16) unsigned char conv_smem[];
  const int ld = conv_ldw(a.cin);
  bf16* ws = reinterpret_cast<bf16*>(conv_smem);
  bf16* xs = ws + 27 * 16 * ld;
  const int co0 = blockIdx.y * 16;
  const int nbx = (a.nx + kBX - 1) / kBX, nby = (a.ny + kBY - 1) / kBY;
  const int bx = blockIdx.x % nbx, by = (blockIdx.x / nbx) % nby, bz = blockIdx.x / (nbx * nby);
  const int x0 = bx * kBX, y0 = by * kBY, z0 = bz * kBZ;
  const int cpr = a.cin / 8;  // 16-byte chunks per row
  for (int idx = threadIdx.x; idx < 27 * 16 * cpr; idx += blockDim.x) {
    const int row = idx / cpr, ch = idx - row * cpr;
    const int tap = row >> 4, o = row & 15;
    const uint4 v = *reinterpret_cast<const uint4*>(a.w + ((long long)tap * a.cout + co0 + o) * a.cin + ch * 8);
    *reinterpret_cast<uint4*>(ws + row * ld + ch * 8) = v;
  }
  for (int idx = threadIdx.x; idx < kHV * cpr; idx += blockDim.x) {
    const int h = idx / cpr, ch = idx - h * cpr;
    const int gx = x0 - 1 + h % kHX, gy = y0 - 1 + (h / kHX) % kHY, gz = z0 - 1 + h / (kHX * kHY);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz)
      v = *reinterpret_cast<const uint4*>(a.x + ((long long)gx + (long long)a.nx * (gy + (long long)a.ny * gz)) * a.cin +
                                         ch * 8);
    *reinterpret_cast<uint4*>(xs + h * ld + ch * 8) = v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int lx = g & 3, ly = g >> 2;  // rows g and g + 8 of an m-tile: (lx, ly) and (lx, ly + 2)
  int base[2][2];
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int h = 0; h < 2; ++h) base[m][h] = ((2 * warp + m + 1) * kHY + (ly + 2 * h + 1)) * kHX + lx + 1;
  float acc[2][2][4];
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[m][n][k] = 0.f;
  const int kchunks = a.cin / 16;
  for (int tap = 0; tap < 27; ++tap) {
    const int off = (tap / 9 - 1) * kHX * kHY + ((tap / 3) % 3 - 1) * kHX + (tap % 3 - 1);
    const bf16* wt = ws + tap * 16 * ld;
    for (int kc = 0; kc < kchunks; ++kc) {
      const int k0 = kc * 16 + 2 * t;
      uint32_t b[2][2];
#pragma unroll
      for (int n = 0; n < 2; ++n) {
        const bf16* wr = wt + (n * 8 + g) * ld + k0;
        b[n][0] = ld_pair(wr);
        b[n][1] = ld_pair(wr + 8);
      }
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const bf16* p0 = xs + (base[m][0] + off) * ld + k0;
        const bf16* p1 = xs + (base[m][1] + off) * ld + k0;
        const uint32_t a0 = ld_pair(p0), a1 = ld_pair(p1), a2 = ld_pair(p0 + 8), a3 = ld_pair(p1 + 8);
#pragma unroll
        for (int n = 0; n < 2; ++n) mma_bf16(acc[m][n], a0, a1, a2, a3, b[n][0], b[n][1]);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int n = 0; n < 2; ++n) {
      const int c = co0 + n * 8 + 2 * t;
      const float b0 = a.b ? a.b[c] : 0.f, b1 = a.b ? a.b[c + 1] : 0.f;
      float v[4] = {acc[m][n][0] + b0, acc[m][n][1] + b1, acc[m][n][2] + b0, acc[m][n][3] + b1};
      if (a.relu)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = fmaxf(v[k], 0.f);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int xx = x0 + lx, yy = y0 + ly + 2 * h, zz = z0 + 2 * warp + m;
        if (xx >= a.nx || yy >= a.ny || zz >= a.nz) continue;
        const long long r = (long long)xx + (long long)a.nx * (yy + (long long)a.ny * zz);
        if (a.y) *reinterpret_cast<__nv_bfloat162*>(a.y + r * a.cout + c) = __floats2bfloat162_rn(v[2 * h], v[2 * h + 1]);
        if (a.yf) { a.yf[r * a.cout + c] = v[2 * h]; a.yf[r * a.cout + c + 1] = v[2 * h + 1]; }
      }
    }
}

struct WgradArgs {
  const bf16* x;   // [nvox][cin]  layer input
  const bf16* dy;  // [nvox][cout] gradient of the layer output (after the ReLU mask)
  float* part;     // [chunks][27][cout][cin] per-block partial sums
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
  // this block's partial sums go to its own slice; k_wgrad_reduce adds the slices in order
  int j = 0;
  for (int nt = nfirst; nt < NTT; nt += nstride, ++j) {
    const int co0 = mt * 16 + g, ci0 = nt * 8 + 2 * t;
    float* base = a.part + ((long long)blockIdx.y * 27 + tap) * a.cout * a.cin;
#pragma unroll
    for (int jj = 0; jj < 12; ++jj) {
      if (jj != j) continue;
      base[(long long)co0 * a.cin + ci0] = acc[jj][0];
      base[(long long)co0 * a.cin + ci0 + 1] = acc[jj][1];
      base[(long long)(co0 + 8) * a.cin + ci0] = acc[jj][2];
      base[(long long)(co0 + 8) * a.cin + ci0 + 1] = acc[jj][3];
    }
  }
}

// dw[e] = sum over the chunks, in chunk order, of part[chunk][e] (e < 27 cout cin)
static __global__ void k_wgrad_reduce(const float* part, float* dw, long long nw, int nchunks) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nw; e += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < nchunks; ++c) s += part[(long long)c * nw + e];
    dw[e] = s;
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
// per-block partial bias gradients part[block][c] = sum over the block's voxel range of
// dy[v][c]: thread (r, c) with r = tid / C sums voxels r, r + R, ... (R = blockDim / C),
// then the R sums are added in order.  C <= 96, blockDim = 256.
static __global__ void k_bias_grad(const bf16* dy, float* part, int C, long long nvox) {
  __shared__ float s[256];
  const int R = blockDim.x / C;
  const int r = threadIdx.x / C, c = threadIdx.x % C;
  const long long per = (nvox + gridDim.x - 1) / gridDim.x;
  const long long v0 = (long long)blockIdx.x * per, v1 = v0 + per < nvox ? v0 + per : nvox;
  float acc = 0.f;
  if (r < R)
    for (long long v = v0 + r; v < v1; v += R) acc += __bfloat162float(dy[v * C + c]);
  s[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < C) {
    float tot = 0.f;
    for (int q = 0; q < R; ++q) tot += s[q * C + threadIdx.x];
    part[(long long)blockIdx.x * C + threadIdx.x] = tot;
  }
}

// db[c] = sum over blocks, in order, of part[block][c]
static __global__ void k_bias_reduce(const float* part, float* db, int C, int nblk) {
  const int c = threadIdx.x;
  if (c >= C) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += part[(long long)b * C + c];
  db[c] = s;
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
// per-block partial sums part[block] = (sum |y - t|^2, sum |t|^2) over channels 0, 1;
// blockDim = 256
static __global__ void k_loss_sums(const float* y, const float* t, long long nvox, double* part) {
  double a = 0.0, b = 0.0;
  GRID_STRIDE(v, nvox) {
    for (int c = 0; c < 2; ++c) {
      const double d = (double)y[v * 16 + c] - t[v * 2 + c];
      a += d * d;
      b += (double)t[v * 2 + c] * t[v * 2 + c];
    }
  }
  __shared__ double red[2][8];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < 8; ++w) { sa += red[0][w]; sb += red[1][w]; }
    part[2 * blockIdx.x] = sa;
    part[2 * blockIdx.x + 1] = sb;
  }
}

// s = sum over blocks, in order, of the partial sums
static __global__ void k_loss_final(const double* part, int nblk, double* s) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int q = 0; q < nblk; ++q) { a += part[2 * q]; b += part[2 * q + 1]; }
  s[0] = a;
  s[1] = b;
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
