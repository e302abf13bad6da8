// The U-Net's 3x3x3 convolution (forward and data gradient) on the 5th-generation
// tensor cores: tcgen05.mma with BF16 operands in shared memory and the FP32
// accumulator in tensor memory (TMEM), read back with tcgen05.ld for the epilogue.
//
// Implicit GEMM without an im2col copy.  A block covers the whole lateral plane of the
// volume for bz consecutive z-planes.  Its input, with a one-voxel zero halo on every
// side, is staged once in shared memory as a box of XH x YH x (bz + 2) positions
// (XH = nx + 2, YH = ny + 2) in the K-major "core matrix" layout of the tensor cores:
// for every group of 8 input channels, one 16-byte row per position, positions in
// box order (x fastest).  The block's output positions, taken in the same box order,
// form M-tiles of 128 consecutive positions (16 groups of 8 rows, 128 bytes apart).
// For tap (dx, dy, dz) the A operand of an M-tile is the same 128 rows shifted by the
// box offset dz XH YH + dy XH + dx, so each tap is a shared-memory descriptor with
// another start address: no data movement between taps.  Rows that fall on halo
// positions compute values that the epilogue discards.  B (the tap's weights, N =
// output channels x K = input channels) is staged in the same layout.  One thread
// issues the MMAs (M = 128, N = cout, K = 16 each), tcgen05.commit signals an
// mbarrier, and the four warps read their 32 TMEM lanes each.
//
// Input channels beyond the shared-memory budget are taken in passes of kc channels
// that accumulate into the same TMEM tiles.  Every wait is bounded: on a timeout the
// block sets *err, skips its epilogue and still frees its tensor memory.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace transec {
namespace unet {

struct ConvTcArgs {
  const bf16* x;   // [nvox][cin]
  const bf16* w;   // [27][cout][cin]
  const float* b;  // [cout] or NULL
  bf16* y;         // [nvox][cout] BF16 output (or NULL)
  float* yf;       // [nvox][cout] FP32 output (or NULL)
  int* err;        // set to 1 when a wait for the tensor cores times out
  int cin, cout, nx, ny, nz, relu;
  int bz;          // output z-planes per block
  int kc;          // input channels per pass (multiple of 16)
  int mt;          // M-tiles of 128 positions
  int tcols;       // TMEM columns allocated (power of two, >= 32, >= mt * cout)
  int npos;        // staged positions (box plus the tiles' overhang)
};

struct ConvTcPlan {
  int bz = 0, kc = 0, mt = 0, tcols = 0, npos = 0;
  size_t smem = 0;
  bool ok = false;
};

constexpr size_t kTcSmemMax = 200 * 1024;

__host__ __device__ inline int tc_qfirst(int nx, int ny) { return (nx + 2) * (ny + 2) + (nx + 2) + 1; }

// Blocks, passes and shared memory of the tensor-core convolution for a volume and a
// layer (cin, cout multiples of 16), or ok = false when the plane does not fit.
inline ConvTcPlan conv_tc_plan(int nx, int ny, int nz, int cin, int cout, int sms) {
  ConvTcPlan p;
  if (cin % 16 || cout % 16 || cout > 256) return p;
  const long long XH = nx + 2, P = XH * (ny + 2);
  // the deepest block that still gives every SM a block
  int bz = 1;
  for (int c = 4; c >= 1; --c)
    if ((nz + c - 1) / c >= sms || c == 1) { bz = c; break; }
  for (; bz >= 1; --bz) {
    const long long nlin = (long long)(bz - 1) * P + (long long)(ny - 1) * XH + nx;
    const int mt = (int)((nlin + 127) / 128);
    if ((long long)mt * cout > 512) continue;
    const long long npos = 2 * (P + XH + 1) + (long long)mt * 128;
    for (int kc = cin; kc >= 16; kc -= 16) {
      const size_t smem = (size_t)npos * kc * 2 + (size_t)27 * kc * cout * 2 + 64;
      if (smem > kTcSmemMax) continue;
      p.bz = bz;
      p.kc = kc;
      p.mt = mt;
      p.npos = (int)npos;
      int tc = 32;
      while (tc < mt * cout) tc *= 2;
      p.tcols = tc;
      p.smem = smem;
      p.ok = true;
      return p;
    }
  }
  return p;
}

__device__ inline uint32_t tc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle; lbo = byte distance of the core
// matrices adjacent in K, sbo = of those adjacent in M (or N)
__device__ inline uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the 5th-generation tensor cores
  return d;
}

// 16-byte global-to-shared copy that does not hold a register (many in flight per
// thread); bytes = 0 writes zeros without reading
__device__ inline void tc_copy16(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

__device__ inline void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// bounded wait for the mbarrier phase of the given parity; false on timeout
__device__ inline bool tc_wait(uint32_t mbar, uint32_t parity) {
  for (int it = 0; it < (1 << 24); ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(128) k_conv_tc(const ConvTcArgs a) {
  extern __shared__ __align__(128) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int XH = nx + 2, YH = ny + 2, P = XH * YH;
  const int z0 = blockIdx.x * a.bz;
  const int qf = tc_qfirst(nx, ny);
  const int npos = a.npos, cout = a.cout;
  uint16_t* box = reinterpret_cast<uint16_t*>(tc_smem);                   // [kc/8][npos][8]
  uint16_t* wsm = box + (size_t)npos * a.kc;                                // [27][kc/8][cout][8]
  const uint32_t mb = tc_smem_u32(&mbar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(&tmem_base)),
                 "r"(a.tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  // instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, N = cout, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(cout >> 3) << 17) | (8u << 24);

  const int npass = (a.cin + a.kc - 1) / a.kc;
  bool ok = true;
  for (int pass = 0; pass < npass; ++pass) {
    const int c0 = pass * a.kc;
    const int kcp = min(a.kc, a.cin - c0);
    const int nch = kcp / 8;
    if (pass > 0) {  // the previous pass's MMAs must be done reading the staged tiles
      if (!tc_wait(mb, (uint32_t)((pass - 1) & 1))) ok = false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (!__syncthreads_and(ok)) break;
    // input box, zero outside the volume and past the box; asynchronous 16-byte copies,
    // all of a thread's copies in flight at once.  A thread walks the positions t, t + S,
    // ... (S threads) with its box coordinates advanced incrementally (no division per
    // copy) and copies every channel group of a position.
    const uint32_t box_s = tc_smem_u32(box), w_s = tc_smem_u32(wsm);
    {
      const int S = blockDim.x;
      const int DX = S % XH, DY = (S / XH) % YH, DZ = S / P;
      int zb = t / P, yb = (t - zb * P) / XH, xb = t - zb * P - yb * XH;
      for (int pos = t; pos < npos; pos += S) {
        const int gx = xb - 1, gy = yb - 1, gz = z0 - 1 + zb;
        const bool in = zb < a.bz + 2 && gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz;
        const bf16* src =
            in ? a.x + ((long long)gx + (long long)nx * (gy + (long long)ny * gz)) * a.cin + c0 : a.x;
        const uint32_t dst = box_s + (uint32_t)pos * 16u;
        for (int ch = 0; ch < nch; ++ch)
          tc_copy16(dst + (uint32_t)ch * (uint32_t)npos * 16u, in ? src + ch * 8 : a.x, in ? 16u : 0u);
        xb += DX;
        if (xb >= XH) { xb -= XH; ++yb; }
        yb += DY;
        if (yb >= YH) { yb -= YH; ++zb; }
        zb += DZ;
      }
    }
    // the pass's weights of every tap: one row (tap, output channel) per thread step
    for (int row = t; row < 27 * cout; row += blockDim.x) {
      const int tap = row / cout, o = row - tap * cout;
      const bf16* src = a.w + (long long)row * a.cin + c0;
      const uint32_t dst = w_s + (uint32_t)((tap * nch * cout + o) * 16);
      for (int ch = 0; ch < nch; ++ch) tc_copy16(dst + (uint32_t)(ch * cout * 16), src + ch * 8, 16u);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (t == 0) {
      const uint32_t box_a = tc_smem_u32(box), w_a = tc_smem_u32(wsm);
      for (int tap = 0; tap < 27; ++tap) {
        const int off = (tap / 9 - 1) * P + ((tap / 3) % 3 - 1) * XH + (tap % 3 - 1);
        for (int ks = 0; ks < nch / 2; ++ks) {
          const uint64_t bd = tc_desc(w_a + (uint32_t)(((tap * nch + 2 * ks) * cout) * 16), (uint32_t)(cout * 16), 128u);
          for (int m = 0; m < a.mt; ++m) {
            const int q = qf + m * 128 + off;
            const uint64_t ad = tc_desc(box_a + (uint32_t)(((2 * ks) * npos + q) * 16), (uint32_t)(npos * 16), 128u);
            tc_mma(tmem + (uint32_t)(m * cout), ad, bd, idesc, (pass | tap | ks) != 0);
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
    }
  }
  if (ok && !tc_wait(mb, (uint32_t)((npass - 1) & 1))) ok = false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok) s_fail = 1;
  __syncthreads();
  if (s_fail) {
    if (t == 0) atomicExch(a.err, 1);
  } else {
    // epilogue: warp w reads TMEM lanes 32w..32w+31 (rows of each M-tile)
    for (int m = 0; m < a.mt; ++m) {
      const int q = qf + m * 128 + 32 * warp + lane;
      const int zb = q / P, rem = q - zb * P;
      const int yb = rem / XH, xb = rem - yb * XH;
      const int gz = z0 - 1 + zb;
      const bool out = zb >= 1 && zb <= a.bz && gz < nz && yb >= 1 && yb <= ny && xb >= 1 && xb <= nx;
      const long long vox = (long long)(xb - 1) + (long long)nx * ((yb - 1) + (long long)ny * gz);
      for (int c = 0; c < cout; c += 16) {
        uint32_t r[16];
        const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(m * cout + c);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!out) continue;
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          v[j] = __uint_as_float(r[j]) + (a.b ? a.b[c + j] : 0.f);
          if (a.relu) v[j] = fmaxf(v[j], 0.f);
        }
        if (a.y) {
          uint32_t pk[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
            pk[j] = *reinterpret_cast<const uint32_t*>(&h);
          }
          uint4* dst = reinterpret_cast<uint4*>(a.y + vox * cout + c);
          dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
        if (a.yf) {
          float4* dst = reinterpret_cast<float4*>(a.yf + vox * cout + c);
#pragma unroll
          for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tcols));
}

}  // namespace unet
}  // namespace transec
