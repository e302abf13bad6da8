// The hot kernels of the multi-shift engine in double-float arithmetic (df64.cuh):
//
//   k_stencil_df   p <- r + beta p, q <- A(E0, +-k) p, sigma += <p~, q> (pairing form)
//   k_update_df    r -= alpha q, rho' = <r~, r>, ||r_h||^2
//   k_ms_shift_df  per-shift p_sigma, x_sigma on the kept planes
//
// The same operator and launch structure as the FP64 kernels of kernels.cuh (paper
// Sec. II.A, Eqs. Bloch and H_k: the order-2R stencil in pair form, Bloch-phased
// lateral wraps, Dirichlet ends in z; half 1 applies A(E, -k) = A(E, k)^T, Sec. II.B),
// with complex vectors stored as float4 double-float values and all arithmetic on the
// FP32 pipes.  The bilinear forms are accumulated in double-float on vectors scaled
// by 2^k (k per run, from the last residual norm) so that small residuals stay well
// inside the float exponent range; the per-block partial sums are returned in FP64.
#pragma once

#include "df64.cuh"
#include "kernels.cuh"

namespace transec {

struct StencilDfArgs {
  const float4* r;        // [slot][half][n]
  const float4* p_in;
  float4* p_out;          // r + beta p_in
  float4* q;              // A p_out
  double* part;           // [slot][nblk][2] partial sums of <p~, A p>
  const Slot* slots;
  const int* escale;      // [slot] k: the pairing dot is taken on 2^k p and 2^k A p
  const float4* phase;    // [nk][2][2][kPhaseN] Bloch phases, complex df64
  const float2* v;        // V per point, df64 (hi, lo)
  const float2* gam;      // Gamma_L + Gamma_R per plane, df64
  float2 kx[kMaxR + 1], ky[kMaxR + 1], kz[kMaxR + 1];  // c_m / (2 h^2), df64
  double diag_c;          // c_0/2 sum_a h_a^-2
  int nx, ny, nz;
  long long nxy, n;
  int H, TX, TY, D, ntx, conj;
  int psym;               // H = 1 and the plane in one tile: <p~, A p> = (P_k p)^T A p
  long long slot_stride;
};

// Up to 896 threads per block (73 registers each): a 20 x 20 plane with both halves
// fits one block, so both lateral halos come from the block's own points.
constexpr int kDfThreads = 896;

// 2^k as a float (|k| <= 126), exact
__device__ inline float pow2f(int k) {
  k = max(-126, min(126, k));
  return __int_as_float((k + 127) << 23);
}

// unnormalised a + b: the TwoSum of the high parts, low parts gathered
__device__ inline df df_pair(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return df{s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}

__device__ inline df acc_df(const dfacc& a) { return df{a.hi, a.lo}; }

// Shared memory of one stencil block: the centre plane of each half with its lateral
// halo, then a ring of the 2R+1 planes around it for every thread's own column (the
// z-neighbours; only the owning thread reads and writes its column, so the ring needs
// no barrier).  Kept out of registers, the ring lets two blocks share an SM.
__host__ __device__ inline size_t stencil_df_smem(int R, int TX, int TY, int H, int threads) {
  return (size_t)H * (TX + 2 * R) * (TY + 2 * R) * sizeof(float4) + (size_t)(2 * R + 1) * threads * sizeof(float4);
}

// ISO: the three axes share the coefficients (hx = hy = hz), so the six neighbours at
// distance m are summed first and multiplied once.
template <int R, bool ISO>
__global__ void __launch_bounds__(kDfThreads, 1) k_stencil_df(const StencilDfArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[2][32];
  float4* sm = reinterpret_cast<float4*>(smem_raw);

  const int slot = blockIdx.z;
  const Slot* stp = a.slots + slot;
  if (stp->status != SLOT_ACTIVE) return;  // uniform over the block
  const dfc beta = dfc{df_split(stp->beta.x), df_split(stp->beta.y)};
  const df ediag = df_split(stp->e + a.diag_c);
  const int ik = stp->ik;
  const int ks = a.escale[slot];
  const float sc = pow2f(ks);

  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const long long nxy = a.nxy;
  const int TX = a.TX, TY = a.TY, D = a.D, ntx = a.ntx;
  const int npt = TX * TY;
  const int t = threadIdx.x;
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
  float4* my = sm + half * SW * SHt;
  float4* ring = sm + a.H * SW * SHt + t;  // this thread's column, stride blockDim.x
  const int rs = blockDim.x;
  const long long base = (long long)slot * a.slot_stride + (long long)half * a.n;
  const float4* __restrict__ r = a.r + base;
  const float4* __restrict__ pin = a.p_in + base;
  float4* __restrict__ pout = a.p_out + base;
  float4* __restrict__ q = a.q + base;
  const float4* ph = a.phase + (size_t)(ik * 2 + (half ^ a.conj)) * 2 * kPhaseN;
  const long long pidx = (long long)gx + (long long)nx * gy;

  auto pnew = [&](long long off) -> dfc { return dfc_fma(beta, dfc_load(pin[off]), dfc_load(r[off])); };
  // p_new at a lateral position of plane zc, wrapped into the cell with its Bloch
  // factor (Eq. Bloch)
  auto wrapped = [&](int xx, int yy, int zc) -> dfc {
    int wx = 0, wy = 0;
    if (xx < 0 || xx >= nx) { wx = floordiv(xx, nx); xx -= wx * nx; }
    if (yy < 0 || yy >= ny) { wy = floordiv(yy, ny); yy -= wy * ny; }
    dfc v = pnew((long long)zc * nxy + xx + (long long)nx * yy);
    if (wx) v = dfc_mul(v, dfc_load(ph[kPhaseW + wx]));
    if (wy) v = dfc_mul(v, dfc_load(ph[kPhaseN + kPhaseW + wy]));
    return v;
  };
  // ring position of plane z (planes z0 - R .. z1 + R - 1 cycle through 2R + 1 slots)
  auto rpos = [&](int z) { return (z - z0 + R) % (2 * R + 1); };

  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int z = z0 - R; z < z0 + R; ++z)
    ring[rpos(z) * rs] = (inside && z >= 0 && z < nz) ? dfc_store(pnew((long long)z * nxy + pidx)) : zero4;
  // the loads of the plane that enters the ring next are issued one plane ahead
  float4 nr = zero4, np = zero4, nv = zero4;
  if (inside && z0 + R < nz) {
    nr = r[(long long)(z0 + R) * nxy + pidx];
    np = pin[(long long)(z0 + R) * nxy + pidx];
  }
  // a tile as wide as the cell (one wrap at most) takes its x-halo from its own
  // points: the cell at x + nx is exp(i k L_a) p(x), the cell at x - nx is exp(-i k L_a) p(x);
  // likewise in y for a tile as high as the cell
  const bool xself = TX == nx && nx >= R;
  const bool yself = TY == ny && ny >= R;

  dfacc sg_re, sg_im;
  // halo cells still computed from global memory: the x-halo rows come first in the
  // enumeration below, then the y-halo columns
  const int nh = yself ? 2 * R * TY : 2 * R * (TX + TY);
  const int h0 = xself ? 2 * R * TY : 0;
  for (int zc = z0; zc < z1; ++zc) {
    {
      const int z = zc + R;
      ring[rpos(z) * rs] = (inside && z < nz) ? dfc_store(dfc_fma(beta, dfc_load(np), dfc_load(nr))) : zero4;
      if (inside && z + 1 < nz) {
        nr = r[(long long)(z + 1) * nxy + pidx];
        np = pin[(long long)(z + 1) * nxy + pidx];
      }
    }
    const dfc c = dfc_load(ring[rpos(zc) * rs]);
    if (inside) {
      const float2 vv = a.v[(long long)zc * nxy + pidx];
      nv = make_float4(vv.x, vv.y, 0.f, 0.f);
    }
    if (worker) my[(ty + R) * SW + tx + R] = dfc_store(inside ? c : wrapped(gx, gy, zc));
    if (xself && inside) {
      if (tx < R) my[(ty + R) * SW + tx + R + nx] = dfc_store(dfc_mul(c, dfc_load(ph[kPhaseW + 1])));
      if (tx >= nx - R) my[(ty + R) * SW + tx + R - nx] = dfc_store(dfc_mul(c, dfc_load(ph[kPhaseW - 1])));
    }
    if (yself && inside) {
      if (ty < R) my[(ty + R + ny) * SW + tx + R] = dfc_store(dfc_mul(c, dfc_load(ph[kPhaseN + kPhaseW + 1])));
      if (ty >= ny - R) my[(ty + R - ny) * SW + tx + R] = dfc_store(dfc_mul(c, dfc_load(ph[kPhaseN + kPhaseW - 1])));
    }
    for (int h = worker ? h0 + lt : nh; h < nh; h += npt) {
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
      my[hy * SW + hx] = dfc_store(wrapped(x0 + hx - R, y0 + hy - R, zc));
    }
    __syncthreads();
    if (inside) {
      const long long off = (long long)zc * nxy + pidx;
      const df dr = df_sub(ediag, df{nv.x, nv.y});
      const float2 gg = a.gam[zc];
      const df di = df{gg.x, gg.y};
      // per-axis accumulators keep independent dependency chains
      dfacc dre, dim_, xre, xim, yre, yim, zre, zim;
      dre.add(df_mul_raw(dr, c.re));
      dre.add(df_neg(df_mul_raw(di, c.im)));
      dim_.add(df_mul_raw(dr, c.im));
      dim_.add(df_mul_raw(di, c.re));
      const float4* ctr = my + (ty + R) * SW + (tx + R);
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        const float4 xa = ctr[m], xb = ctr[-m], ya = ctr[m * SW], yb = ctr[-m * SW];
        const float4 za = ring[rpos(zc + m) * rs], zb = ring[rpos(zc - m + 2 * R + 1) * rs];
        const df ckx = df{a.kx[m].x, a.kx[m].y}, cky = df{a.ky[m].x, a.ky[m].y},
                 ckz = df{a.kz[m].x, a.kz[m].y};
        const df sxr = df_pair(df{xa.x, xa.y}, df{xb.x, xb.y}), sxi = df_pair(df{xa.z, xa.w}, df{xb.z, xb.w});
        const df syr = df_pair(df{ya.x, ya.y}, df{yb.x, yb.y}), syi = df_pair(df{ya.z, ya.w}, df{yb.z, yb.w});
        const df szr = df_pair(df{za.x, za.y}, df{zb.x, zb.y}), szi = df_pair(df{za.z, za.w}, df{zb.z, zb.w});
        if (ISO) {
          xre.add(df_mul_raw(df_pair(df_pair(sxr, syr), szr), ckx));
          xim.add(df_mul_raw(df_pair(df_pair(sxi, syi), szi), ckx));
        } else {
          xre.add(df_mul_raw(sxr, ckx));
          xim.add(df_mul_raw(sxi, ckx));
          yre.add(df_mul_raw(syr, cky));
          yim.add(df_mul_raw(syi, cky));
          zre.add(df_mul_raw(szr, ckz));
          zim.add(df_mul_raw(szi, ckz));
        }
      }
      dre.add(acc_df(xre));
      dre.add(acc_df(yre));
      dre.add(acc_df(zre));
      dim_.add(acc_df(xim));
      dim_.add(acc_df(yim));
      dim_.add(acc_df(zim));
      const dfc acc = dfc{dre.value(), dim_.value()};
      q[off] = dfc_store(acc);
      pout[off] = dfc_store(c);
      // pairing form: half h pairs with half 1-h at the same point (or itself); the
      // P-symmetric form pairs p with P_k p, its in-plane inversion about grid point
      // (0, 0) with the Bloch factor exp(-i k_a L_a) of each axis whose mirror wraps
      dfc o = c;
      if (a.H == 2) {
        o = dfc_load(sm[(1 - half) * SW * SHt + (ty + R) * SW + tx + R]);
      } else if (a.psym) {
        const int mx = gx ? nx - gx : 0, my_ = gy ? ny - gy : 0;
        o = dfc_load(my[(my_ + R) * SW + mx + R]);
        if (gx) o = dfc_mul(o, dfc_load(ph[kPhaseW - 1]));
        if (gy) o = dfc_mul(o, dfc_load(ph[kPhaseN + kPhaseW - 1]));
      }
      dfc_dot_add(sg_re, sg_im, dfc{df_scale(o.re, sc), df_scale(o.im, sc)},
                  dfc{df_scale(acc.re, sc), df_scale(acc.im, sc)});
    }
    __syncthreads();
  }
  const double unscale = ldexp(1.0, -2 * max(-126, min(126, ks)));
  double v2[2] = {df_value(sg_re.value()) * unscale, df_value(sg_im.value()) * unscale};
  block_sum<2>(v2, red);
  if (threadIdx.x == 0) {
    const int nblk = gridDim.x * gridDim.y;
    const int b = blockIdx.x + gridDim.x * blockIdx.y;
    double* o = a.part + ((size_t)slot * nblk + b) * 2;
    o[0] = v2[0];
    o[1] = v2[1];
  }
}

struct UpdateDfArgs {
  float4* r;
  const float4* q;
  const double* sig_part;  // [slot][sig_nblk][2]
  int sig_nblk;
  double* rho_part;        // [slot][gridDim.x][4]: rho re, rho im, |r_0|^2, |r_1|^2
  const Slot* slots;
  const int* escale;
  long long n, slot_stride;
  int H;
};

// r -= alpha q on both halves, partial <r~, r> (pairing form) and ||r_h||^2.
// grid (blocks, slots), 256 threads
__global__ void __launch_bounds__(256) k_update_df(const UpdateDfArgs a) {
  __shared__ double red[4][32];
  __shared__ double2 s_alpha;
  const int slot = blockIdx.y;
  const Slot* stp = a.slots + slot;
  if (stp->status != SLOT_ACTIVE) return;
  if (threadIdx.x < 32) {
    const double2 al = slot_alpha(a.sig_part + (size_t)slot * a.sig_nblk * 2, a.sig_nblk, stp->rho);
    if (threadIdx.x == 0) s_alpha = al;
  }
  __syncthreads();
  const dfc mal = dfc{df_split(-s_alpha.x), df_split(-s_alpha.y)};
  const int ks = a.escale[slot];
  const float sc = pow2f(ks);
  const long long n = a.n;
  const long long base = (long long)slot * a.slot_stride;
  dfacc rr_re, rr_im;
  float n0 = 0.f, n1 = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    dfc rv[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h >= a.H) break;
      const long long off = base + (long long)h * n + i;
      rv[h] = dfc_fma(mal, dfc_load(a.q[off]), dfc_load(a.r[off]));
      a.r[off] = dfc_store(rv[h]);
    }
    const dfc s0 = dfc{df_scale(rv[0].re, sc), df_scale(rv[0].im, sc)};
    n0 = __fmaf_rn(s0.re.hi, s0.re.hi, __fmaf_rn(s0.im.hi, s0.im.hi, n0));
    if (a.H == 2) {
      const dfc s1 = dfc{df_scale(rv[1].re, sc), df_scale(rv[1].im, sc)};
      n1 = __fmaf_rn(s1.re.hi, s1.re.hi, __fmaf_rn(s1.im.hi, s1.im.hi, n1));
      dfc_dot_add(rr_re, rr_im, s0, s1);  // <r, r> = 2 r_+ . r_-
    } else {
      dfc_dot_add(rr_re, rr_im, s0, s0);
    }
  }
  const double unscale = ldexp(1.0, -2 * max(-126, min(126, ks)));
  const double rscale = (a.H == 2 ? 2.0 : 1.0) * unscale;
  double v4[4] = {rscale * df_value(rr_re.value()), rscale * df_value(rr_im.value()), unscale * (double)n0,
                  unscale * (double)n1};
  block_sum<4>(v4, red);
  if (threadIdx.x == 0) {
    double* o = a.rho_part + ((size_t)slot * gridDim.x + blockIdx.x) * 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) o[k] = v4[k];
  }
}

// The P-symmetric form (H = 1): r -= alpha q, rho' = (P_k r)^T r and ||r||^2.  P_k
// pairs a point with its in-plane mirror (same plane), so a thread updates both points
// of a pair (the lower index owns it) and adds 2 phi r_i r_mirror (phi r_i^2 at a point
// that is its own mirror).  grid (blocks, slots), 256 threads
struct UpdateDfPsymArgs {
  float4* r;
  const float4* q;
  const double* sig_part;  // [slot][sig_nblk][2]
  int sig_nblk;
  double* rho_part;        // [slot][gridDim.x][4]: rho re, rho im, |r|^2, |r|^2
  const Slot* slots;
  const int* escale;
  const float4* phase;     // [nk][2][2][kPhaseN] Bloch phases, complex df64
  int nx, ny;
  long long nxy, n, slot_stride;
};

__global__ void __launch_bounds__(256) k_update_df_psym(const UpdateDfPsymArgs a) {
  __shared__ double red[4][32];
  __shared__ double2 s_alpha;
  const int slot = blockIdx.y;
  const Slot* stp = a.slots + slot;
  if (stp->status != SLOT_ACTIVE) return;
  if (threadIdx.x < 32) {
    const double2 al = slot_alpha(a.sig_part + (size_t)slot * a.sig_nblk * 2, a.sig_nblk, stp->rho);
    if (threadIdx.x == 0) s_alpha = al;
  }
  __syncthreads();
  const dfc mal = dfc{df_split(-s_alpha.x), df_split(-s_alpha.y)};
  const int ks = a.escale[slot];
  const float sc = pow2f(ks);
  const float4* ph = a.phase + (size_t)(stp->ik * 2) * 2 * kPhaseN;
  const dfc phx = dfc_load(ph[kPhaseW - 1]), phy = dfc_load(ph[kPhaseN + kPhaseW - 1]);
  const long long base = (long long)slot * a.slot_stride;
  const int nx = a.nx, ny = a.ny;
  dfacc rr_re, rr_im;
  float n0 = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long z = i / a.nxy;
    const int w = (int)(i - z * a.nxy);
    const int y = w / nx, x = w - y * nx;
    const long long im = z * a.nxy + (x ? nx - x : 0) + (long long)nx * (y ? ny - y : 0);
    if (im < i) continue;
    const dfc rv = dfc_fma(mal, dfc_load(a.q[base + i]), dfc_load(a.r[base + i]));
    a.r[base + i] = dfc_store(rv);
    const dfc s0 = dfc{df_scale(rv.re, sc), df_scale(rv.im, sc)};
    n0 = __fmaf_rn(s0.re.hi, s0.re.hi, __fmaf_rn(s0.im.hi, s0.im.hi, n0));
    dfc t = s0;
    if (x) t = dfc_mul(t, phx);
    if (y) t = dfc_mul(t, phy);
    if (im == i) {
      dfc_dot_add(rr_re, rr_im, t, s0);
    } else {
      const dfc rm = dfc_fma(mal, dfc_load(a.q[base + im]), dfc_load(a.r[base + im]));
      a.r[base + im] = dfc_store(rm);
      const dfc s1 = dfc{df_scale(rm.re, sc), df_scale(rm.im, sc)};
      n0 = __fmaf_rn(s1.re.hi, s1.re.hi, __fmaf_rn(s1.im.hi, s1.im.hi, n0));
      // phi r_i r_m + phi r_m r_i (the phase of a pair is the same from either end)
      dfc_dot_add(rr_re, rr_im, dfc{df_scale(t.re, 2.f), df_scale(t.im, 2.f)}, s1);
    }
  }
  const double unscale = ldexp(1.0, -2 * max(-126, min(126, ks)));
  double v4[4] = {unscale * df_value(rr_re.value()), unscale * df_value(rr_im.value()), unscale * (double)n0,
                  unscale * (double)n0};
  block_sum<4>(v4, red);
  if (threadIdx.x == 0) {
    double* o = a.rho_part + ((size_t)slot * gridDim.x + blockIdx.x) * 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) o[k] = v4[k];
  }
}

}  // namespace transec
