// Device code shared by the single-layout and the multi-layout symmetric
// repulsion kernels: the work of one tile pair (see repulsion_sym.cu for the
// decomposition and the ring schedule).
//
// Forces leave a unit as fixed-point integers: each FP32 partial (one
// point's sum over the other tile) is scaled by 2^s, rounded to the nearest
// int64 and added with an integer atomic into the point's accumulator
// acc[2 p + {0, 1}].  Integer addition is associative, so the total is the
// same bits whatever order the units finish in, and the accumulators take
// 16 bytes per point instead of one partial per tile.  fix_shift() picks s
// from n so that no sum can overflow (see tsgne_internal.cuh).
//
// Z: each lane's FP32 partial of a point covers one 64-point ring group
// (64 terms w in (0, 1]), is then added into a second FP32 partial over the
// unit's groups (at most 16 for 1,024-point tiles) and leaves the unit in
// FP64.  The worst-case relative rounding of a unit's row sum is then about
// (63 + 15) 2^-24 = 4.6e-6, against 1,023 2^-24 = 6.1e-5 for one FP32 sum over
// the whole tile.
#pragma once

#include "f32x2.cuh"
#include "storage.cuh"
#include "tsgne_internal.cuh"

namespace tsgne {

constexpr int kRI = 16;             // i-points per lane (default shape)
constexpr int kWarpsPerSm = 8;      // resident warps per SM the grid is sized for (16 i-points per lane)
constexpr int kGroup = 64;          // j-points per ring group (32 lanes x 2)

// Resident warps per SM the grid is sized for, by i-points per lane: 16
// i-points need about 200 registers a thread (8 warps), 8 about half.
__host__ __device__ constexpr int warps_per_sm(int RI) { return RI >= 16 ? 8 : 16; }

__device__ __forceinline__ int row_start(int a, int nt) { return a * nt - (a * (a - 1)) / 2; }

// One j-point against the lane's 8 i-points; acc (x, y) is the running sum
// of w^2 (y_i - y_j) over i for this j.
template <int kH>
__device__ __forceinline__ void ring_pair(const float4 q, float& accx, float& accy, const u64 (&X2)[kH],
                                          const u64 (&Y2)[kH], u64 (&FX)[kH], u64 (&FY)[kH], u64 (&Z2)[kH],
                                          const u64 one2) {
  const u64 nx = pk(q.x, q.y);
  const u64 ny = pk(q.z, q.w);
  u64 PX = pk(accx, 0.f), PY = pk(accy, 0.f);
#pragma unroll
  for (int h = 0; h < kH; ++h) {
    const u64 dx = add2(X2[h], nx);
    const u64 dy = add2(Y2[h], ny);
    u64 qq = fma2(dx, dx, one2);
    qq = fma2(dy, dy, qq);
    float q0, q1;
    upk(qq, q0, q1);
    const u64 w = pk(rcp_approx(q0), rcp_approx(q1));
    Z2[h] = add2(Z2[h], w);
    const u64 w2 = mul2(w, w);
    FX[h] = fma2(w2, dx, FX[h]);
    FY[h] = fma2(w2, dy, FY[h]);
    PX = fma2(w2, dx, PX);
    PY = fma2(w2, dy, PY);
  }
  float a0, a1;
  upk(PX, a0, a1);
  accx = a0 + a1;
  upk(PY, a0, a1);
  accy = a0 + a1;
}

// Adds v (one coordinate of a partial force) to a fixed-point accumulator.
__device__ __forceinline__ void red_fix(unsigned long long* p, float v, float scale) {
  const long long q = __float2ll_rn(v * scale);  // v * 2^s is exact: scale is a power of two
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"((unsigned long long)q) : "memory");
}

// One tile pair (a, b), a <= b, of one layout: stages tile b, evaluates the
// pairs and adds tile a's forces and (a < b) tile b's forces into the
// fixed-point accumulators acc[2 p], acc[2 p + 1] of their real points
// (p < n).  Returns this thread's share of the unit's Z (ordered pairs; the
// diagonal unit includes the w_ii = 1 terms of its real points).  Every
// thread of the CTA must call it; it ends with the shared tiles free for reuse
// only after a __syncthreads by the caller.
template <int W, int RI = kRI, class YT = float2>
__device__ __forceinline__ double sym_unit(const YT* __restrict__ Y, int n, unsigned long long* __restrict__ acc,
                                           float fscale, int a, int b, float4* sj, float2* sacc) {
  constexpr int kH = RI / 2;  // FP32x2 pairs of i-points per lane
  constexpr int T = W * 32 * RI;
  constexpr int G = T / kGroup;  // = W RI / 2 groups (a power of two)
  static_assert((G & (G - 1)) == 0, "ring groups are picked modulo G");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u64 one2 = pk(1.f, 1.f);

  // j tile b into shared memory
  for (int k = tid; k < T; k += W * 32) {
    const float2 p = ld_y(Y, (size_t)b * T + k);
    sj[k] = make_float4(-p.x, -p.x, -p.y, -p.y);
    sacc[k] = make_float2(0.f, 0.f);
  }
  // i points of tile a: lane holds i = a*T + warp*32*RI + r*32 + lane, r < RI
  const int ibase = a * T + warp * (32 * RI) + lane;
  u64 X2[kH], Y2[kH], FX[kH], FY[kH], Z2[kH], ZG[kH];
#pragma unroll
  for (int h = 0; h < kH; ++h) {
    const float2 p0 = ld_y(Y, ibase + (2 * h) * 32);
    const float2 p1 = ld_y(Y, ibase + (2 * h + 1) * 32);
    X2[h] = pk(p0.x, p1.x);
    Y2[h] = pk(p0.y, p1.y);
    FX[h] = FY[h] = Z2[h] = ZG[h] = 0ull;
  }
  __syncthreads();

  double zt = 0.0;
  if (a != b) {
    for (int ph = 0; ph < G; ++ph) {
      const int g = (warp + ph) & (G - 1);
      const float4* gj = sj + g * kGroup;
      float2* ga = sacc + g * kGroup;
      float2 c0 = ga[2 * lane], c1 = ga[2 * lane + 1];
      float ax0 = c0.x, ay0 = c0.y, ax1 = c1.x, ay1 = c1.y;
      const int src = (lane + 1) & 31;
#pragma unroll 4
      for (int s = 0; s < 32; ++s) {
        const int jj = (lane + s) & 31;
        const float4 q0 = gj[2 * jj];
        const float4 q1 = gj[2 * jj + 1];
        ring_pair<kH>(q0, ax0, ay0, X2, Y2, FX, FY, Z2, one2);
        ring_pair<kH>(q1, ax1, ay1, X2, Y2, FX, FY, Z2, one2);
        ax0 = __shfl_sync(0xffffffffu, ax0, src);
        ay0 = __shfl_sync(0xffffffffu, ay0, src);
        ax1 = __shfl_sync(0xffffffffu, ax1, src);
        ay1 = __shfl_sync(0xffffffffu, ay1, src);
      }
      ga[2 * lane] = make_float2(ax0, ay0);
      ga[2 * lane + 1] = make_float2(ax1, ay1);
#pragma unroll
      for (int h = 0; h < kH; ++h) {  // the group's 64 terms into the unit's partial
        ZG[h] = add2(ZG[h], Z2[h]);
        Z2[h] = 0ull;
      }
      __syncthreads();
    }
#pragma unroll
    for (int h = 0; h < kH; ++h) {
      float z0, z1;
      upk(ZG[h], z0, z1);
      zt += 2.0 * ((double)z0 + (double)z1);  // tile a holds no padding
    }
    // j side: F_j = -sum_i w^2 (y_i - y_j) for tile b's real points
    const int jb = b * T;
    for (int k = tid; k < T; k += W * 32)
      if (jb + k < n) {
        const float2 v = sacc[k];
        red_fix(acc + 2 * (size_t)(jb + k), -v.x, fscale);
        red_fix(acc + 2 * (size_t)(jb + k) + 1, -v.y, fscale);
      }
  } else {
    // diagonal unit: ordered pairs within the tile, i side only, in groups
    // of 64 j-points for Z
    for (int j0 = 0; j0 < T; j0 += kGroup) {
#pragma unroll 2
      for (int j = j0; j < j0 + kGroup; ++j) {
        const float4 q = sj[j];
        const u64 nx = pk(q.x, q.y);
        const u64 ny = pk(q.z, q.w);
#pragma unroll
        for (int h = 0; h < kH; ++h) {
          const u64 dx = add2(X2[h], nx);
          const u64 dy = add2(Y2[h], ny);
          u64 qq = fma2(dx, dx, one2);
          qq = fma2(dy, dy, qq);
          float q0, q1;
          upk(qq, q0, q1);
          const u64 w = pk(rcp_approx(q0), rcp_approx(q1));
          Z2[h] = add2(Z2[h], w);
          const u64 w2 = mul2(w, w);
          FX[h] = fma2(w2, dx, FX[h]);
          FY[h] = fma2(w2, dy, FY[h]);
        }
      }
#pragma unroll
      for (int h = 0; h < kH; ++h) {
        ZG[h] = add2(ZG[h], Z2[h]);
        Z2[h] = 0ull;
      }
    }
#pragma unroll
    for (int h = 0; h < kH; ++h) {
      float z0, z1;
      upk(ZG[h], z0, z1);
      if (ibase + (2 * h) * 32 < n) zt += (double)z0;
      if (ibase + (2 * h + 1) * 32 < n) zt += (double)z1;
    }
  }
  // i side of tile a's real points
#pragma unroll
  for (int h = 0; h < kH; ++h) {
    float fx0, fx1, fy0, fy1;
    upk(FX[h], fx0, fx1);
    upk(FY[h], fy0, fy1);
    const int p0 = ibase + (2 * h) * 32, p1 = ibase + (2 * h + 1) * 32;
    if (p0 < n) {
      red_fix(acc + 2 * (size_t)p0, fx0, fscale);
      red_fix(acc + 2 * (size_t)p0 + 1, fy0, fscale);
    }
    if (p1 < n) {
      red_fix(acc + 2 * (size_t)p1, fx1, fscale);
      red_fix(acc + 2 * (size_t)p1 + 1, fy1, fscale);
    }
  }
  return zt;
}

// (a, b) of unit u of a layout with nt tiles, numbered diagonal by diagonal:
// diagonal d = b - a holds the nt - d units (0, d), (1, d + 1), ..., so it
// starts at sum_{d' < d} (nt - d') = row_start(d, nt).  Units taken one after
// the other by the persistent grid then touch different tiles: the integer
// atomics of concurrently finishing units go to different points instead of
// all to the shared tile a of one row of the triangle.
__device__ __forceinline__ void unit_tiles(int u, int nt, int* a_out, int* b_out) {
  int lo = 0, hi = nt - 1;  // largest d with row_start(d) <= u
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (row_start(mid, nt) <= u) lo = mid; else hi = mid - 1;
  }
  *a_out = u - row_start(lo, nt);
  *b_out = *a_out + lo;
}

}  // namespace tsgne
