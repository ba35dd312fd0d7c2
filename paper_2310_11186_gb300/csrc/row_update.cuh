// Device code shared by the single-layout and multi-layout update kernels:
// the attraction of one row and the optimiser step of one point.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "storage.cuh"
#include "tsgne_internal.cuh"

namespace tsgne {

// This lane's share of F^a_i = sum_{j in N(i)} p_ij w_ij (y_i - y_j),
// w = (1 + ||y_i - y_j||^2)^-1, over entries rp[i] + lane, + G, ...
// Entries [a, b) of the row; 4 entries per lane are in flight at once (their
// column / P loads, then their gathers), accumulated in entry order, so the
// result is the same as one entry at a time.
// dbg (debug build only): status word for the check 0 <= column < nY.
template <int G, class PT = float, class YT = float2>
__device__ __forceinline__ void attract_entries(int64_t a, int64_t b, const int32_t* __restrict__ col,
                                                const PT* __restrict__ P, const YT* __restrict__ Y,
                                                int64_t i, int lane, float2 yi, float& ax, float& ay,
                                                int64_t nY = 0, uint32_t* dbg = nullptr) {
  constexpr int U = 4;
  for (int64_t e0 = a + lane; e0 < b; e0 += U * G) {
    int32_t j[U];
    float p[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t e = e0 + (int64_t)u * G;
      const bool ok = e < b;
      j[u] = ok ? col[e] : (int32_t)i;
      p[u] = ok ? ld_p(P, e) : 0.f;
      if (dbg && !TS_IN(j[u], 0, nY, dbg)) j[u] = (int32_t)i;
    }
    float2 yj[U];
#pragma unroll
    for (int u = 0; u < U; ++u) yj[u] = ld_y(Y, j[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (e0 + (int64_t)u * G < b) {
        const float dx = yi.x - yj[u].x, dy = yi.y - yj[u].y;
        const float w = 1.0f / fmaf(dy, dy, fmaf(dx, dx, 1.0f));
        const float pw = p[u] * w;
        ax = fmaf(pw, dx, ax);
        ay = fmaf(pw, dy, ay);
      }
    }
  }
}

// attract_entries with the column / P loads of the next batch issued before
// the current batch's gathers are used (software pipelining), for the long
// rows' chunks where a lane runs through many batches.  Same terms in the
// same order: the same result.  Used where registers are not capped (the
// separate hub-row kernel); under the fused kernel's cap it spills and is
// slower.
template <int G, class PT = float, class YT = float2>
__device__ __forceinline__ void attract_entries_pipelined(int64_t a, int64_t b, const int32_t* __restrict__ col,
                                                          const PT* __restrict__ P, const YT* __restrict__ Y,
                                                          int64_t i, int lane, float2 yi, float& ax, float& ay) {
  constexpr int U = 4;
  int64_t e0 = a + lane;
  if (e0 >= b) return;
  int32_t j[U];
  float p[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t e = e0 + (int64_t)u * G;
    j[u] = e < b ? col[e] : (int32_t)i;
    p[u] = e < b ? ld_p(P, e) : 0.f;
  }
  for (;;) {
    float2 yj[U];
#pragma unroll
    for (int u = 0; u < U; ++u) yj[u] = ld_y(Y, j[u]);
    const int64_t e1 = e0 + U * G;
    const bool more = e1 < b;
    int32_t jn[U];
    float pn[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t e = e1 + (int64_t)u * G;
      jn[u] = e < b ? col[e] : (int32_t)i;
      pn[u] = e < b ? ld_p(P, e) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (e0 + (int64_t)u * G < b) {
        const float dx = yi.x - yj[u].x, dy = yi.y - yj[u].y;
        const float w = 1.0f / fmaf(dy, dy, fmaf(dx, dx, 1.0f));
        const float pw = p[u] * w;
        ax = fmaf(pw, dx, ax);
        ay = fmaf(pw, dy, ay);
      }
    }
    if (!more) break;
    e0 = e1;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      j[u] = jn[u];
      p[u] = pn[u];
    }
  }
}

template <int G>
__device__ __forceinline__ void attract_row(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                            const float* __restrict__ P, const float2* __restrict__ Y, int64_t i,
                                            int lane, float2 yi, float& ax, float& ay) {
  attract_entries<G>(rp[i], rp[i + 1], col, P, Y, i, lane, yi, ax, ay);
}

// Sum over the G lanes of a row group (xor butterfly: every lane gets the
// same value, so later decisions are uniform).
template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}

// Optimiser step (the published t-SNE rule; the paper gives none): per
// coordinate gain += 0.2 if g and the previous update have opposite signs,
// else gain *= 0.8, floored at min_gain; upd = mu upd - eta gain g.
// Returns y + upd and updates u, gn in place.
__device__ __forceinline__ float2 optimizer_step(float gx, float gy, float2& u, float2& gn, float mu, float eta,
                                                 float min_gain, float2 yi) {
  const bool incx = (gx > 0.f && u.x < 0.f) || (gx < 0.f && u.x > 0.f);
  const bool incy = (gy > 0.f && u.y < 0.f) || (gy < 0.f && u.y > 0.f);
  gn.x = fmaxf(incx ? gn.x + 0.2f : gn.x * 0.8f, min_gain);
  gn.y = fmaxf(incy ? gn.y + 0.2f : gn.y * 0.8f, min_gain);
  u.x = mu * u.x - eta * gn.x * gx;
  u.y = mu * u.y - eta * gn.y * gy;
  return make_float2(yi.x + u.x, yi.y + u.y);
}

__device__ __forceinline__ uint32_t atom_add_acq_rel_u32(uint32_t* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Gradient of row i from its attraction sum fa, then (EXPORT) the gradient
// export or the optimiser step into the next layout.
template <bool EXPORT>
__device__ __forceinline__ void finish_row(int64_t i, float2 fa, const float2* __restrict__ frep_part, int chunks,
                                           int n_pad, Sched* sched, float alpha_export, float2* __restrict__ g_out,
                                           const float2* __restrict__ Ym, float2* __restrict__ Ynext,
                                           bf162* __restrict__ Ynext16, float2* __restrict__ upd,
                                           float2* __restrict__ gains, float eta, float min_gain) {
  float rx = 0.f, ry = 0.f;
  for (int c = 0; c < chunks; ++c) {
    const float2 f = frep_part[(size_t)c * n_pad + i];
    rx += f.x;
    ry += f.y;
  }
  const float invZ = sched->inv_z;
  const float alpha = EXPORT ? alpha_export : sched->alpha;
  const float gx = 4.0f * (alpha * fa.x - rx * invZ);
  const float gy = 4.0f * (alpha * fa.y - ry * invZ);
  if (EXPORT) {
    g_out[i] = make_float2(gx, gy);
    return;
  }
  const float mu = sched->mu;
  float2 u = upd[i], gn = gains[i];
  const float2 y = optimizer_step(gx, gy, u, gn, mu, eta, min_gain, Ym[i]);
  upd[i] = u;
  gains[i] = gn;
  Ynext[i] = y;
  if (Ynext16) Ynext16[i] = __float22bfloat162_rn(y);
  if (!isfinite(y.x) || !isfinite(y.y)) atomicOr(&sched->flags, kFlagNonfiniteY);
}

}  // namespace tsgne
