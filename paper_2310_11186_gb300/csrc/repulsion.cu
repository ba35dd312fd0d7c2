// Exact all-pairs Student-t repulsion of t-SNE / t-SGNE (Sec. 2.1, Eq. 4):
//   F^r_i = sum_{j != i} w_ij^2 (y_i - y_j),   Z = sum_{k != l} w_kl,
//   w_ij = (1 + ||y_i - y_j||^2)^-1.
// This O(N^2) pass is the hot loop of every iteration.
//
// Work decomposition.  Points are padded to n_pad with sentinel points
// (1e30, 1e30) whose squared distance to any real point overflows to +inf,
// so w = 0 exactly and no mask is needed in the inner loop.  The i-range is
// cut into i-blocks of BLOCK*R points (R per thread, in registers) and the
// j-range into tiles of JT points; the tiles are grouped into `chunks`
// contiguous j-ranges.  A unit of work is (i-block, chunk); units are dealt
// round-robin to a grid that is a multiple of the SM count, with the chunk
// count chosen so the units fill the grid evenly.  Each unit writes its
// partial forces to frep_part[chunk][i]; the update kernel adds the chunks in
// a fixed order, so the forces are bit-reproducible.
//
// Inner loop.  A j-tile is staged in shared memory as {-x, -x, -y, -y} so that
// one broadcast 128-bit load yields both packed operands; the thread's R
// i-points are held as FP32x2 pairs and every step but the reciprocal runs as
// packed fma/add/mul.f32x2 (sm_100+), i.e. per ordered pair:
//   dx, dy (add), q = 1 + dx^2 + dy^2 (2 fma), w = rcp(q) (MUFU),
//   z += w (add), w2 = w*w (mul), fx += w2 dx, fy += w2 dy (2 fma).
// Z: FP32 per thread over one tile (JT terms), flushed to an FP64 register,
// FP64 per-CTA partial, fixed-order FP64 total in the last CTA, which also
// removes the n diagonal terms (w_ii = 1) and sets the iteration schedule.
#include <cstdio>

#include "f32x2.cuh"
#include "reduce.cuh"
#include "tsgne_internal.cuh"

namespace tsgne {

namespace {

constexpr int kBlock = 256;  // threads per CTA
constexpr int kR = 8;        // i-points per thread
constexpr int kJT = 512;     // j-points per shared-memory tile
constexpr int kIB = kBlock * kR;
constexpr int kCtasPerSm = 2;

template <int BLOCK, int R, int JT>
__global__ void __launch_bounds__(BLOCK, kCtasPerSm)
    k_repulsion(const float2* __restrict__ Y, int n, int n_iblk, int n_jtiles, int chunks,
                float2* __restrict__ frep_part, int n_pad, double* __restrict__ zpart, Sched* sched, int advance,
                float ee, int ee_iters, float mom0, float mom1) {
  static_assert(R % 2 == 0, "R must be even (points are processed in f32x2 pairs)");
  constexpr int H = R / 2;
  __shared__ float4 tile[JT];
  const int tid = threadIdx.x;
  const u64 one2 = pk(1.f, 1.f);
  double zacc = 0.0;
  const int units = n_iblk * chunks;
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int ib = u / chunks;
    const int c = u - ib * chunks;
    const int t0 = (int)((int64_t)c * n_jtiles / chunks);
    const int t1 = (int)((int64_t)(c + 1) * n_jtiles / chunks);
    const int ibase = ib * BLOCK * R + tid;
    u64 X2[H], Y2[H], FX[H], FY[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const float2 p0 = Y[ibase + (2 * h) * BLOCK];
      const float2 p1 = Y[ibase + (2 * h + 1) * BLOCK];
      X2[h] = pk(p0.x, p1.x);
      Y2[h] = pk(p0.y, p1.y);
      FX[h] = 0ull;
      FY[h] = 0ull;
    }
    for (int t = t0; t < t1; ++t) {
      __syncthreads();
      for (int k = tid; k < JT; k += BLOCK) {
        const float2 p = Y[t * JT + k];
        tile[k] = make_float4(-p.x, -p.x, -p.y, -p.y);
      }
      __syncthreads();
      u64 Z2[H];
#pragma unroll
      for (int h = 0; h < H; ++h) Z2[h] = 0ull;
#pragma unroll 4
      for (int j = 0; j < JT; ++j) {
        const float4 q = tile[j];
        const u64 nx = pk(q.x, q.y);
        const u64 ny = pk(q.z, q.w);
#pragma unroll
        for (int h = 0; h < H; ++h) {
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
      for (int h = 0; h < H; ++h) {
        float z0, z1;
        upk(Z2[h], z0, z1);
        if (ibase + (2 * h) * BLOCK < n) zacc += (double)z0;
        if (ibase + (2 * h + 1) * BLOCK < n) zacc += (double)z1;
      }
    }
    float2* out = frep_part + (size_t)c * n_pad;
#pragma unroll
    for (int h = 0; h < H; ++h) {
      float fx0, fx1, fy0, fy1;
      upk(FX[h], fx0, fx1);
      upk(FY[h], fy0, fy1);
      out[ibase + (2 * h) * BLOCK] = make_float2(fx0, fy0);
      out[ibase + (2 * h + 1) * BLOCK] = make_float2(fx1, fy1);
    }
  }
  const double zc = block_sum_d(zacc);
  if (tid == 0) zpart[blockIdx.x] = zc;
  if (arrive_last(&sched->rep_done)) {
    const double total = sum_partials(zpart, gridDim.x);
    if (tid == 0) {
      sched->Z = total - (double)n;
      sched->inv_z = (float)(1.0 / sched->Z);
      const int t = sched->t;
      sched->alpha = t < ee_iters ? ee : 1.0f;
      sched->mu = t < ee_iters ? mom0 : mom1;
      if (advance) sched->t = t + 1;
    }
  }
}

}  // namespace

RepShape repulsion_shape(int n, int sm_count) {
  RepShape sh;
  sh.block = kBlock;
  sh.R = kR;
  sh.jtile = kJT;
  sh.n_iblk = (n + kIB - 1) / kIB;
  sh.n_jtiles = (n + kJT - 1) / kJT;
  sh.n_pad = sh.n_iblk * kIB;
  const int slots = sm_count * kCtasPerSm;
  // chunk count: the fewest chunks whose unit count fills the grid slots to
  // >= 97 % (units are dealt round-robin), capped by the number of tiles
  int best_c = 1;
  double best_eff = -1.0;
  const int cmax = sh.n_jtiles < 64 ? sh.n_jtiles : 64;
  for (int c = 1; c <= cmax; ++c) {
    const long units = (long)sh.n_iblk * c;
    const long waves = (units + slots - 1) / slots;
    const double eff = (double)units / (double)(waves * slots);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best_c = c;
    }
    if (eff >= 0.97) break;
  }
  sh.chunks = best_c;
  const long units = (long)sh.n_iblk * sh.chunks;
  sh.grid = (int)(units < slots ? units : slots);
  return sh;
}

size_t repulsion_zpart_count(const RepShape& sh) { return (size_t)(sh.grid > 0 ? sh.grid : 1); }

tsgne_status launch_repulsion(const RepShape& sh, int n, const float2* Y, float2* frep_part, double* zpart,
                              Sched* sched, int advance, float ee, int ee_iters, float mom0, float mom1,
                              cudaStream_t s) {
  k_repulsion<kBlock, kR, kJT><<<sh.grid, sh.block, 0, s>>>(Y, n, sh.n_iblk, sh.n_jtiles, sh.chunks, frep_part,
                                                           sh.n_pad, zpart, sched, advance, ee, ee_iters, mom0,
                                                           mom1);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

}  // namespace tsgne
