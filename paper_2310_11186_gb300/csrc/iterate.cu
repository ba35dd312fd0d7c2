// Per-iteration kernels other than the repulsion.
//
// k_attract (S3, with S5 in update mode): the attraction of a CTA's rows
//   (short rows as G slot partials per row computed by (row, slot) pairs
//   packed over the CTA; long rows in 1024-entry warp chunks), then one
//   thread per row forms the gradient.  It defines the order of every row's
//   sum; the gradient export runs it, and the update pass runs
//   k_attract_plan (attract_plan.cu), which gives the same sums.  Per row:
//     F^a_i = sum_{j in N(i)} p_ij w_ij (y_i - y_j),  w = (1 + ||y_i-y_j||^2)^-1,
//   add the repulsion forces of the row (chunk order), and form the
//   gradient of Eq. 5 with P scaled by alpha (early exaggeration):
//     g_i = 4 (alpha F^a_i - F^r_i / Z).
//   In update mode the row's thread then applies the optimiser (the paper gives none;
//   the published t-SNE rule): per coordinate gain += 0.2 if g and the
//   previous update have opposite signs, else gain *= 0.8, floored at
//   min_gain; upd = mu upd - eta gain g; y_next = y + upd.  Reading Y_cur and
//   writing Y_next (double buffer) keeps every row's neighbours at the old
//   layout.  In export mode it writes g and changes nothing.
// k_fix_forces (end of S4): converts each point's fixed-point repulsion
//   accumulators into F^r (the update then reads one float2 per row) and
//   clears them for the next pass.
// k_kl (S6): sum_e p_e ln(p_e / w_e) and sum_e p_e in FP64 (terms in FP32),
//   fixed-order totals; KL = first + second * ln Z on the host (Eq. 5 with
//   q = w / Z).
#include <cmath>
#include <vector>

#include "reduce.cuh"
#include "row_update.cuh"
#include "storage.cuh"
#include "tsgne_internal.cuh"

namespace tsgne {

namespace {

constexpr int kAttrCta = 256;
constexpr int kAttrPairs = 3;  // (row, slot) pairs a thread has in flight at once
static_assert(kAttrCta <= 256, "rows of a CTA are numbered in one byte");
constexpr int kG = 8;  // lanes per row

// Exclusive scan of v over a CTA of kAttrCta threads into off[0..kAttrCta],
// off[kAttrCta] = total (wsum: kAttrCta / 32 ints of scratch).  Ends with
// a __syncthreads before off is complete for every thread: the caller syncs.
__device__ __forceinline__ void block_excl_scan(int v, int* off, int* wsum) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += u;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  int base = 0;
  for (int k = 0; k < w; ++k) base += wsum[k];
  off[threadIdx.x] = base + x - v;
  if (threadIdx.x == kAttrCta - 1) off[kAttrCta] = base + x;
}

// Three phases per CTA of kAttrCta rows.  A short row's attraction is, by
// definition of the sum order, G slot partials -- slot s accumulates entries
// s, s + G, ... with an fmaf chain (attract_entries with lane = s) -- added
// in the order of the G-lane xor butterfly.  (1) each row counts its slots
// in use (min(degree, G)); (2) one thread per (row, slot) in use, packed
// over the CTA's rows, computes the slot partials into shared memory, so
// short rows leave no lane idle and a thread has its own gathers in flight;
// (3) one thread per row adds its slots in the butterfly's order, reads F^r,
// the optimiser state and Y_i and writes the update (coalesced).  The sums
// are the bits G lanes per row with group_sum<G> produce.
//
// This is the definition of every row's summation order; the gradient
// export runs it (rows above kHeavyDeg entries take their chunk sums from
// k_attract_heavy), and the update pass (k_attract_plan, attract_plan.cu)
// reproduces the same sums bit for bit on a schedule fixed with P.
template <int G, bool EXPORT, class PT, class YT>
__global__ void __launch_bounds__(kAttrCta, 6)
    k_attract(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const PT* __restrict__ P,
              const YT* __restrict__ Ycur, const float2* __restrict__ Ym, float2* __restrict__ Ynext,
              bf162* __restrict__ Ynext16, float2* __restrict__ upd, float2* __restrict__ gains,
              const float2* __restrict__ frep_part, int chunks, int n_pad, Sched* sched, float eta, float min_gain,
              float alpha_export, float2* __restrict__ g_out, HeavyRows hv) {
  __shared__ float2 spart[kAttrCta][G];
  __shared__ int64_t srp[kAttrCta + 1];
  __shared__ int soff[kAttrCta + 1];
  __shared__ int swarp[kAttrCta / 32];
  __shared__ uint8_t srow[kAttrCta * G];  // (row, slot) pair -> row
  __shared__ int slevels;
  const int64_t row0 = (int64_t)blockIdx.x * kAttrCta;
  const int tid = threadIdx.x;
  for (int t = tid; t <= kAttrCta; t += kAttrCta) srp[t] = row0 + t <= n ? rp[row0 + t] : 0;
  if (tid == 0) slevels = 0;
  __syncthreads();
  // (1) the slots of this thread's row: slot s < G sums entries s, s + G, ...
  // of the row (short rows only); a hub row's chunk sums go to slot 0
  const int64_t i = row0 + tid;
  int ns = 0;
#pragma unroll
  for (int q = 0; q < G; ++q) spart[tid][q] = make_float2(0.f, 0.f);
  if (i < n) {
    const int64_t d = srp[tid + 1] - srp[tid];
    if (d <= kHeavyDeg) {
      ns = (int)(d < G ? d : G);
      if (d > 0) atomicMax(&slevels, (int)((d + G - 1) / G));  // entries per slot, at most
    } else {  // chunk sums from k_attract_heavy, in chunk order
      int lo = 0, hi = hv.count - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (hv.rows[mid] < i) lo = mid + 1; else hi = mid;
      }
      float ax = 0.f, ay = 0.f;
      for (int c = hv.chunk_off[lo]; c < hv.chunk_off[lo + 1]; ++c) {
        const float2 f = hv.fa[c];
        ax += f.x;
        ay += f.y;
      }
      spart[tid][0] = make_float2(ax, ay);
    }
  }
  block_excl_scan(ns, soff, swarp);
  __syncthreads();
  for (int q = 0; q < ns; ++q) srow[soff[tid] + q] = (uint8_t)tid;
  __syncthreads();
  // (2) the (row, slot) pairs in use, packed over the CTA's rows, level by
  // level: level k adds entry s + G k of each slot to its partial (the
  // fmaf chain of attract_entries, in the same order).  A pair belongs to
  // one thread at every level; each thread keeps kAttrPairs pairs' loads in
  // flight at once.
  const int nslots = soff[kAttrCta], levels = slevels;
  for (int k = 0; k < levels; ++k)
    for (int q0 = tid; q0 < nslots; q0 += kAttrPairs * kAttrCta) {
      int r[kAttrPairs], sl[kAttrPairs];
      int64_t e[kAttrPairs];
      bool ok[kAttrPairs];
#pragma unroll
      for (int m = 0; m < kAttrPairs; ++m) {
        const int q = q0 + m * kAttrCta;
        ok[m] = false;
        r[m] = 0;
        sl[m] = 0;
        e[m] = 0;
        if (q < nslots) {
          r[m] = srow[q];
          sl[m] = q - soff[r[m]];
          e[m] = srp[r[m]] + sl[m] + (int64_t)G * k;
          ok[m] = e[m] < srp[r[m] + 1];
        }
      }
      int32_t j[kAttrPairs];
      float pe[kAttrPairs];
#pragma unroll
      for (int m = 0; m < kAttrPairs; ++m) {
        j[m] = ok[m] ? col[e[m]] : 0;
        pe[m] = ok[m] ? ld_p(P, e[m]) : 0.f;
      }
      float2 yj[kAttrPairs], yi[kAttrPairs];
#pragma unroll
      for (int m = 0; m < kAttrPairs; ++m) {
        yj[m] = ok[m] ? ld_y(Ycur, j[m]) : make_float2(0.f, 0.f);
        yi[m] = ok[m] ? ld_y(Ycur, row0 + r[m]) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int m = 0; m < kAttrPairs; ++m)
        if (ok[m]) {
          float2 acc = spart[r[m]][sl[m]];
          const float dx = yi[m].x - yj[m].x, dy = yi[m].y - yj[m].y;
          const float w = 1.0f / fmaf(dy, dy, fmaf(dx, dx, 1.0f));
          const float pw = pe[m] * w;
          acc.x = fmaf(pw, dx, acc.x);
          acc.y = fmaf(pw, dy, acc.y);
          spart[r[m]][sl[m]] = acc;
        }
    }
  __syncthreads();
  if (i >= n) return;
  // (3) the row's sum in the order of group_sum<G> (xor butterfly: slot l
  // plus slot l ^ o for o = G/2, ..., 1), then the update
  static_assert(G == 8, "the butterfly below is written out for 8 slots");
  const float2* sp = spart[tid];
  float2 a0 = sp[0], a1 = sp[1], t = sp[4];
  a0 = make_float2(a0.x + t.x, a0.y + t.y);  // o = 4: slot l + slot l + 4
  t = sp[5];
  a1 = make_float2(a1.x + t.x, a1.y + t.y);
  float2 a2 = sp[2];
  t = sp[6];
  a2 = make_float2(a2.x + t.x, a2.y + t.y);
  float2 a3 = sp[3];
  t = sp[7];
  a3 = make_float2(a3.x + t.x, a3.y + t.y);
  a0 = make_float2(a0.x + a2.x, a0.y + a2.y);  // o = 2
  a1 = make_float2(a1.x + a3.x, a1.y + a3.y);
  const float2 fa = make_float2(a0.x + a1.x, a0.y + a1.y);  // o = 1
  finish_row<EXPORT>(i, fa, frep_part, chunks, n_pad, sched, alpha_export, g_out, Ym, Ynext, Ynext16, upd, gains,
                     eta, min_gain);
}

// Attraction of the long rows (more than kHeavyDeg entries), in chunks of at
// most kHeavyChunk entries: one warp per chunk, xor-butterfly reduction
// (fixed order), so no group of lanes serialises on a hub row.
template <class PT, class YT>
__global__ void __launch_bounds__(256)
    k_attract_heavy(HeavyRows hv, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                    const PT* __restrict__ P, const YT* __restrict__ Y) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < hv.chunks; c += warps) {
    const int64_t i = hv.chunk_row[c];
    const float2 yi = ld_y(Y, i);
    float ax = 0.f, ay = 0.f;
    attract_entries_pipelined<32, PT, YT>(hv.chunk_begin[c], hv.chunk_end[c], col, P, Y, i, lane, yi, ax, ay);
    ax = group_sum<32>(ax);
    ay = group_sum<32>(ay);
    if (lane == 0) hv.fa[c] = make_float2(ax, ay);
  }
}

__global__ void k_heavy_bounds(int H, const int32_t* __restrict__ rows, const int64_t* __restrict__ rp,
                               int64_t* __restrict__ bounds) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < H; k += gridDim.x * blockDim.x) {
    bounds[k] = rp[rows[k]];
    bounds[H + k] = rp[rows[k] + 1];
  }
}

__global__ void k_heavy_flags(int n, const int64_t* __restrict__ rp, int32_t* __restrict__ flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    flag[i] = (rp[i + 1] - rp[i]) > kHeavyDeg ? 1 : 0;
}

__global__ void k_heavy_scatter(int n, const int32_t* __restrict__ flag, const int64_t* __restrict__ pos,
                                int32_t* __restrict__ rows) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    if (flag[i]) rows[pos[i]] = (int32_t)i;
}

// F^r_i from the fixed-point accumulators (one rounding of the exact integer
// sum), which are cleared for the next pass; one thread per point.
__global__ void __launch_bounds__(kAttrCta)
    k_fix_forces(int n, unsigned long long* __restrict__ acc, float unscale, float2* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    ulonglong2* a = reinterpret_cast<ulonglong2*>(acc) + i;
    const ulonglong2 v = *a;
    out[i] = make_float2(__ll2float_rn((long long)v.x) * unscale, __ll2float_rn((long long)v.y) * unscale);
    *a = make_ulonglong2(0ull, 0ull);
  }
}

// F^r_i = the ordered-pair kernel's partial forces added in chunk order
// (fixed order: bit-reproducible); one thread per point.
__global__ void __launch_bounds__(kAttrCta)
    k_reduce_slots(int n, const float2* __restrict__ part, int slots, int n_pad, float2* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    float fx = 0.f, fy = 0.f;
    for (int k = 0; k < slots; ++k) {
      const float2 f = part[(size_t)k * n_pad + i];
      fx += f.x;
      fy += f.y;
    }
    out[i] = make_float2(fx, fy);
  }
}

// Pulls the layout into L2 (one sequential read) so that the neighbour
// gathers of the attraction hit L2 rather than DRAM sectors.
__global__ void k_prefetch_l2(const char* __restrict__ p, int64_t bytes) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * 128;
  for (int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 128; o < bytes; o += stride)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p + o));
}

template <class PT, class YT>
__global__ void __launch_bounds__(kAttrCta)
    k_kl(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const PT* __restrict__ P,
         const YT* __restrict__ Y, double* __restrict__ parts, Sched* sched) {
  double s1 = 0.0, s2 = 0.0;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const float2 yi = ld_y(Y, i);
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += 32) {
      const float p = ld_p(P, e);
      if (!(p > 0.f)) continue;
      if (!TS_IN(col[e], 0, n, &sched->flags)) continue;
      const float2 yj = ld_y(Y, col[e]);
      const float dx = yi.x - yj.x, dy = yi.y - yj.y;
      // ln(p / w) = ln p + ln(1 + d^2)
      s1 += (double)p * ((double)logf(p) + (double)log1pf(fmaf(dy, dy, dx * dx)));
      s2 += (double)p;
    }
  }
  const double b1 = block_sum_d(s1);
  const double b2 = block_sum_d(s2);
  if (threadIdx.x == 0) {
    parts[2 * blockIdx.x] = b1;
    parts[2 * blockIdx.x + 1] = b2;
  }
  if (arrive_last(&sched->red_done)) {
    double t1 = 0.0, t2 = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
      t1 += __ldcg(parts + 2 * k);
      t2 += __ldcg(parts + 2 * k + 1);
    }
    t1 = block_sum_d(t1);
    t2 = block_sum_d(t2);
    if (threadIdx.x == 0) {
      sched->red[0] = t1;
      sched->red[1] = t2;
    }
  }
}

// SplitMix64 (Steele, Lea, Flood 2014) in counter mode: draw c of a key.
__device__ __forceinline__ uint64_t splitmix_at(uint64_t key, uint64_t c) {
  uint64_t z = key + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_init_Y(int n, uint64_t key, float sigma, float2* __restrict__ Y) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    // Box-Muller on two 53-bit uniforms: u1 in (0, 1], u2 in [0, 1)
    const double u1 = 1.0 - (double)(splitmix_at(key, 2 * i) >> 11) * (1.0 / 9007199254740992.0);
    const double u2 = (double)(splitmix_at(key, 2 * i + 1) >> 11) * (1.0 / 9007199254740992.0);
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    Y[i] = make_float2((float)(sigma * r * cs), (float)(sigma * r * sn));
  }
}

__global__ void k_fill2(float2* a, int64_t lo, int64_t hi, float v) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < hi; k += stride) a[k] = make_float2(v, v);
}

__global__ void k_to_bf16(const float* __restrict__ in, bf16* __restrict__ out, int64_t count) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride)
    out[k] = __float2bfloat16_rn(in[k]);
}

int grid_rows(int64_t n, int per_cta) {
  int64_t g = (n + per_cta - 1) / per_cta;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

int kl_partial_count(int sm_count) { return sm_count * 4; }

tsgne_status launch_reduce_slots(int n, const float2* part, int slots, int n_pad, float2* out, cudaStream_t s) {
  k_reduce_slots<<<grid_rows(n, kAttrCta), kAttrCta, 0, s>>>(n, part, slots, n_pad, out);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

tsgne_status launch_fix_forces(int n, unsigned long long* acc, float2* out, cudaStream_t s) {
  const int g = grid_rows(n, kAttrCta);
  k_fix_forces<<<g, kAttrCta, 0, s>>>(n, acc, fix_unscale(n), out);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

tsgne_status launch_prefetch_l2(const void* p, int64_t bytes, cudaStream_t s) {
  if (bytes < (1 << 20)) return TSGNE_OK;  // small layouts stay in L2 anyway
  const int64_t lines = (bytes + 127) / 128;
  const int g = (int)((lines + 255) / 256 < 2048 ? (lines + 255) / 256 : 2048);
  k_prefetch_l2<<<g, 256, 0, s>>>(static_cast<const char*>(p), bytes);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

tsgne_status find_heavy_rows(int n, const int64_t* rp, HeavyStore& hs, cudaStream_t s) {
  DevBuf<int32_t> flag;
  DevBuf<int64_t> pos, scr;
  TS_TRY(flag.alloc((size_t)n));
  TS_TRY(pos.alloc((size_t)n + 1));
  TS_TRY(scr.alloc(scan_scratch_bytes(n) / sizeof(int64_t)));
  const int g = grid_rows(n, 256) < 4096 ? grid_rows(n, 256) : 4096;
  k_heavy_flags<<<g, 256, 0, s>>>(n, rp, flag.get());
  TS_TRY(scan_i32_to_i64(flag.get(), pos.get(), n, scr.get(), s));
  int64_t total = 0;
  TS_CUDA(cudaMemcpyAsync(&total, pos.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TS_CUDA(cudaStreamSynchronize(s));
  const int H = (int)total;
  hs.count = H;
  TS_TRY(hs.rows.alloc((size_t)(H > 0 ? H : 1)));
  if (H > 0) k_heavy_scatter<<<g, 256, 0, s>>>(n, flag.get(), pos.get(), hs.rows.get());
  TS_CUDA(cudaGetLastError());
  // chunk lists on the host (the hub rows are few)
  std::vector<int32_t> rows(H > 0 ? H : 1);
  std::vector<int64_t> b(H > 0 ? H : 1), e(H > 0 ? H : 1);
  if (H > 0) {
    DevBuf<int64_t> bounds;
    TS_TRY(bounds.alloc(2 * (size_t)H));
    k_heavy_bounds<<<(H + 255) / 256, 256, 0, s>>>(H, hs.rows.get(), rp, bounds.get());
    TS_CUDA(cudaGetLastError());
    TS_CUDA(cudaMemcpyAsync(rows.data(), hs.rows.get(), sizeof(int32_t) * H, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaMemcpyAsync(b.data(), bounds.get(), sizeof(int64_t) * H, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaMemcpyAsync(e.data(), bounds.get() + H, sizeof(int64_t) * H, cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<int32_t> off(1, 0), crow, cheavy;
  std::vector<int64_t> cb, ce;
  for (int k = 0; k < H; ++k) {
    for (int64_t x = b[k]; x < e[k]; x += kHeavyChunk) {
      crow.push_back(rows[k]);
      cheavy.push_back(k);
      cb.push_back(x);
      ce.push_back(x + kHeavyChunk < e[k] ? x + kHeavyChunk : e[k]);
    }
    off.push_back((int32_t)crow.size());
  }
  const int C = (int)crow.size();
  hs.chunks = C;
  TS_TRY(hs.chunk_off.alloc(off.size()));
  TS_TRY(hs.chunk_row.alloc((size_t)(C > 0 ? C : 1)));
  TS_TRY(hs.chunk_begin.alloc((size_t)(C > 0 ? C : 1)));
  TS_TRY(hs.chunk_end.alloc((size_t)(C > 0 ? C : 1)));
  TS_TRY(hs.fa.alloc((size_t)(C > 0 ? C : 1)));
  TS_TRY(hs.chunk_heavy.alloc((size_t)(C > 0 ? C : 1)));
  TS_TRY(hs.arrivals.alloc((size_t)(H > 0 ? H : 1)));
  TS_CUDA(cudaMemsetAsync(hs.arrivals.get(), 0, sizeof(uint32_t) * (size_t)(H > 0 ? H : 1), s));
  TS_CUDA(cudaMemcpyAsync(hs.chunk_off.get(), off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice, s));
  if (C > 0) {
    TS_CUDA(cudaMemcpyAsync(hs.chunk_heavy.get(), cheavy.data(), sizeof(int32_t) * C, cudaMemcpyHostToDevice, s));
    TS_CUDA(cudaMemcpyAsync(hs.chunk_row.get(), crow.data(), sizeof(int32_t) * C, cudaMemcpyHostToDevice, s));
    TS_CUDA(cudaMemcpyAsync(hs.chunk_begin.get(), cb.data(), sizeof(int64_t) * C, cudaMemcpyHostToDevice, s));
    TS_CUDA(cudaMemcpyAsync(hs.chunk_end.get(), ce.data(), sizeof(int64_t) * C, cudaMemcpyHostToDevice, s));
  }
  TS_CUDA(cudaStreamSynchronize(s));
  return TSGNE_OK;
}

tsgne_status launch_kl(int n, const int64_t* rp, const int32_t* col, const void* P, int p_bf16, const void* Y,
                       int y_bf16, double* partials, int nparts, Sched* sched, cudaStream_t s) {
  if (p_bf16 && y_bf16)
    k_kl<bf16, bf162><<<nparts, kAttrCta, 0, s>>>(n, rp, col, static_cast<const bf16*>(P),
                                                  static_cast<const bf162*>(Y), partials, sched);
  else if (!p_bf16 && !y_bf16)
    k_kl<float, float2><<<nparts, kAttrCta, 0, s>>>(n, rp, col, static_cast<const float*>(P),
                                                    static_cast<const float2*>(Y), partials, sched);
  else {
    last_msg() = "KL needs P and Y in the same storage precision";
    return TSGNE_ERR_INVALID_ARG;
  }
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

namespace {

template <bool EXPORT, class PT, class YT>
tsgne_status attract_t(const AttractArgs& a, float alpha, float2* g, cudaStream_t s) {
  k_attract<kG, EXPORT, PT, YT><<<grid_rows(a.n, kAttrCta), kAttrCta, 0, s>>>(
      a.n, a.rp, a.col, static_cast<const PT*>(a.P), static_cast<const YT*>(a.Yr), a.Ym, a.Ynext,
      static_cast<bf162*>(a.Ynext16), a.upd, a.gains, a.frep, a.chunks, a.n_pad, a.sched, a.eta, a.min_gain, alpha,
      g, a.hv);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

template <bool EXPORT>
tsgne_status attract_dispatch(const AttractArgs& a, float alpha, float2* g, cudaStream_t s) {
  if (a.p_bf16 && a.y_bf16) return attract_t<EXPORT, bf16, bf162>(a, alpha, g, s);
  if (!a.p_bf16 && !a.y_bf16) return attract_t<EXPORT, float, float2>(a, alpha, g, s);
  last_msg() = "P and Y must share a storage precision";
  return TSGNE_ERR_INVALID_ARG;
}

template <class PT, class YT>
tsgne_status heavy_t(const AttractArgs& a, cudaStream_t s) {
  const int g = (a.hv.chunks + 7) / 8 < 16384 ? (a.hv.chunks + 7) / 8 : 16384;
  k_attract_heavy<PT, YT><<<g, 256, 0, s>>>(a.hv, a.rp, a.col, static_cast<const PT*>(a.P),
                                            static_cast<const YT*>(a.Yr));
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

}  // namespace

tsgne_status launch_attract_heavy(const AttractArgs& a, cudaStream_t s) {
  if (a.hv.chunks <= 0) return TSGNE_OK;
  if (a.p_bf16 && a.y_bf16) return heavy_t<bf16, bf162>(a, s);
  if (!a.p_bf16 && !a.y_bf16) return heavy_t<float, float2>(a, s);
  last_msg() = "P and Y must share a storage precision";
  return TSGNE_ERR_INVALID_ARG;
}

tsgne_status launch_gradient(const AttractArgs& a, float alpha, float2* g, cudaStream_t s) {
  TS_TRY(launch_prefetch_l2(a.Yr, (int64_t)a.n * (a.y_bf16 ? 4 : 8), s));
  TS_TRY(launch_attract_heavy(a, s));
  return attract_dispatch<true>(a, alpha, g, s);
}

tsgne_status launch_to_bf16(const float* in, void* out, int64_t count, cudaStream_t s) {
  if (count <= 0) return TSGNE_OK;
  const int g = grid_rows(count, 256) < 8192 ? grid_rows(count, 256) : 8192;
  k_to_bf16<<<g, 256, 0, s>>>(in, static_cast<bf16*>(out), count);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

tsgne_status launch_init_Y(int n, uint64_t seed, float sigma, float2* Y, cudaStream_t s) {
  // key = SplitMix64 output of the seed itself (stream separation from user seeds)
  uint64_t z = seed + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  const uint64_t key = z ^ (z >> 31);
  k_init_Y<<<grid_rows(n, 256) < 4096 ? grid_rows(n, 256) : 4096, 256, 0, s>>>(n, key, sigma, Y);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

tsgne_status launch_fill_sentinel(float2* Y, int lo, int hi, cudaStream_t s) {
  if (hi <= lo) return TSGNE_OK;
  k_fill2<<<grid_rows(hi - lo, 256) < 1024 ? grid_rows(hi - lo, 256) : 1024, 256, 0, s>>>(Y, lo, hi, kSentinel);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

tsgne_status launch_fill2(float2* a, int n, float v, cudaStream_t s) {
  if (n <= 0) return TSGNE_OK;
  k_fill2<<<grid_rows(n, 256) < 1024 ? grid_rows(n, 256) : 1024, 256, 0, s>>>(a, 0, n, v);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

}  // namespace tsgne
