// Neighbour structure of t-SGNE (Eq. 7 with the graph's own edges as the
// neighbour set, Sec. 2.2): N(i) = { j != i : (i,j) or (j,i) in G }, rows
// sorted ascending and unique, plus the transpose-slot map tslot[e] = position
// of (j,i) for entry e = (i,j).
//
// Pipeline (all on the device):
//   validate -> count both directions -> scan -> fill (atomic cursors, any
//   order) -> per-row sort + unique (three tiers by row length: a warp in
//   registers, a CTA in shared memory, or a CTA with a bitmap over [0, n) for
//   hub rows) -> scan of unique counts -> compact -> tslot by binary search.
// The per-row sort makes the result independent of the fill order, so the
// structure is bit-identical from run to run.
#include <climits>

#include "tsgne_internal.cuh"

namespace tsgne {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanPerBlock = 2 * kScanThreads;
static_assert(kScanPerBlock == kScanBlock, "block size of scan_i32_to_i64_blocks");
constexpr int kMidCap = 4096;  // longest row sorted in shared memory

// Exclusive block-wide scan of one value per thread; *total gets the block sum.
__device__ int64_t block_excl_scan(int64_t v, int64_t* total) {
  __shared__ int64_t wsum[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t s = lane < nw ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    wsum[lane] = s;
  }
  __syncthreads();
  int64_t pre = wid ? wsum[wid - 1] : 0;
  *total = wsum[nw - 1];
  __syncthreads();
  return pre + x - v;
}

__global__ void k_scan_local(const int32_t* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                             int64_t* __restrict__ bsum) {
  const int64_t base = (int64_t)blockIdx.x * kScanPerBlock + 2 * threadIdx.x;
  int64_t a = base < n ? in[base] : 0;
  int64_t b = base + 1 < n ? in[base + 1] : 0;
  int64_t tot;
  int64_t pre = block_excl_scan(a + b, &tot);
  if (base < n) out[base] = pre;
  if (base + 1 < n) out[base + 1] = pre + a;
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// Single CTA: exclusive scan of the block sums in place, total to bsum[nb].
__global__ void k_scan_sums(int64_t* bsum, int nb) {
  int64_t carry = 0;
  for (int c = 0; c < nb; c += blockDim.x) {
    int k = c + threadIdx.x;
    int64_t v = k < nb ? bsum[k] : 0;
    int64_t tot;
    int64_t pre = block_excl_scan(v, &tot);
    if (k < nb) bsum[k] = carry + pre;
    carry += tot;
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ bsum, int nb) {
  const int64_t base = (int64_t)blockIdx.x * kScanPerBlock + 2 * threadIdx.x;
  const int64_t add = bsum[blockIdx.x];
  if (base < n) out[base] += add;
  if (base + 1 < n) out[base + 1] += add;
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = bsum[nb];
}

// ------------------------------------------------------------------ K0

__global__ void k_validate(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t m,
                           uint32_t* bad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    if (rp[i] > rp[i + 1]) atomicOr(bad, 1u);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    int32_t j = col[e];
    if (j < 0 || j >= n) atomicOr(bad, 2u);
  }
}

// One warp per row: both directions of every non-loop entry.
__global__ void k_count(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int32_t* cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += 32) {
      int32_t j = col[e];
      if (j == i) continue;
      atomicAdd(&cnt[i], 1);
      atomicAdd(&cnt[j], 1);
    }
  }
}

__global__ void k_fill(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                       const int64_t* __restrict__ off, int32_t* cur, int32_t* __restrict__ raw) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += 32) {
      int32_t j = col[e];
      if (j == i) continue;
      raw[off[i] + atomicAdd(&cur[i], 1)] = j;
      raw[off[j] + atomicAdd(&cur[j], 1)] = (int32_t)i;
    }
  }
}

// Rows longer than a warp go to the CTA tiers.
__global__ void k_classify(int n, const int64_t* __restrict__ off, int32_t* mid, int32_t* hub, int32_t* counts) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    int64_t len = off[i + 1] - off[i];
    if (len > 32 && len <= kMidCap) mid[atomicAdd(&counts[0], 1)] = (int32_t)i;
    else if (len > kMidCap) hub[atomicAdd(&counts[1], 1)] = (int32_t)i;
  }
}

// Tier A: rows of <= 32 entries, one warp, bitonic sort across lanes.
__global__ void k_sort_small(int n, const int64_t* __restrict__ off, int32_t* __restrict__ raw,
                             int32_t* __restrict__ ucnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const int64_t a = off[i];
    const int64_t len = off[i + 1] - a;
    if (len > 32) continue;  // uniform across the warp
    int32_t v = lane < len ? raw[a + lane] : INT_MAX;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        int32_t p = __shfl_xor_sync(0xffffffffu, v, j);
        bool take_min = ((lane & j) == 0) == ((lane & k) == 0);
        v = take_min ? min(v, p) : max(v, p);
      }
    }
    int32_t prev = __shfl_up_sync(0xffffffffu, v, 1);
    bool keep = v != INT_MAX && (lane == 0 || v != prev);
    unsigned mask = __ballot_sync(0xffffffffu, keep);
    if (keep) raw[a + __popc(mask & ((1u << lane) - 1u))] = v;
    if (lane == 0) ucnt[i] = __popc(mask);
  }
}

// Tier B: 32 < len <= kMidCap, one CTA per row, bitonic sort in shared memory.
__global__ void __launch_bounds__(512) k_sort_mid(const int32_t* __restrict__ rows, int nrows,
                                                  const int64_t* __restrict__ off, int32_t* __restrict__ raw,
                                                  int32_t* __restrict__ ucnt) {
  __shared__ int32_t s[kMidCap];
  constexpr int kPer = kMidCap / 512;
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int i = rows[r];
    const int64_t a = off[i];
    const int len = (int)(off[i + 1] - a);
    int L = 64;
    while (L < len) L <<= 1;
    for (int t = threadIdx.x; t < L; t += blockDim.x) s[t] = t < len ? raw[a + t] : INT_MAX;
    __syncthreads();
    for (int k = 2; k <= L; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < L; t += blockDim.x) {
          int x = t ^ j;
          if (x > t) {
            int32_t u = s[t], w = s[x];
            bool asc = (t & k) == 0;
            if (asc ? (u > w) : (u < w)) { s[t] = w; s[x] = u; }
          }
        }
        __syncthreads();
      }
    }
    // unique + compaction: thread t owns s[t*kPer .. t*kPer+kPer)
    int cntk = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      int t = threadIdx.x * kPer + q;
      if (t < L && s[t] != INT_MAX && (t == 0 || s[t] != s[t - 1])) ++cntk;
    }
    int64_t tot;
    int64_t pos = block_excl_scan(cntk, &tot);
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      int t = threadIdx.x * kPer + q;
      if (t < L && s[t] != INT_MAX && (t == 0 || s[t] != s[t - 1])) raw[a + pos++] = s[t];
    }
    if (threadIdx.x == 0) ucnt[i] = (int32_t)tot;
    __syncthreads();
  }
}

// Tier C: hub rows, one CTA per row with a private bitmap over [0, n).
__global__ void __launch_bounds__(512) k_sort_hub(const int32_t* __restrict__ rows, int nrows,
                                                  const int64_t* __restrict__ off, int32_t* __restrict__ raw,
                                                  int32_t* __restrict__ ucnt, uint32_t* __restrict__ bitmaps,
                                                  int words) {
  constexpr int kPer = 8;
  uint32_t* bm = bitmaps + (size_t)blockIdx.x * words;
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int i = rows[r];
    const int64_t a = off[i];
    const int64_t len = off[i + 1] - a;
    for (int w = threadIdx.x; w < words; w += blockDim.x) bm[w] = 0u;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
      int32_t v = raw[a + t];
      atomicOr(&bm[v >> 5], 1u << (v & 31));
    }
    __syncthreads();
    int64_t base = 0;
    for (int c = 0; c < words; c += blockDim.x * kPer) {
      int cntk = 0;
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        int w = c + threadIdx.x * kPer + q;
        if (w < words) cntk += __popc(bm[w]);
      }
      int64_t tot;
      int64_t pos = base + block_excl_scan(cntk, &tot);
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        int w = c + threadIdx.x * kPer + q;
        if (w < words) {
          uint32_t bits = bm[w];
          while (bits) {
            int b = __ffs(bits) - 1;
            bits &= bits - 1u;
            raw[a + pos++] = w * 32 + b;
          }
        }
      }
      base += tot;
    }
    if (threadIdx.x == 0) ucnt[i] = (int32_t)base;
    __syncthreads();
  }
}

__global__ void k_compact(int n, const int64_t* __restrict__ off, const int32_t* __restrict__ raw,
                          const int64_t* __restrict__ rp, int32_t* __restrict__ col) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const int64_t a = off[i], b = rp[i], len = rp[i + 1] - b;
    for (int64_t t = lane; t < len; t += 32) col[b + t] = raw[a + t];
  }
}

__global__ void k_tslot(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                        int64_t* __restrict__ tslot, uint32_t* bad) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += 32) {
      const int32_t j = col[e];
      int64_t lo = rp[j], hi = rp[j + 1] - 1, found = -1;
      while (lo <= hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        int32_t v = col[mid];
        if (v == (int32_t)i) { found = mid; break; }
        if (v < (int32_t)i) lo = mid + 1; else hi = mid - 1;
      }
      if (found < 0) { atomicOr(bad, 4u); found = e; }
      tslot[e] = found;
    }
  }
}

// k nearest neighbours by breadth-first search on the structure (Eq. 7 with
// k nodes per list, Sec. 2.2): one warp per source i; its list in shared
// memory doubles as the BFS queue.  Levels come in order because the queue is
// processed in order; each node's sorted neighbours are taken 32 at a time,
// lanes test their candidate against the list (and i), and the fresh ones are
// appended in lane (= ascending id) order until k are found.
constexpr int kKnnMax = 256;
constexpr int kKnnWarps = 8;

__global__ void __launch_bounds__(32 * kKnnWarps)
    k_bfs_knn(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int k,
              int32_t* __restrict__ out, int32_t* __restrict__ cnt) {
  __shared__ int32_t lists[kKnnWarps][kKnnMax];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* L = lists[wid];
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < n; s += warps) {
    int c = 0;
    for (int head = -1; head < c && c < k; ++head) {
      const int64_t u = head < 0 ? s : L[head];
      const int64_t b = rp[u + 1];
      for (int64_t e0 = rp[u]; e0 < b && c < k; e0 += 32) {
        const int64_t e = e0 + lane;
        const int32_t v = e < b ? col[e] : -1;
        bool fresh = v >= 0 && v != (int32_t)s;
        for (int t = 0; fresh && t < c; ++t)
          if (L[t] == v) fresh = false;
        const unsigned mask = __ballot_sync(0xffffffffu, fresh);
        const int pos = c + __popc(mask & ((1u << lane) - 1u));
        if (fresh && pos < k) L[pos] = v;
        c = min(k, c + __popc(mask));
        __syncwarp();
      }
    }
    for (int t = lane; t < c; t += 32) out[s * k + t] = L[t];
    if (lane == 0) cnt[s] = c;
    __syncwarp();
  }
}

__global__ void k_iota_stride(int n, int64_t stride_k, int64_t* __restrict__ off) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
    off[i] = i * stride_k;
}

int grid_for(int64_t work, int per_cta, int cap) {
  int64_t g = (work + per_cta - 1) / per_cta;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

size_t scan_scratch_bytes(int64_t n) {
  int64_t nb = (n + kScanPerBlock - 1) / kScanPerBlock;
  if (nb < 1) nb = 1;
  return sizeof(int64_t) * (size_t)(nb + 1);
}

tsgne_status scan_i32_to_i64_blocks(const int32_t* in, int64_t* out, int64_t n, void* scratch, cudaStream_t s) {
  int64_t nb = (n + kScanPerBlock - 1) / kScanPerBlock;
  if (nb < 1) nb = 1;
  int64_t* bsum = static_cast<int64_t*>(scratch);
  k_scan_local<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, bsum);
  k_scan_sums<<<1, kScanThreads, 0, s>>>(bsum, (int)nb);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

tsgne_status scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, void* scratch, cudaStream_t s) {
  int64_t nb = (n + kScanPerBlock - 1) / kScanPerBlock;
  if (nb < 1) nb = 1;
  int64_t* bsum = static_cast<int64_t*>(scratch);
  k_scan_local<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, bsum);
  k_scan_sums<<<1, kScanThreads, 0, s>>>(bsum, (int)nb);
  k_scan_add<<<(unsigned)nb, kScanThreads, 0, s>>>(out, n, bsum, (int)nb);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

tsgne_status build_structure(int n, const int64_t* rp_in, const int32_t* col_in, int64_t m, DevBuf<int64_t>& rp_out,
                             DevBuf<int32_t>& col_out, DevBuf<int64_t>& tslot_out, int64_t* nnz_out, Sched* sched,
                             cudaStream_t s) {
  (void)sched;
  const int kWarpRowsCta = 256;  // 8 warps per CTA for warp-per-row kernels
  int dev = 0, sms = 1;
  TS_CUDA(cudaGetDevice(&dev));
  TS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int cap = sms * 32;

  DevBuf<uint32_t> flag;
  TS_TRY(flag.alloc(1));
  TS_CUDA(cudaMemsetAsync(flag.get(), 0, sizeof(uint32_t), s));
  k_validate<<<grid_for(m > n ? m : n, 256, cap), 256, 0, s>>>(n, rp_in, col_in, m, flag.get());
  TS_CUDA(cudaGetLastError());
  uint32_t bad = 0;
  TS_CUDA(cudaMemcpyAsync(&bad, flag.get(), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  TS_CUDA(cudaStreamSynchronize(s));
  if (bad) {
    last_msg() = (bad & 1u) ? "row_ptr is decreasing" : "column index outside [0, n)";
    return TSGNE_ERR_BAD_CSR;
  }

  DevBuf<int32_t> cnt, cur, raw, ucnt, lists, counts;
  DevBuf<int64_t> off, scr;
  TS_TRY(cnt.alloc(n));
  TS_TRY(cur.alloc(n));
  TS_TRY(ucnt.alloc(n));
  TS_TRY(off.alloc((size_t)n + 1));
  TS_TRY(raw.alloc((size_t)(2 * m)));
  TS_TRY(lists.alloc((size_t)2 * n));
  TS_TRY(counts.alloc(2));
  TS_TRY(scr.alloc(scan_scratch_bytes(n) / sizeof(int64_t)));
  TS_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t) * n, s));
  TS_CUDA(cudaMemsetAsync(cur.get(), 0, sizeof(int32_t) * n, s));
  TS_CUDA(cudaMemsetAsync(counts.get(), 0, sizeof(int32_t) * 2, s));

  const int wgrid = grid_for((int64_t)n * 32, kWarpRowsCta, cap);
  k_count<<<wgrid, kWarpRowsCta, 0, s>>>(n, rp_in, col_in, cnt.get());
  TS_TRY(scan_i32_to_i64(cnt.get(), off.get(), n, scr.get(), s));
  k_fill<<<wgrid, kWarpRowsCta, 0, s>>>(n, rp_in, col_in, off.get(), cur.get(), raw.get());
  k_classify<<<grid_for(n, 256, cap), 256, 0, s>>>(n, off.get(), lists.get(), lists.get() + n, counts.get());
  k_sort_small<<<wgrid, kWarpRowsCta, 0, s>>>(n, off.get(), raw.get(), ucnt.get());
  TS_CUDA(cudaGetLastError());
  int32_t hc[2] = {0, 0};
  TS_CUDA(cudaMemcpyAsync(hc, counts.get(), sizeof(hc), cudaMemcpyDeviceToHost, s));
  TS_CUDA(cudaStreamSynchronize(s));
  if (hc[0] > 0) k_sort_mid<<<hc[0] < cap ? hc[0] : cap, 512, 0, s>>>(lists.get(), hc[0], off.get(), raw.get(), ucnt.get());
  DevBuf<uint32_t> bitmaps;
  if (hc[1] > 0) {
    const int words = (n + 31) / 32;
    const int hgrid = hc[1] < 2 * sms ? hc[1] : 2 * sms;
    TS_TRY(bitmaps.alloc((size_t)words * hgrid));
    k_sort_hub<<<hgrid, 512, 0, s>>>(lists.get() + n, hc[1], off.get(), raw.get(), ucnt.get(), bitmaps.get(), words);
  }
  TS_CUDA(cudaGetLastError());

  TS_TRY(rp_out.alloc((size_t)n + 1));
  TS_TRY(scan_i32_to_i64(ucnt.get(), rp_out.get(), n, scr.get(), s));
  int64_t nnz = 0;
  TS_CUDA(cudaMemcpyAsync(&nnz, rp_out.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TS_CUDA(cudaStreamSynchronize(s));
  TS_TRY(col_out.alloc((size_t)nnz));
  TS_TRY(tslot_out.alloc((size_t)nnz));
  k_compact<<<wgrid, kWarpRowsCta, 0, s>>>(n, off.get(), raw.get(), rp_out.get(), col_out.get());
  TS_CUDA(cudaMemsetAsync(flag.get(), 0, sizeof(uint32_t), s));
  k_tslot<<<wgrid, kWarpRowsCta, 0, s>>>(n, rp_out.get(), col_out.get(), tslot_out.get(), flag.get());
  TS_CUDA(cudaGetLastError());
  TS_CUDA(cudaMemcpyAsync(&bad, flag.get(), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  TS_CUDA(cudaStreamSynchronize(s));
  if (bad) {
    last_msg() = "internal: structure is not symmetric";
    return TSGNE_ERR_CUDA;
  }
  *nnz_out = nnz;
  return TSGNE_OK;
}

}  // namespace tsgne

namespace tsgne {

tsgne_status build_neighbor_structure(int n, const int64_t* rp_in, const int32_t* col_in, int64_t m, int k_nn,
                                      DevBuf<int64_t>& rp_out, DevBuf<int32_t>& col_out, DevBuf<int64_t>& tslot_out,
                                      int64_t* nnz_out, cudaStream_t s) {
  if (k_nn <= 0) return build_structure(n, rp_in, col_in, m, rp_out, col_out, tslot_out, nnz_out, nullptr, s);
  if (k_nn > kKnnMax) {
    last_msg() = "k_nn above 256";
    return TSGNE_ERR_INVALID_ARG;
  }
  DevBuf<int64_t> rp1, tslot1, off, krp, scr;
  DevBuf<int32_t> col1, lists, cnt, kcol;
  int64_t nnz1 = 0;
  TS_TRY(build_structure(n, rp_in, col_in, m, rp1, col1, tslot1, &nnz1, nullptr, s));
  tslot1.reset();
  int dev = 0, sms = 1;
  TS_CUDA(cudaGetDevice(&dev));
  TS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  TS_TRY(lists.alloc((size_t)n * k_nn));
  TS_TRY(cnt.alloc((size_t)n));
  const int g = grid_for((int64_t)n * 32, 32 * kKnnWarps, sms * 32);
  k_bfs_knn<<<g, 32 * kKnnWarps, 0, s>>>(n, rp1.get(), col1.get(), k_nn, lists.get(), cnt.get());
  TS_CUDA(cudaGetLastError());
  TS_TRY(krp.alloc((size_t)n + 1));
  TS_TRY(scr.alloc(scan_scratch_bytes(n) / sizeof(int64_t)));
  TS_TRY(scan_i32_to_i64(cnt.get(), krp.get(), n, scr.get(), s));
  int64_t total = 0;
  TS_CUDA(cudaMemcpyAsync(&total, krp.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TS_CUDA(cudaStreamSynchronize(s));
  TS_TRY(kcol.alloc((size_t)(total > 0 ? total : 1)));
  TS_TRY(off.alloc((size_t)n + 1));
  k_iota_stride<<<grid_for((int64_t)n + 1, 256, sms * 8), 256, 0, s>>>(n, k_nn, off.get());
  k_compact<<<grid_for((int64_t)n * 32, 256, sms * 32), 256, 0, s>>>(n, off.get(), lists.get(), krp.get(), kcol.get());
  TS_CUDA(cudaGetLastError());
  lists.reset();
  return build_structure(n, krp.get(), kcol.get(), total, rp_out, col_out, tslot_out, nnz_out, nullptr, s);
}

}  // namespace tsgne
