// Random-walk estimate of the conditional affinities (Sec. 2.1, Eq. 6) on
// the neighbour graph of Eq. 7, the paper's alternative to the perplexity
// bisection of Eq. 2:
//
//   - a step from u goes to v in N(u) with probability proportional to
//     exp(-||x_u - x_v||^2) (the printed exponent's sign read as negative;
//     squared distances are shifted by the row minimum first, which leaves
//     the probabilities unchanged); a node without neighbours keeps the walk;
//   - R walks of L steps start at every node; p_{j|i} = (walks from i that
//     end at j) / R for j != i (walks back at i are dropped, p_ii = 0);
//   - the joint P is then Eq. 3 on the symmetrised set of walk pairs.
//
// Step s of walk r from node i draws U from output k = 1 + (i R + r) L + s of
// the SplitMix64 sequence seeded with seed ^ 0xD1B54A32D192ED03 (state =
// seed + k * 0x9E3779B97F4A7C15, then the published mix), U = (out >> 11) *
// 2^-53, and takes the first neighbour whose running weight sum exceeds
// U * (row total).  Distances (dimensions in index order) and the running
// sums are FP64 with _rn intrinsics, so the choices are those of the CPU
// reference up to the last-ulp behaviour of exp().
//
// Kernels: per-entry squared distances (warp per row), per-row running
// weight sums (thread per row, sequential like the definition), one thread
// per walk, then one warp per node sorts its R end points in shared memory
// and keeps the distinct ones with their counts.
#include <cmath>

#include "tsgne_internal.cuh"

namespace tsgne {

namespace {

constexpr int kRwWarps = 8;

__device__ __forceinline__ uint64_t sm64_output(uint64_t seed, uint64_t k) {
  uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void __launch_bounds__(32 * kRwWarps)
    k_rw_dist(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const float* __restrict__ X,
              int d, double* __restrict__ d2) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * kRwWarps;
  for (int64_t u = (int64_t)blockIdx.x * kRwWarps + (threadIdx.x >> 5); u < n; u += warps) {
    const float* xu = X + u * d;
    for (int64_t e = rp[u] + lane; e < rp[u + 1]; e += 32) {
      const float* xv = X + (int64_t)col[e] * d;
      double s = 0.0;
      for (int k = 0; k < d; ++k) {
        const double t = __dsub_rn((double)xu[k], (double)xv[k]);
        s = __dadd_rn(s, __dmul_rn(t, t));
      }
      d2[e] = s;
    }
  }
}

__global__ void k_rw_cumw(int n, const int64_t* __restrict__ rp, const double* __restrict__ d2,
                          double* __restrict__ cw) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  const int64_t a = rp[u], b = rp[u + 1];
  double dmin = INFINITY;
  for (int64_t e = a; e < b; ++e) dmin = fmin(dmin, d2[e]);
  double run = 0.0;
  for (int64_t e = a; e < b; ++e) {
    run = __dadd_rn(run, exp(-__dsub_rn(d2[e], dmin)));
    cw[e] = run;
  }
}

__global__ void k_rw_walks(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double* __restrict__ cw, int R, int L, uint64_t s0, int32_t* __restrict__ ends) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= (int64_t)n * R) return;
  const int64_t i = w / R;
  int32_t u = (int32_t)i;
  for (int s = 0; s < L; ++s) {
    const uint64_t k = 1ull + (uint64_t)w * (uint64_t)L + (uint64_t)s;
    const double U = (double)(sm64_output(s0, k) >> 11) * (1.0 / 9007199254740992.0);
    const int64_t a = rp[u], b = rp[u + 1];
    if (a == b) continue;
    const double target = __dmul_rn(U, cw[b - 1]);
    int64_t lo = a, hi = b - 1;  // first e with cw[e] > target; the last entry if none
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (cw[mid] > target) hi = mid; else lo = mid + 1;
    }
    u = col[lo];
  }
  ends[w] = u == (int32_t)i ? -1 : u;
}

// Warp per node: its R end points sorted (rank by counting), distinct
// values kept with their multiplicities; -1 (returned walks) dropped.
__global__ void __launch_bounds__(32 * kRwWarps)
    k_rw_count(int n, int R, const int32_t* __restrict__ ends, int32_t* __restrict__ ucol,
               int32_t* __restrict__ ucnt, int32_t* __restrict__ nuniq) {
  extern __shared__ int32_t sh[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* v = sh + (size_t)wid * 2 * R;
  int32_t* srt = v + R;
  const int64_t warps = (int64_t)gridDim.x * kRwWarps;
  for (int64_t i = (int64_t)blockIdx.x * kRwWarps + wid; i < n; i += warps) {
    for (int t = lane; t < R; t += 32) v[t] = ends[i * R + t];
    __syncwarp();
    for (int t = lane; t < R; t += 32) {
      const int32_t x = v[t];
      int rank = 0;
      for (int q = 0; q < R; ++q) {
        const int32_t y = v[q];
        rank += (y < x) || (y == x && q < t);
      }
      srt[rank] = x;
    }
    __syncwarp();
    int base = 0;
    for (int t0 = 0; t0 < R; t0 += 32) {
      const int t = t0 + lane;
      const bool head = t < R && srt[t] >= 0 && (t == 0 || srt[t - 1] != srt[t]);
      const uint32_t hm = __ballot_sync(0xffffffffu, head);
      if (head) {
        int e = t + 1;
        while (e < R && srt[e] == srt[t]) ++e;
        const int slot = base + __popc(hm & ((1u << lane) - 1u));
        ucol[i * R + slot] = srt[t];
        ucnt[i * R + slot] = e - t;
      }
      base += __popc(hm);
    }
    if (lane == 0) nuniq[i] = base;
    __syncwarp();
  }
}

__global__ void k_rw_compact(int n, int R, const int32_t* __restrict__ ucol, const int32_t* __restrict__ ucnt,
                             const int64_t* __restrict__ wrp, int32_t* __restrict__ wcol, int32_t* __restrict__ wcnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    const int64_t a = wrp[i], m = wrp[i + 1] - a;
    for (int64_t t = lane; t < m; t += 32) {
      wcol[a + t] = ucol[i * R + t];
      wcnt[a + t] = ucnt[i * R + t];
    }
  }
}

// pcond[e] = count(i, col[e]) / R on the symmetrised structure (0 when no
// walk from i ended at col[e]); warp per row, binary search in i's list.
__global__ void k_rw_pcond(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const int64_t* __restrict__ wrp, const int32_t* __restrict__ wcol,
                           const int32_t* __restrict__ wcnt, int R, float* __restrict__ pcond) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    const int64_t a = wrp[i], b = wrp[i + 1];
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += 32) {
      const int32_t j = col[e];
      int64_t lo = a, hi = b;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (wcol[mid] < j) lo = mid + 1; else hi = mid;
      }
      const int c = (lo < b && wcol[lo] == j) ? wcnt[lo] : 0;
      pcond[e] = (float)((double)c / (double)R);
    }
  }
}

int grid_cap(int64_t items, int per_block, int cap) {
  int64_t g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

}  // namespace

tsgne_status random_walk_affinities(int n, const int64_t* rp, const int32_t* col, int64_t nnz, const float* X, int d,
                                    int R, int L, uint64_t seed, DevBuf<int64_t>& rp_out, DevBuf<int32_t>& col_out,
                                    DevBuf<float>& P_out, int64_t* nnz_out, Sched* sched, cudaStream_t s) {
  int dev = 0, sms = 1;
  TS_CUDA(cudaGetDevice(&dev));
  TS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int wgrid = grid_cap(n, kRwWarps, sms * 64);
  DevBuf<double> d2, cw;
  TS_TRY(d2.alloc((size_t)nnz));
  TS_TRY(cw.alloc((size_t)nnz));
  if (nnz > 0) {
    k_rw_dist<<<wgrid, 32 * kRwWarps, 0, s>>>(n, rp, col, X, d, d2.get());
    k_rw_cumw<<<grid_cap(n, 256, 1 << 30), 256, 0, s>>>(n, rp, d2.get(), cw.get());
    TS_CUDA(cudaGetLastError());
  }
  d2.reset();
  const int64_t walks = (int64_t)n * R;
  DevBuf<int32_t> ends, ucol, ucnt, nuniq;
  TS_TRY(ends.alloc((size_t)walks));
  TS_TRY(ucol.alloc((size_t)walks));
  TS_TRY(ucnt.alloc((size_t)walks));
  TS_TRY(nuniq.alloc((size_t)n));
  k_rw_walks<<<grid_cap(walks, 256, 1 << 30), 256, 0, s>>>(n, rp, col, cw.get(), R, L,
                                                           seed ^ 0xD1B54A32D192ED03ull, ends.get());
  const size_t smem = (size_t)kRwWarps * 2 * R * sizeof(int32_t);
  TS_CUDA(cudaFuncSetAttribute(k_rw_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_rw_count<<<wgrid, 32 * kRwWarps, smem, s>>>(n, R, ends.get(), ucol.get(), ucnt.get(), nuniq.get());
  TS_CUDA(cudaGetLastError());
  ends.reset();
  cw.reset();
  DevBuf<int64_t> wrp, scr;
  TS_TRY(wrp.alloc((size_t)n + 1));
  TS_TRY(scr.alloc(scan_scratch_bytes(n) / sizeof(int64_t)));
  TS_TRY(scan_i32_to_i64(nuniq.get(), wrp.get(), n, scr.get(), s));
  int64_t m = 0;
  TS_CUDA(cudaMemcpyAsync(&m, wrp.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TS_CUDA(cudaStreamSynchronize(s));
  DevBuf<int32_t> wcol, wcnt;
  TS_TRY(wcol.alloc((size_t)m));
  TS_TRY(wcnt.alloc((size_t)m));
  k_rw_compact<<<wgrid, 32 * kRwWarps, 0, s>>>(n, R, ucol.get(), ucnt.get(), wrp.get(), wcol.get(), wcnt.get());
  TS_CUDA(cudaGetLastError());
  ucol.reset();
  ucnt.reset();
  // symmetrised structure of the walk pairs, then Eq. 3 over it
  DevBuf<int64_t> tslot;
  int64_t snnz = 0;
  TS_TRY(build_structure(n, wrp.get(), wcol.get(), m, rp_out, col_out, tslot, &snnz, sched, s));
  DevBuf<float> pcond;
  TS_TRY(pcond.alloc((size_t)snnz));
  TS_TRY(P_out.alloc((size_t)snnz));
  k_rw_pcond<<<wgrid, 32 * kRwWarps, 0, s>>>(n, rp_out.get(), col_out.get(), wrp.get(), wcol.get(), wcnt.get(), R,
                                             pcond.get());
  TS_CUDA(cudaGetLastError());
  TS_TRY(joint_affinities(snnz, pcond.get(), tslot.get(), P_out.get(), sched, s));
  *nnz_out = snnz;
  return TSGNE_OK;
}

}  // namespace tsgne
