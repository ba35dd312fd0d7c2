// ShortestPath graph embedding (Sec. 2.3, Eq. 8): for d target nodes,
//   X[i][t] = dist(v_i, target_t)  if that distance is <= l0,
//             l0 + 1               otherwise (or if no path exists),
// with l0 = sqrt(|E|) by default (distances are integers, so floor).
//
// All d breadth-first searches run together, level-synchronously: every node
// keeps two d-bit masks (targets that have reached it, and targets that
// reached it in the previous level).  Level L pulls, for each node, the OR of
// its neighbours' previous-level masks, keeps the bits it has not seen, and
// writes L for them.  One level is one pass over the adjacency (d/32 words
// per neighbour); nodes that every target has reached skip the pass.  The
// host stops at the first level that reaches no new (node, target) pair or at
// l0.  The result is exact integer work, independent of scheduling.
#include <cmath>

#include "tsgne_internal.cuh"

namespace tsgne {

namespace {

__global__ void k_sp_init(int n, int d, int words, const int32_t* __restrict__ targets, float far,
                          uint32_t* __restrict__ frontier, uint32_t* __restrict__ seen, float* __restrict__ X) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t total = (int64_t)n * d;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += stride) X[k] = far;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < (int64_t)n * words; k += stride) {
    frontier[k] = 0u;
    seen[k] = 0u;
  }
}

// targets may repeat; each sets its own bit
__global__ void k_sp_seed(int d, int words, const int32_t* __restrict__ targets, uint32_t* __restrict__ frontier,
                          uint32_t* __restrict__ seen, float* __restrict__ X) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < d; t += gridDim.x * blockDim.x) {
    const int64_t v = targets[t];
    atomicOr(&frontier[v * words + (t >> 5)], 1u << (t & 31));
    atomicOr(&seen[v * words + (t >> 5)], 1u << (t & 31));
    X[v * d + t] = 0.f;
  }
}

template <int WORDS>
__global__ void __launch_bounds__(256)
    k_sp_level(int n, int d, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
               const uint32_t* __restrict__ cur, uint32_t* __restrict__ next, uint32_t* __restrict__ seen,
               const uint32_t* __restrict__ full, float level, float* __restrict__ X, uint32_t* any) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    uint32_t s[WORDS], acc[WORDS];
    bool done = true;
#pragma unroll
    for (int w = 0; w < WORDS; ++w) {
      s[w] = seen[v * WORDS + w];
      acc[w] = 0u;
      done &= (s[w] == full[w]);
    }
    if (!done) {
      for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
        const int64_t u = col[e];
#pragma unroll
        for (int w = 0; w < WORDS; ++w) acc[w] |= cur[u * WORDS + w];
      }
    }
    bool any_new = false;
#pragma unroll
    for (int w = 0; w < WORDS; ++w) {
      uint32_t nw = done ? 0u : (acc[w] & ~s[w]);
      next[v * WORDS + w] = nw;
      if (nw) {
        any_new = true;
        seen[v * WORDS + w] = s[w] | nw;
        while (nw) {
          const int b = __ffs(nw) - 1;
          nw &= nw - 1u;
          X[v * d + w * 32 + b] = level;
        }
      }
    }
    if (any_new) atomicOr(any, 1u);
  }
}

template <int WORDS>
tsgne_status run_levels(int n, int d, const int64_t* rp, const int32_t* col, uint32_t* f0, uint32_t* f1,
                        uint32_t* seen, const uint32_t* full, int l0, float* X, uint32_t* any, int grid,
                        cudaStream_t s) {
  uint32_t* cur = f0;
  uint32_t* nxt = f1;
  for (int L = 1; L <= l0; ++L) {
    TS_CUDA(cudaMemsetAsync(any, 0, sizeof(uint32_t), s));
    k_sp_level<WORDS><<<grid, 256, 0, s>>>(n, d, rp, col, cur, nxt, seen, full, (float)L, X, any);
    TS_CUDA(cudaGetLastError());
    uint32_t h = 0;
    TS_CUDA(cudaMemcpyAsync(&h, any, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaStreamSynchronize(s));
    if (!h) break;
    uint32_t* t = cur;
    cur = nxt;
    nxt = t;
  }
  return TSGNE_OK;
}

}  // namespace

tsgne_status shortest_path_embedding(int n, const int64_t* rp, const int32_t* col, int64_t nnz,
                                     const int32_t* targets, int d, int l0, float* X, cudaStream_t s) {
  if (l0 <= 0) l0 = (int)std::floor(std::sqrt((double)(nnz / 2)));
  if (l0 < 0) l0 = 0;
  const int words = (d + 31) / 32;
  int W = 1;
  while (W < words) W <<= 1;
  if (W > 32) {
    last_msg() = "ShortestPath embedding supports at most 1024 targets";
    return TSGNE_ERR_INVALID_ARG;
  }
  int dev = 0, sms = 1;
  TS_CUDA(cudaGetDevice(&dev));
  TS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DevBuf<uint32_t> f0, f1, seen, full, any;
  TS_TRY(f0.alloc((size_t)n * W));
  TS_TRY(f1.alloc((size_t)n * W));
  TS_TRY(seen.alloc((size_t)n * W));
  TS_TRY(full.alloc((size_t)W));
  TS_TRY(any.alloc(1));
  uint32_t hfull[32];
  for (int w = 0; w < W; ++w) {
    const int bits = d - 32 * w;
    hfull[w] = bits >= 32 ? 0xffffffffu : (bits <= 0 ? 0u : ((1u << bits) - 1u));
  }
  TS_CUDA(cudaMemcpyAsync(full.get(), hfull, sizeof(uint32_t) * W, cudaMemcpyHostToDevice, s));
  const int grid = sms * 8;
  k_sp_init<<<grid, 256, 0, s>>>(n, d, W, targets, (float)(l0 + 1), f0.get(), seen.get(), X);
  k_sp_seed<<<(d + 255) / 256, 256, 0, s>>>(d, W, targets, f0.get(), seen.get(), X);
  TS_CUDA(cudaGetLastError());
  switch (W) {
    case 1: return run_levels<1>(n, d, rp, col, f0.get(), f1.get(), seen.get(), full.get(), l0, X, any.get(), grid, s);
    case 2: return run_levels<2>(n, d, rp, col, f0.get(), f1.get(), seen.get(), full.get(), l0, X, any.get(), grid, s);
    case 4: return run_levels<4>(n, d, rp, col, f0.get(), f1.get(), seen.get(), full.get(), l0, X, any.get(), grid, s);
    case 8: return run_levels<8>(n, d, rp, col, f0.get(), f1.get(), seen.get(), full.get(), l0, X, any.get(), grid, s);
    case 16: return run_levels<16>(n, d, rp, col, f0.get(), f1.get(), seen.get(), full.get(), l0, X, any.get(), grid, s);
    default: return run_levels<32>(n, d, rp, col, f0.get(), f1.get(), seen.get(), full.get(), l0, X, any.get(), grid, s);
  }
}

}  // namespace tsgne

extern "C" tsgne_status tsgne_shortest_path_embedding(int32_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                                      const int32_t* targets, int32_t d, int32_t l0, float* X_out,
                                                      int32_t ptr_kind, void* cuda_stream) {
  using namespace tsgne;
  last_msg().clear();
  if (n < 1 || d < 1 || d > 1024 || !row_ptr || !targets || !X_out ||
      !(ptr_kind == TSGNE_PTR_HOST || ptr_kind == TSGNE_PTR_DEVICE)) {
    last_msg() = "need n >= 1, 1 <= d <= 1024, non-NULL row_ptr, targets and X_out, and a valid ptr_kind";
    return TSGNE_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const cudaMemcpyKind kin = ptr_kind == TSGNE_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  int64_t first = 0, m = 0;
  if (ptr_kind == TSGNE_PTR_HOST) {
    first = row_ptr[0];
    m = row_ptr[n];
    for (int t = 0; t < d; ++t)
      if (targets[t] < 0 || targets[t] >= n) return TSGNE_ERR_INVALID_ARG;
  } else {
    TS_CUDA(cudaMemcpy(&first, row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost));
    TS_CUDA(cudaMemcpy(&m, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost));
    int32_t* ht = new int32_t[d];
    cudaError_t e = cudaMemcpy(ht, targets, sizeof(int32_t) * d, cudaMemcpyDeviceToHost);
    bool bad = false;
    for (int t = 0; t < d && e == cudaSuccess; ++t) bad |= (ht[t] < 0 || ht[t] >= n);
    delete[] ht;
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy", __FILE__, __LINE__);
    if (bad) return TSGNE_ERR_INVALID_ARG;
  }
  if (first != 0 || m < 0) return TSGNE_ERR_BAD_CSR;
  if (m > 0 && !col_idx) return TSGNE_ERR_INVALID_ARG;
  DevBuf<int64_t> rp_in, rp, tslot;
  DevBuf<int32_t> col_in, col, tg;
  DevBuf<float> Xd;
  TS_TRY(rp_in.alloc((size_t)n + 1));
  TS_TRY(col_in.alloc((size_t)m));
  TS_TRY(tg.alloc((size_t)d));
  TS_CUDA(cudaMemcpyAsync(rp_in.get(), row_ptr, sizeof(int64_t) * ((size_t)n + 1), kin, s));
  if (m > 0) TS_CUDA(cudaMemcpyAsync(col_in.get(), col_idx, sizeof(int32_t) * (size_t)m, kin, s));
  TS_CUDA(cudaMemcpyAsync(tg.get(), targets, sizeof(int32_t) * d, kin, s));
  int64_t nnz = 0;
  TS_TRY(build_structure(n, rp_in.get(), col_in.get(), m, rp, col, tslot, &nnz, nullptr, s));
  float* Xo = X_out;
  if (ptr_kind == TSGNE_PTR_HOST) {
    TS_TRY(Xd.alloc((size_t)n * d));
    Xo = Xd.get();
  }
  TS_TRY(shortest_path_embedding(n, rp.get(), col.get(), nnz, tg.get(), d, l0, Xo, s));
  if (ptr_kind == TSGNE_PTR_HOST)
    TS_CUDA(cudaMemcpyAsync(X_out, Xo, sizeof(float) * (size_t)n * d, cudaMemcpyDeviceToHost, s));
  TS_CUDA(cudaStreamSynchronize(s));
  return TSGNE_OK;
}
