// Tree-code approximation of the repulsive sums and of Z (an extension: the
// paper sums Eq. 4 exactly, at O(|V|^2) cost, Sec. 2.1 "Time complexity").
//
// Definition (the oracle restates the same steps in plain C):
//  1. bounding square of the layout: lo = (min x, min y), side = the longer
//     extent (floored at 1e-30), scale = 65536 / side;
//  2. cell of a point per axis = trunc((v - lo) * scale) clamped to
//     [0, 65535]; key = Morton interleave (x in the even bits);
//  3. points sorted by (key, index); sorted position k has the augmented key
//     (key << 32) | k;
//  4. the binary radix tree of the augmented keys (a node over positions
//     [f, l] splits at the highest bit in which keys f and l differ);
//  5. node summaries in FP32: coordinate sums (left + right), box, centre =
//     sums / count, r2 = (longer box side)^2;
//  6. groups of 32 consecutive sorted positions, with their bounding box;
//  7. per group, a depth-first walk from the root, left child first: a leaf
//     is an exact interaction; a node whose r2 < theta^2 d2 (d = distance
//     from its centre to the group box) is one interaction of weight count
//     at its centre; an opened node of at most kTreeBucket points is
//     summed exactly over its points; other nodes are opened.
// Every decision (keys, tree shape, acceptance) is taken with IEEE FP32
// operations written as _rn intrinsics, so no FMA contraction changes it and
// the CPU reference takes the same decisions.
//
// GPU mapping.  Keys: one thread per point.  Sort: LSD radix sort, 8 bits per
// pass, stable: a warp owns a chunk of 512 keys; per-(digit, chunk) counts
// are scanned digit-major, and the scatter ranks equal digits within a round
// of 32 keys with __match_any_sync, so equal keys keep their input order.
// The last pass also gathers the layout into sorted order.  Tree: one thread
// per internal node finds its range and split from the sorted keys alone
// (binary search over the common-prefix length); summaries bottom-up, one
// thread per leaf climbing until it is the first of two children to arrive.
// Walk: one warp per group, lane = point; the stack of node ids is in shared
// memory and every lane takes the same branch, so the traversal is free of
// divergence and every node load is a broadcast.  Z: FP32 partial sums
// flushed into FP64 every 64 interactions, a fixed xor butterfly per warp,
// one FP64 partial per group, and the group partials added in group order by
// the last CTA -- bit-reproducible from run to run.
#include <cmath>

#include "f32x2.cuh"
#include "reduce.cuh"
#include "tsgne_internal.cuh"

namespace tsgne {

namespace {

constexpr int kRadixItems = 16;                // keys per lane of a warp chunk
constexpr int kRadixChunk = 32 * kRadixItems;  // keys per warp chunk
constexpr int kRadixWarps = 8;
constexpr int kRadixBins = 256;
constexpr int kWalkWarps = 8;
constexpr int kStack = 72;  // a root-to-leaf path has at most 64 splits (one per key bit)
constexpr int kZFlush = 64;

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------- 1. bounding box

__global__ void __launch_bounds__(256) k_tree_box(const float2* __restrict__ Y, int n, float4* __restrict__ part,
                                                  TreeState* st) {
  __shared__ float4 ws[8];
  float lx = INFINITY, ly = INFINITY, hx = -INFINITY, hy = -INFINITY;
  for (int i = blockIdx.x * 256 + threadIdx.x; i < n; i += gridDim.x * 256) {
    const float2 p = Y[i];
    lx = fminf(lx, p.x);
    ly = fminf(ly, p.y);
    hx = fmaxf(hx, p.x);
    hy = fmaxf(hy, p.y);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  lx = warp_min(lx);
  ly = warp_min(ly);
  hx = warp_max(hx);
  hy = warp_max(hy);
  if (lane == 0) ws[w] = make_float4(lx, ly, hx, hy);
  __syncthreads();
  if (threadIdx.x == 0) {
    float4 b = ws[0];
    for (int k = 1; k < 8; ++k) {
      b.x = fminf(b.x, ws[k].x);
      b.y = fminf(b.y, ws[k].y);
      b.z = fmaxf(b.z, ws[k].z);
      b.w = fmaxf(b.w, ws[k].w);
    }
    part[blockIdx.x] = b;
  }
  if (arrive_last(&st->box_done)) {
    if (threadIdx.x == 0) {
      float4 b = __ldcg(part);
      for (unsigned k = 1; k < gridDim.x; ++k) {
        const float4 q = __ldcg(part + k);
        b.x = fminf(b.x, q.x);
        b.y = fminf(b.y, q.y);
        b.z = fmaxf(b.z, q.z);
        b.w = fmaxf(b.w, q.w);
      }
      const float side = fmaxf(fmaxf(__fsub_rn(b.z, b.x), __fsub_rn(b.w, b.y)), 1e-30f);
      st->lo_x = b.x;
      st->lo_y = b.y;
      st->scale = __fdiv_rn(65536.0f, side);
    }
  }
}

// ---------------------------------------------------------------- 2. keys

__device__ __forceinline__ uint32_t spread16(uint32_t v) {
  v &= 0xffffu;
  v = (v | (v << 8)) & 0x00ff00ffu;
  v = (v | (v << 4)) & 0x0f0f0f0fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

__device__ __forceinline__ uint32_t cell16(float v, float lo, float scale) {
  const float c = __fmul_rn(__fsub_rn(v, lo), scale);
  if (!(c >= 0.0f)) return 0u;
  if (c >= 65535.0f) return 65535u;
  return (uint32_t)c;
}

__global__ void k_tree_keys(const float2* __restrict__ Y, int n, const TreeState* __restrict__ st,
                            uint32_t* __restrict__ keys, int32_t* __restrict__ vals) {
  const float lx = st->lo_x, ly = st->lo_y, sc = st->scale;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 p = Y[i];
    keys[i] = spread16(cell16(p.x, lx, sc)) | (spread16(cell16(p.y, ly, sc)) << 1);
    vals[i] = i;
  }
}

// ---------------------------------------------------------------- 3. sort

__global__ void __launch_bounds__(32 * kRadixWarps)
    k_radix_hist(const uint32_t* __restrict__ keys, int n, int shift, int nchunks, int32_t* __restrict__ counts) {
  __shared__ uint32_t h[kRadixWarps][kRadixBins];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * kRadixWarps + w;
  for (int d = lane; d < kRadixBins; d += 32) h[w][d] = 0u;
  __syncwarp();
  if (c >= nchunks) return;
  const int64_t base = (int64_t)c * kRadixChunk + lane;
  uint32_t kk[kRadixItems];
#pragma unroll
  for (int r = 0; r < kRadixItems; ++r) {
    const int64_t k = base + 32 * r;
    kk[r] = k < n ? keys[k] : 0u;
  }
#pragma unroll
  for (int r = 0; r < kRadixItems; ++r)
    if (base + 32 * r < n) atomicAdd(&h[w][(kk[r] >> shift) & 255u], 1u);
  __syncwarp();
  for (int d = lane; d < kRadixBins; d += 32) counts[(int64_t)d * nchunks + c] = (int32_t)h[w][d];
}

// Stable scatter of one pass.  offs = exclusive scan of counts (digit-major).
// With Y != NULL the layout is gathered into sorted order (ys[pos] = Y[val]).
__global__ void __launch_bounds__(32 * kRadixWarps)
    k_radix_scatter(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin, int n, int shift, int nchunks,
                    const int64_t* __restrict__ offs, uint32_t* __restrict__ kout, int32_t* __restrict__ vout,
                    const float2* __restrict__ Y, float2* __restrict__ ys) {
  __shared__ int32_t base[kRadixWarps][kRadixBins];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * kRadixWarps + w;
  if (c >= nchunks) return;
  for (int d = lane; d < kRadixBins; d += 32) base[w][d] = (int32_t)offs[(int64_t)d * nchunks + c];
  __syncwarp();
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t k0 = (int64_t)c * kRadixChunk + lane;
  for (int r = 0; r < kRadixItems; ++r) {
    const int64_t k = k0 + 32 * r;
    const bool valid = k < n;
    const uint32_t key = valid ? kin[k] : 0u;
    const int32_t val = valid ? vin[k] : 0;
    const uint32_t d = valid ? (key >> shift) & 255u : 256u + (uint32_t)lane;  // invalid lanes match only themselves
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    int pos = 0;
    if (valid) pos = base[w][d] + rank;
    __syncwarp();
    if (valid && rank == 0) base[w][d] += __popc(peers);
    __syncwarp();
    if (valid) {
      kout[pos] = key;
      vout[pos] = val;
      if (ys) ys[pos] = Y[val];
    }
  }
}

// ---------------------------------------------------------------- 4. tree

// Common-prefix length of the augmented keys of sorted positions i and j
// (-1 when j is outside [0, n)).
__device__ __forceinline__ int tree_delta(const uint32_t* __restrict__ keys, int n, int i, int64_t j) {
  if (j < 0 || j >= n) return -1;
  const uint32_t a = keys[i], b = keys[j];
  return a != b ? __clz(a ^ b) : 32 + __clz((uint32_t)i ^ (uint32_t)j);
}

// Internal node i (0 <= i < n - 1; node 0 is the root).  Children: >= 0 an
// internal node, < 0 the leaf at sorted position ~c.  parent: internal nodes
// at [0, n - 1), leaf k at n - 1 + k; the root's parent is -1.
__global__ void k_tree_build(const uint32_t* __restrict__ keys, int n, int4* __restrict__ nodeB,
                             int32_t* __restrict__ parent) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const int d = tree_delta(keys, n, i, (int64_t)i + 1) > tree_delta(keys, n, i, (int64_t)i - 1) ? 1 : -1;
  const int dmin = tree_delta(keys, n, i, (int64_t)i - d);
  int64_t lmax = 2;
  while (tree_delta(keys, n, i, (int64_t)i + lmax * d) > dmin) lmax <<= 1;
  int64_t l = 0;
  for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
    if (tree_delta(keys, n, i, (int64_t)i + (l + t) * d) > dmin) l += t;
  const int64_t j = (int64_t)i + l * d;
  const int dn = tree_delta(keys, n, i, j);
  int64_t s = 0;
  for (int64_t div = 2;; div <<= 1) {
    const int64_t t = (l + div - 1) / div;
    if (tree_delta(keys, n, i, (int64_t)i + (s + t) * d) > dn) s += t;
    if (t <= 1) break;
  }
  const int64_t gamma = (int64_t)i + s * d + (d < 0 ? -1 : 0);
  const int first = (int)(j < i ? j : i), last = (int)(j < i ? i : j);
  const int left = first == gamma ? ~(int)gamma : (int)gamma;
  const int right = last == gamma + 1 ? ~(int)(gamma + 1) : (int)(gamma + 1);
  nodeB[i] = make_int4(left, right, first, last);
  parent[left >= 0 ? left : n - 1 + ~left] = i;
  parent[right >= 0 ? right : n - 1 + ~right] = i;
  if (i == 0) parent[0] = -1;
}

__device__ __forceinline__ void child_summary(int c, const float2* __restrict__ ys, const float4* box,
                                              const float2* sum, float4& b, float2& s) {
  if (c < 0) {
    const float2 q = ys[~c];
    b = make_float4(q.x, q.y, q.x, q.y);
    s = q;
  } else {
    b = __ldcg(box + c);
    s = __ldcg(sum + c);
  }
}

// Summaries bottom-up: the second child to arrive at a node computes it
// (left + right, whichever thread that is) and climbs on; flags are reset
// on the way so the next pass starts from zero.
__global__ void k_tree_up(int n, const int4* __restrict__ nodeB, const int32_t* __restrict__ parent,
                          const float2* __restrict__ ys, uint32_t* flags, float4* box, float2* sum,
                          float4* __restrict__ nodeA) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int p = parent[n - 1 + k];
  while (p >= 0) {
    __threadfence();
    if (atomicAdd(&flags[p], 1u) == 0u) return;
    __threadfence();
    flags[p] = 0u;
    const int4 b = nodeB[p];
    float4 bl, br;
    float2 sl, sr;
    child_summary(b.x, ys, box, sum, bl, sl);
    child_summary(b.y, ys, box, sum, br, sr);
    const float2 sp = make_float2(__fadd_rn(sl.x, sr.x), __fadd_rn(sl.y, sr.y));
    const float4 bp = make_float4(fminf(bl.x, br.x), fminf(bl.y, br.y), fmaxf(bl.z, br.z), fmaxf(bl.w, br.w));
    box[p] = bp;
    sum[p] = sp;
    const float cnt = (float)(b.w - b.z + 1);
    const float r = fmaxf(__fsub_rn(bp.z, bp.x), __fsub_rn(bp.w, bp.y));
    nodeA[p] = make_float4(__fdiv_rn(sp.x, cnt), __fdiv_rn(sp.y, cnt), __fmul_rn(r, r), cnt);
    p = parent[p];
  }
}

// ---------------------------------------------------------------- 7. walk

// One interaction of weight c at q (c = 0 for the lane's own point and for
// lanes past the end of the layout).
__device__ __forceinline__ void interact(float2 p, float qx, float qy, float c, float& fx, float& fy, float& zf) {
  const float dx = p.x - qx, dy = p.y - qy;
  const float w = rcp_approx(fmaf(dy, dy, fmaf(dx, dx, 1.0f)));
  const float cw = c * w;
  zf += cw;
  const float cw2 = cw * w;
  fx = fmaf(cw2, dx, fx);
  fy = fmaf(cw2, dy, fy);
}

__global__ void __launch_bounds__(32 * kWalkWarps)
    k_tree_walk(int n, const float2* __restrict__ ys, const int32_t* __restrict__ perm,
                const float4* __restrict__ nodeA, const int4* __restrict__ nodeB, float theta2,
                float2* __restrict__ frep, double* __restrict__ zgroup, int ngroups, Sched* sched, TreeState* st,
                int advance, float ee, int ee_iters, float mom0, float mom1) {
  __shared__ int stk[kWalkWarps][kStack];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.x * kWalkWarps + w;
  if (g < ngroups) {
    const int k0 = 32 * g, k = k0 + lane;
    const bool act = k < n;
    const float2 p = ys[act ? k : k0];
    const float gx0 = warp_min(p.x), gy0 = warp_min(p.y), gx1 = warp_max(p.x), gy1 = warp_max(p.y);
    const float self = act ? 1.0f : 0.0f;
    float fx = 0.f, fy = 0.f, zf = 0.f;
    double zd = 0.0;
    int nacc = 0;
    bool overflow = false;
    if (lane == 0) stk[w][0] = n > 1 ? 0 : ~0;
    int sp = 1;
    __syncwarp();
    while (sp > 0) {
      const int v = stk[w][--sp];
      __syncwarp();
      if (v < 0) {
        const int j = ~v;
        const float2 q = ys[j];
        interact(p, q.x, q.y, j == k ? 0.f : self, fx, fy, zf);
        ++nacc;
      } else {
        const float4 A = nodeA[v];
        const float dx = fmaxf(fmaxf(__fsub_rn(gx0, A.x), __fsub_rn(A.x, gx1)), 0.0f);
        const float dy = fmaxf(fmaxf(__fsub_rn(gy0, A.y), __fsub_rn(A.y, gy1)), 0.0f);
        const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        if (A.z < __fmul_rn(theta2, d2)) {
          interact(p, A.x, A.y, act ? A.w : 0.f, fx, fy, zf);
          ++nacc;
        } else {
          const int4 B = nodeB[v];
          if (B.w - B.z + 1 <= kTreeBucket) {
            for (int j = B.z; j <= B.w; ++j) {
              const float2 q = ys[j];
              interact(p, q.x, q.y, j == k ? 0.f : self, fx, fy, zf);
            }
            nacc += B.w - B.z + 1;
          } else if (sp + 2 <= kStack) {
            if (lane == 0) {
              stk[w][sp] = B.y;
              stk[w][sp + 1] = B.x;
            }
            sp += 2;
            __syncwarp();
          } else {
            overflow = true;  // cannot happen for a radix tree of 64-bit keys; recorded, never indexed past
          }
        }
      }
      if (nacc >= kZFlush) {
        zd += (double)zf;
        zf = 0.f;
        nacc = 0;
      }
    }
    zd += (double)zf;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zd += __shfl_xor_sync(0xffffffffu, zd, o);
    if (lane == 0) {
      zgroup[g] = zd;
      if (overflow) atomicOr(&sched->flags, kFlagTreeOverflow);
    }
    if (act) frep[perm[k]] = make_float2(fx, fy);
  }
  if (arrive_last(&st->walk_done)) {
    const double total = sum_partials(zgroup, ngroups);
    if (threadIdx.x == 0) {
      sched->Z = total;
      const int t = sched->t;
      sched->alpha = t < ee_iters ? ee : 1.0f;
      sched->mu = t < ee_iters ? mom0 : mom1;
      if (advance) sched->t = t + 1;
    }
  }
}

int grid_for(int64_t items, int per_block, int cap) {
  int64_t g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

tsgne_status TreeBufs::alloc(int n_points, int sm_count, cudaStream_t s) {
  n = n_points;
  nchunks = (n + kRadixChunk - 1) / kRadixChunk;
  ngroups = (n + 31) / 32;
  box_blocks = grid_for(n, 256, 2 * sm_count);
  const size_t nn = (size_t)(n > 1 ? n - 1 : 1);
  TS_TRY(keys[0].alloc((size_t)n));
  TS_TRY(keys[1].alloc((size_t)n));
  TS_TRY(vals[0].alloc((size_t)n));
  TS_TRY(vals[1].alloc((size_t)n));
  TS_TRY(ys.alloc((size_t)n));
  TS_TRY(counts.alloc((size_t)kRadixBins * nchunks));
  TS_TRY(offs.alloc((size_t)kRadixBins * nchunks + 1));
  TS_TRY(scan_scr.alloc(scan_scratch_bytes((int64_t)kRadixBins * nchunks) / sizeof(int64_t)));
  TS_TRY(nodeA.alloc(nn));
  TS_TRY(nodeB.alloc(nn));
  TS_TRY(box.alloc(nn));
  TS_TRY(sum.alloc(nn));
  TS_TRY(flags.alloc(nn));
  TS_TRY(parent.alloc(2 * (size_t)n));
  TS_TRY(boxpart.alloc((size_t)box_blocks));
  TS_TRY(zgroup.alloc((size_t)ngroups));
  TS_TRY(state.alloc(1));
  TS_CUDA(cudaMemsetAsync(flags.get(), 0, sizeof(uint32_t) * nn, s));
  TS_CUDA(cudaMemsetAsync(state.get(), 0, sizeof(TreeState), s));
  return TSGNE_OK;
}

tsgne_status launch_tree_build(TreeBufs& tb, const float2* Y, cudaStream_t s) {
  const int n = tb.n;
  k_tree_box<<<tb.box_blocks, 256, 0, s>>>(Y, n, tb.boxpart.get(), tb.state.get());
  k_tree_keys<<<grid_for(n, 256, 1 << 20), 256, 0, s>>>(Y, n, tb.state.get(), tb.keys[0].get(), tb.vals[0].get());
  TS_CUDA(cudaGetLastError());
  const int rblocks = (tb.nchunks + kRadixWarps - 1) / kRadixWarps;
  const int64_t ncount = (int64_t)kRadixBins * tb.nchunks;
  for (int pass = 0; pass < 4; ++pass) {
    const int in = pass & 1, out = in ^ 1;
    k_radix_hist<<<rblocks, 32 * kRadixWarps, 0, s>>>(tb.keys[in].get(), n, 8 * pass, tb.nchunks, tb.counts.get());
    TS_CUDA(cudaGetLastError());
    TS_TRY(scan_i32_to_i64(tb.counts.get(), tb.offs.get(), ncount, tb.scan_scr.get(), s));
    const bool last = pass == 3;
    k_radix_scatter<<<rblocks, 32 * kRadixWarps, 0, s>>>(tb.keys[in].get(), tb.vals[in].get(), n, 8 * pass,
                                                         tb.nchunks, tb.offs.get(), tb.keys[out].get(),
                                                         tb.vals[out].get(), last ? Y : nullptr,
                                                         last ? tb.ys.get() : nullptr);
    TS_CUDA(cudaGetLastError());
  }
  // four passes: sorted keys / permutation are back in slot 0
  if (n > 1) {
    k_tree_build<<<grid_for(n - 1, 256, 1 << 30), 256, 0, s>>>(tb.keys[0].get(), n, tb.nodeB.get(),
                                                               tb.parent.get());
    k_tree_up<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(n, tb.nodeB.get(), tb.parent.get(), tb.ys.get(),
                                                       tb.flags.get(), tb.box.get(), tb.sum.get(), tb.nodeA.get());
    TS_CUDA(cudaGetLastError());
  }
  return TSGNE_OK;
}

tsgne_status launch_tree_walk(TreeBufs& tb, float theta, float2* frep, Sched* sched, int advance, float ee,
                              int ee_iters, float mom0, float mom1, cudaStream_t s) {
  const float theta2 = theta * theta;
  const int blocks = (tb.ngroups + kWalkWarps - 1) / kWalkWarps;
  k_tree_walk<<<blocks, 32 * kWalkWarps, 0, s>>>(tb.n, tb.ys.get(), tb.vals[0].get(), tb.nodeA.get(),
                                                 tb.nodeB.get(), theta2, frep, tb.zgroup.get(), tb.ngroups, sched,
                                                 tb.state.get(), advance, ee, ee_iters, mom0, mom1);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

}  // namespace tsgne
