// Tree-code approximation of the repulsive sums and of Z (an extension: the
// paper sums Eq. 4 exactly, at O(|V|^2) cost, Sec. 2.1 "Time complexity").
//
// Definition (the oracle restates the same steps in plain C):
//  1. bounding square of the layout (FP32): lo = (min x, min y), side = the
//     longer extent (floored at 1e-30); scale = 2^32 / side in FP64;
//  2. cell of a point per axis = trunc((v - lo) * scale) in FP64, clamped
//     to [0, 2^32 - 1]; key = 64-bit Morton interleave (x in the even bits).
//     32 bits per axis keep the bulk resolved when a few outliers stretch
//     the square to thousands of times its size;
//  3. points sorted by (key, index); sorted position k has the 96-bit
//     augmented key (key, k);
//  4. the binary radix tree of the augmented keys (a node over positions
//     [f, l] splits at the highest bit in which keys f and l differ);
//  5. node summaries in FP32: coordinate sums (left + right), box, centre =
//     sums / count, r2 = (longer box side)^2;
//  6. groups: the maximal subtrees of at most 32 points (nodes of <= 32
//     points whose parent has more), in sorted order -- compact Morton
//     cells, so no group box straddles a jump of the curve;
//  7. per group, a depth-first walk from the root, left child first: a leaf
//     is an exact interaction; a node whose r2 < theta^2 d2 (d = distance
//     from its centre to the group box) is one interaction of weight count
//     at its centre; an opened node of at most kTreeBucket points is
//     summed exactly over its points; other nodes are opened.
// Every decision (keys, tree shape, acceptance) is taken with IEEE FP32 /
// FP64 operations written as _rn intrinsics, so no FMA contraction changes
// it and the CPU reference takes the same decisions.
//
// GPU mapping.  Keys: one thread per point, which also counts the digits of
// all eight sort passes.  Sort: LSD radix sort, 8 stable passes of 8 bits,
// one launch each: a CTA ranks a tile of 2048 keys (__match_any_sync within
// warps, offsets across warps) and takes the tile's global offsets from the
// tiles before it by a decoupled look-back (a bounded wait).  The last pass
// also gathers the layout into sorted order.  Tree, summaries and group
// starts: one bottom-up pass, one thread per leaf climbing (each node's
// parent follows from two neighbouring key prefixes) until it is the first of
// two children to arrive; a scan numbers the groups in sorted order.  Walk: a persistent grid takes groups from a queue, one warp per
// group, lane = point; per round the lanes decide up to 32 stack entries at
// once and then all apply the round's accepted nodes and exact points, so
// the dependent node loads along the tree are issued 32 at a time.  Z: FP32
// partial sums flushed into FP64 every round, a fixed xor butterfly per warp,
// one FP64 partial per group, and the group partials added in group order by
// the last CTA -- bit-reproducible from run to run.
#include <cmath>

#include "f32x2.cuh"
#include "reduce.cuh"
#include "tsgne_internal.cuh"

namespace tsgne {

namespace {

constexpr int kRadixPasses = 8;  // 8-bit digits of the 64-bit keys
constexpr int kRadixBins = 256;
constexpr int kSortWarps = 8;
constexpr int kSortThreads = 32 * kSortWarps;        // one thread per digit in the look-back
constexpr int kSortItems = 8;                        // keys per lane
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per tile (per CTA)
static_assert(kSortThreads == kRadixBins, "the look-back maps one thread to one digit");
constexpr int kWalkWarps = 8;

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

// Min / max over a 256-thread CTA (exact in any order); valid in thread 0.
__device__ __forceinline__ float4 block_box(float lx, float ly, float hx, float hy, float4* ws) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  lx = warp_min(lx);
  ly = warp_min(ly);
  hx = warp_max(hx);
  hy = warp_max(hy);
  if (lane == 0) ws[w] = make_float4(lx, ly, hx, hy);
  __syncthreads();
  float4 b = ws[0];
  if (threadIdx.x == 0)
    for (int k = 1; k < 8; ++k) {
      b.x = fminf(b.x, ws[k].x);
      b.y = fminf(b.y, ws[k].y);
      b.z = fmaxf(b.z, ws[k].z);
      b.w = fmaxf(b.w, ws[k].w);
    }
  __syncthreads();
  return b;
}

// Also clears the sort's digit counts, tile counters and tile status words
// (zero[0..nzero)), the group starts (is_start[0..n)) and the stall mark for
// the build that follows.
__global__ void __launch_bounds__(256) k_tree_box(const float2* __restrict__ Y, int n, float4* __restrict__ part,
                                                  TreeState* st, uint32_t* __restrict__ zero, int64_t nzero,
                                                  int32_t* __restrict__ is_start) {
  __shared__ float4 ws[8];
  for (int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x; k < nzero; k += (int64_t)gridDim.x * 256) zero[k] = 0u;
  for (int k = blockIdx.x * 256 + threadIdx.x; k < n; k += gridDim.x * 256) is_start[k] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) st->sort_stall = 0u;
  float lx = INFINITY, ly = INFINITY, hx = -INFINITY, hy = -INFINITY;
  for (int i = blockIdx.x * 256 + threadIdx.x; i < n; i += gridDim.x * 256) {
    const float2 p = Y[i];
    lx = fminf(lx, p.x);
    ly = fminf(ly, p.y);
    hx = fmaxf(hx, p.x);
    hy = fmaxf(hy, p.y);
  }
  float4 b = block_box(lx, ly, hx, hy, ws);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
  if (arrive_last(&st->box_done)) {
    lx = ly = INFINITY;
    hx = hy = -INFINITY;
    for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
      const float4 q = __ldcg(part + k);
      lx = fminf(lx, q.x);
      ly = fminf(ly, q.y);
      hx = fmaxf(hx, q.z);
      hy = fmaxf(hy, q.w);
    }
    b = block_box(lx, ly, hx, hy, ws);
    if (threadIdx.x == 0) {
      const float side = fmaxf(fmaxf(__fsub_rn(b.z, b.x), __fsub_rn(b.w, b.y)), 1e-30f);
      st->lo_x = b.x;
      st->lo_y = b.y;
      st->scale = __ddiv_rn(4294967296.0, (double)side);
    }
  }
}

// ---------------------------------------------------------------- 2. keys

__device__ __forceinline__ uint64_t spread32(uint32_t v) {
  uint64_t x = v;
  x = (x | (x << 16)) & 0x0000ffff0000ffffull;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

__device__ __forceinline__ uint32_t cell32(float v, double lo, double scale) {
  const double c = __dmul_rn(__dsub_rn((double)v, lo), scale);
  if (!(c >= 0.0)) return 0u;
  if (c >= 4294967295.0) return 0xffffffffu;
  return (uint32_t)c;
}

// Keys and the identity permutation, plus the counts of every 8-bit digit
// of every key for all eight passes at once (ghist[pass][digit], zeroed by
// k_tree_box): one read of the layout serves the whole sort.
__global__ void __launch_bounds__(256) k_tree_keys(const float2* __restrict__ Y, int n,
                                                   const TreeState* __restrict__ st, uint64_t* __restrict__ keys,
                                                   int32_t* __restrict__ vals, uint32_t* __restrict__ ghist) {
  __shared__ uint32_t h[kRadixPasses * kRadixBins];
  for (int k = threadIdx.x; k < kRadixPasses * kRadixBins; k += 256) h[k] = 0u;
  __syncthreads();
  const double lx = st->lo_x, ly = st->lo_y, sc = st->scale;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 p = Y[i];
    const uint64_t key = spread32(cell32(p.x, lx, sc)) | (spread32(cell32(p.y, ly, sc)) << 1);
    keys[i] = key;
    vals[i] = i;
#pragma unroll
    for (int q = 0; q < kRadixPasses; ++q) atomicAdd(&h[q * kRadixBins + (int)((key >> (8 * q)) & 255u)], 1u);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kRadixPasses * kRadixBins; k += 256)
    if (h[k]) atomicAdd(ghist + k, h[k]);
}

// ---------------------------------------------------------------- 3. sort

// One stable pass of the LSD radix sort, digit (key >> 8 pass) & 255, as a
// single launch (one-sweep: the digit counts of all passes come from
// k_tree_keys; the offsets of a tile come from its predecessors through a
// decoupled look-back, Merrill & Garland's single-pass prefix scan, instead
// of a separate count / scan / scatter per pass).
//
// A CTA takes tiles in launch order from a counter (ctl[pass]), so it only
// ever waits on tiles that running CTAs own.  Tile t covers keys
// [t T, t T + T), T = kSortTile; warp w holds keys w 256 + 32 r + lane,
// r < 8, so (w, r, lane) order is input order.
//  1. ranks within the warp: per round of 32 keys __match_any_sync groups
//     equal digits; rank = running count of the digit in the warp + the
//     number of lower lanes with the same digit;
//  2. per digit d (thread d): the warps' exclusive offsets and the tile's
//     count c_d, published at once as status[pass][t][d] = (AGG, c_d)
//     (tile 0: (INCL, c_d));
//  3. look-back, thread d: walk tiles t-1, t-2, ... (8 status words loaded
//     at once) adding AGG counts until an INCL one (the inclusive count of
//     digit d over all tiles before);
//     then publish (INCL, excl + c_d).  A wait for a tile that has published
//     nothing yet spins at most `budget` clock cycles; past that the pass
//     records sort_stall and publishes what it has, so no wait chains on it,
//     every later kernel of the build sees the stall and does nothing, and
//     the walk reports kFlagWaitTimeout;
//  4. keys staged in shared memory in (digit, input) order, then written
//     out: element i of the staged tile, digit d, goes to
//     digit_start[d] + excl_d + (i - local_start[d]), so consecutive threads
//     write consecutive addresses inside a digit's run.
// With Y != NULL (last pass) the layout is gathered into sorted order.
// status words: bits 31..30 flag (0 empty, 1 AGG, 2 INCL), 29..0 count
// (n < 2^30).
constexpr uint32_t kStAgg = 1u << 30, kStIncl = 2u << 30, kStCount = (1u << 30) - 1u;
constexpr int kLookWindow = 8;  // predecessor tiles a look-back step reads at once

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Exclusive scans over the 256 threads of a CTA of two values at once
// (thread x gets the sums over threads < x).
__device__ __forceinline__ void block_excl_scan2(uint32_t a, uint32_t b, uint32_t& ea, uint32_t& eb,
                                                 uint2* wsum) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t ua = __shfl_up_sync(0xffffffffu, ia, o), ub = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) {
      ia += ua;
      ib += ub;
    }
  }
  if (lane == 31) wsum[w] = make_uint2(ia, ib);
  __syncthreads();
  uint32_t oa = 0u, ob = 0u;
  for (int v = 0; v < w; ++v) {
    oa += wsum[v].x;
    ob += wsum[v].y;
  }
  ea = oa + ia - a;
  eb = ob + ib - b;
}

__global__ void __launch_bounds__(kSortThreads)
    k_radix_onesweep(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin, int n, int pass,
                     const uint32_t* __restrict__ ghist, uint32_t* ctl, uint32_t* status, int ntiles,
                     long long budget, TreeState* st, uint64_t* __restrict__ kout, int32_t* __restrict__ vout,
                     const float2* __restrict__ Y, float2* __restrict__ ys) {
  __shared__ uint32_t hw[kSortWarps][kRadixBins];
  __shared__ uint64_t skey[kSortTile];
  __shared__ int32_t sval[kSortTile];
  __shared__ uint32_t lstart[kRadixBins], gbase[kRadixBins];
  __shared__ uint2 wsum[kSortWarps];
  __shared__ int tile_s;
  if (__ldcg(&st->sort_stall)) return;  // an earlier pass gave up: nothing of this build is valid
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  if (tid == 0) tile_s = (int)atomicAdd(ctl + pass, 1u);
  for (int k = tid; k < kSortWarps * kRadixBins; k += kSortThreads) (&hw[0][0])[k] = 0u;
  __syncthreads();
  const int t = tile_s;
  if (t >= ntiles) return;  // uniform: more CTAs than tiles never happens, kept as a guard
  const int64_t t0 = (int64_t)t * kSortTile;
  const int tn = (int)min((int64_t)kSortTile, (int64_t)n - t0);
  const int shift = 8 * pass;
  const uint32_t lt = (1u << lane) - 1u;
  const int wb = w * (32 * kSortItems) + lane;
  uint64_t key[kSortItems];
  int32_t val[kSortItems];
  uint32_t rk[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {  // all loads of the tile in flight at once
    const int i = wb + 32 * r;
    key[r] = i < tn ? kin[t0 + i] : 0ull;
    val[r] = i < tn ? vin[t0 + i] : 0;
  }
  // 1. ranks within the warp
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const bool valid = wb + 32 * r < tn;
    const uint32_t d = valid ? (uint32_t)(key[r] >> shift) & 255u : 256u + (uint32_t)lane;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = valid ? hw[w][d] : 0u;
    rk[r] = before + (uint32_t)__popc(peers & lt);
    __syncwarp();
    if (valid && (peers & lt) == 0u) hw[w][d] = before + (uint32_t)__popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // 2. per digit: offsets of the warps, count of the tile, published
  const int d = tid;
  uint32_t cnt = 0u;
#pragma unroll
  for (int v = 0; v < kSortWarps; ++v) {
    const uint32_t x = hw[v][d];
    hw[v][d] = cnt;
    cnt += x;
  }
  uint32_t* const sbase = status + (size_t)pass * ntiles * kRadixBins;
  st_relaxed_u32(sbase + (size_t)t * kRadixBins + d, (t == 0 ? kStIncl : kStAgg) | cnt);
  uint32_t dstart, lst;
  block_excl_scan2(__ldg(ghist + pass * kRadixBins + d), cnt, dstart, lst, wsum);
  // 3. look-back
  uint32_t excl = 0u;
  if (t > 0) {
    const long long c0 = clock64();
    bool stalled = false, done = false;
    // windows of kLookWindow predecessors, loaded at once, read nearest first
    for (int k = t - 1; !done && !stalled; k -= kLookWindow) {
      uint32_t sw[kLookWindow];
#pragma unroll
      for (int u = 0; u < kLookWindow; ++u)
        sw[u] = k - u >= 0 ? ld_relaxed_u32(sbase + (size_t)(k - u) * kRadixBins + d) : kStIncl;
#pragma unroll
      for (int u = 0; u < kLookWindow; ++u) {
        uint32_t v = sw[u];
        while ((v >> 30) == 0u) {  // tile k - u (>= 0: tiles < 0 read as INCL 0) has published nothing yet
          if (clock64() - c0 > budget) {
            stalled = true;
            break;
          }
          v = ld_relaxed_u32(sbase + (size_t)(k - u) * kRadixBins + d);
        }
        if (stalled) break;
        excl += v & kStCount;
        if ((v & kStIncl) != 0u) {  // tile 0 always publishes INCL
          done = true;
          break;
        }
      }
    }
    if (stalled) atomicExch(&st->sort_stall, 1u);
    st_relaxed_u32(sbase + (size_t)t * kRadixBins + d, kStIncl | ((excl + cnt) & kStCount));
  }
  gbase[d] = dstart + excl;
  lstart[d] = lst;
  __syncthreads();
  // 4. stage in (digit, input) order, then write out
#pragma unroll
  for (int r = 0; r < kSortItems; ++r)
    if (wb + 32 * r < tn) {
      const uint32_t dg = (uint32_t)(key[r] >> shift) & 255u;
      const uint32_t lp = lstart[dg] + hw[w][dg] + rk[r];
      skey[lp] = key[r];
      sval[lp] = val[r];
    }
  __syncthreads();
  for (int i = tid; i < tn; i += kSortThreads) {
    const uint64_t kk = skey[i];
    const uint32_t dg = (uint32_t)(kk >> shift) & 255u;
    const uint32_t pos = gbase[dg] + ((uint32_t)i - lstart[dg]);
    if (pos < (uint32_t)n) {  // always true unless a wait ran out
      const int32_t v = sval[i];
      kout[pos] = kk;
      vout[pos] = v;
      if (ys != nullptr && (uint32_t)v < (uint32_t)n) ys[pos] = Y[v];
    }
  }
}

// ---------------------------------------------------------------- 4. tree

// Tree, summaries and group starts in one bottom-up pass (agglomerative
// construction of the binary radix tree, Apetrei 2014): the thread of leaf k
// holds a node with range [L, R] and climbs.  The parent of [L, R] is the
// node split between R and R + 1 if the augmented keys R, R + 1 share a
// longer prefix than keys L - 1, L (a range end counts as -1), else the node
// split between L - 1 and L; this gives exactly the tree of the definition
// (the one whose node over [f, l] splits at the highest differing bit).
// Internal node ids are their split positions (node g has children over
// [f, g] and [g + 1, l]); leaves are ~position.  A child reaching its parent
// exchanges (the end of the parent's range it knows, its own id) with the
// parent's slot: the first arrival leaves, the second learns the sibling,
// computes the parent (left + right: FP32 addition is commutative, so it
// does not matter which child's thread that is) and climbs on.  A completed
// node of more than kGroupMax points marks the first positions of its
// children that hold at most kGroupMax (the groups: maximal subtrees of at
// most kGroupMax points).
constexpr int kGroupMax = 32;
constexpr unsigned long long kSlotEmpty = ~0ull;

// Common-prefix length of the augmented keys (ka, a) and (kb, b).
__device__ __forceinline__ int aug_prefix(uint64_t ka, uint64_t kb, int a, int b) {
  return ka != kb ? __clzll((long long)(ka ^ kb)) : 64 + __clz((uint32_t)a ^ (uint32_t)b);
}

// Exchange at a node: acquire-release, so the summary a child's thread
// stored before its exchange is visible to the sibling's thread after its own.
__device__ __forceinline__ unsigned long long atom_exch_acq_rel(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.exch.b64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}

__global__ void k_tree_climb(int n, const uint64_t* __restrict__ keys, const float2* __restrict__ ys,
                             unsigned long long* slot, float4* box, float2* sum, float4* __restrict__ nodeA,
                             int4* __restrict__ nodeB, int32_t* __restrict__ is_start, TreeState* st) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n || __ldcg(&st->sort_stall)) return;
  if (n == 1) {
    is_start[0] = 1;
    st->root = ~0;
    return;
  }
  int L = k, R = k, id = ~k;
  const float2 q = ys[k];
  float4 bc = make_float4(q.x, q.y, q.x, q.y);
  float2 sc = q;
  uint64_t kL = keys[k], kR = kL;
  uint64_t kLm = k > 0 ? keys[k - 1] : 0ull, kRp = k < n - 1 ? keys[k + 1] : 0ull;
  for (;;) {
    const int dl = L > 0 ? aug_prefix(kLm, kL, L - 1, L) : -1;
    const int dr = R < n - 1 ? aug_prefix(kR, kRp, R, R + 1) : -1;
    const bool toward_right = dr > dl;  // this node is the left child
    const int p = toward_right ? R : L - 1;
    const int bound = toward_right ? L : R;
    const unsigned long long old =
        atom_exch_acq_rel(slot + p, ((unsigned long long)(uint32_t)bound << 32) | (uint32_t)id);
    if (old == kSlotEmpty) return;
    slot[p] = kSlotEmpty;  // both arrivals are in: ready for the next pass
    const int sbound = (int)(old >> 32), sid = (int)(uint32_t)old;
    const int pL = toward_right ? L : sbound, pR = toward_right ? sbound : R;
    // the sibling's summary and the keys at the parent's new end, at once
    float4 bs;
    float2 ss;
    if (sid < 0) {
      const float2 t = ys[~sid];
      bs = make_float4(t.x, t.y, t.x, t.y);
      ss = t;
    } else {
      bs = __ldcg(box + sid);
      ss = __ldcg(sum + sid);
    }
    if (toward_right) {
      kR = keys[pR];
      kRp = pR < n - 1 ? keys[pR + 1] : 0ull;
    } else {
      kL = keys[pL];
      kLm = pL > 0 ? keys[pL - 1] : 0ull;
    }
    sc = make_float2(__fadd_rn(sc.x, ss.x), __fadd_rn(sc.y, ss.y));
    bc = make_float4(fminf(bc.x, bs.x), fminf(bc.y, bs.y), fmaxf(bc.z, bs.z), fmaxf(bc.w, bs.w));
    box[p] = bc;
    sum[p] = sc;
    const int cntp = pR - pL + 1;
    const float cnt = (float)cntp;
    const float r = fmaxf(__fsub_rn(bc.z, bc.x), __fsub_rn(bc.w, bc.y));
    nodeA[p] = make_float4(__fdiv_rn(sc.x, cnt), __fdiv_rn(sc.y, cnt), __fmul_rn(r, r), cnt);
    nodeB[p] = toward_right ? make_int4(id, sid, pL, pR) : make_int4(sid, id, pL, pR);
    if (cntp > kGroupMax) {
      if (p - pL + 1 <= kGroupMax) is_start[pL] = 1;     // left child [pL, p]
      if (pR - p <= kGroupMax) is_start[p + 1] = 1;      // right child [p + 1, pR]
    }
    if (pL == 0 && pR == n - 1) {  // the root
      st->root = p;
      if (cntp <= kGroupMax) is_start[0] = 1;
      return;
    }
    L = pL;
    R = pR;
    id = p;
  }
}

// --------------------------------------------------------------- 6. groups

// gstart[g] = first position of group g; gstart[ngroups] = n.
__global__ void k_tree_group_list(int n, const TreeState* st, const int32_t* __restrict__ is_start,
                                  const int64_t* __restrict__ gscan, int32_t* __restrict__ gstart) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n || __ldcg(&st->sort_stall)) return;
  if (is_start[k]) gstart[gscan[k]] = k;
  if (k == 0) gstart[gscan[n]] = n;
}

// ---------------------------------------------------------------- 7. walk

// Walk of one group, 32 stack entries per round: each lane takes one entry
// (the top of the stack), loads its node record and decides: accept (r2 <
// theta^2 d2: one interaction of weight count at the centre), sum exactly
// (at most kTreeBucket points) or open (push both children).  Ballots
// compact the three outcomes into shared-memory lists in lane order; then
// every lane applies all accepted nodes and all exact points of the round
// to its own point.  A leaf (sorted position j) is the record (y_j, r2 = 0,
// count 1): accepting it is the exact interaction with its point, and it is
// never accepted by its own group (distance 0 to the box), which takes the
// exact path with the self term removed.  The set of interactions is the
// definition's; only the order of the sums differs from a depth-first walk.
// A round's interactions form one list: an accepted node is one item
// (centre, count), an exact entry is one item per point (point, 1).  The
// deciding lanes write their items at offsets from a warp scan of the item
// counts, as negated x, negated y and weight arrays, so two items are read as
// three FP32x2 words and go through the packed arithmetic unchanged.  A
// lane's own point, when an exact entry holds it, is summed like any other
// item: its force term is exactly zero (dx = dy = 0) and its Z term, 1 / (1 +
// 0) as computed, is subtracted once at the end (the entries mark which lanes
// they cover) instead of masking every item.  An accepted node may also hold
// the group's own points (coincident points: a centre one rounding away from
// them, a box of size zero); it is then one monopole term as the definition
// says, with nothing subtracted.
// Stack bound: a round that starts at <= kWalkStack - 200 entries pops up to
// 32 and pushes up to 64, ending at <= kWalkStack - 168; above kWalkStack -
// 200 rounds pop one entry (a depth-first walk, which adds at most one entry
// per tree level, and the tree has at most 94 levels: 64 key bits and 30
// index bits), so the stack stays below kWalkStack - 74.
constexpr int kWalkStack = 512;
constexpr int kWalkList = 32 * kTreeBucket + 4;  // items of one round at most, plus padding (even)

// Two interactions at once: items (-x, -y, c) packed in pairs against p; FX,
// FY, Z hold two partial sums each.
__device__ __forceinline__ void interact2(u64 PX, u64 PY, u64 NX, u64 NY, u64 C, u64& FX, u64& FY, u64& Z) {
  const u64 dx = add2(PX, NX);
  const u64 dy = add2(PY, NY);
  u64 q = fma2(dx, dx, pk(1.0f, 1.0f));
  q = fma2(dy, dy, q);
  float q0, q1;
  upk(q, q0, q1);
  const u64 w = pk(rcp_approx(q0), rcp_approx(q1));
  const u64 cw = mul2(C, w);
  Z = add2(Z, cw);
  const u64 cw2 = mul2(cw, w);
  FX = fma2(cw2, dx, FX);
  FY = fma2(cw2, dy, FY);
}

__global__ void __launch_bounds__(32 * kWalkWarps, 4)
    k_tree_walk(int n, const float2* __restrict__ ys, const int32_t* __restrict__ perm,
                const float4* __restrict__ nodeA, const int4* __restrict__ nodeB, const int32_t* __restrict__ gstart,
                const int64_t* __restrict__ gscan, float theta2, float2* __restrict__ frep,
                double* __restrict__ zgroup, Sched* sched, TreeState* st, int advance, float ee, int ee_iters,
                float mom0, float mom1) {
  __shared__ int stk[kWalkWarps][kWalkStack];
  __shared__ __align__(8) float lnx[kWalkWarps][kWalkList];
  __shared__ __align__(8) float lny[kWalkWarps][kWalkList];
  __shared__ __align__(8) float lc[kWalkWarps][kWalkList];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  // A sort wait that ran out leaves no valid tree: the pass only zeroes the
  // forces and reports the timeout.
  const bool stalled = __ldcg(&st->sort_stall) != 0u;
  const int ngroups = stalled ? 0 : (int)gscan[n];
  const int root = __ldcg(&st->root);  // internal node id, or ~0 for a single point
  if (stalled)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      frep[i] = make_float2(0.f, 0.f);
  for (;;) {
    int g = 0;
    if (lane == 0) g = (int)atomicAdd(&st->next_group, 1u);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= ngroups) break;
    const int k0 = gstart[g], k1 = gstart[g + 1];
    const int k = k0 + lane;
    const bool act = k < k1;
    const float2 p = ys[act ? k : k0];
    const float gx0 = warp_min(p.x), gy0 = warp_min(p.y), gx1 = warp_max(p.x), gy1 = warp_max(p.y);
    const u64 PX = pk(p.x, p.x), PY = pk(p.y, p.y);
    u64 FX = 0ull, FY = 0ull;
    double zd = 0.0;
    bool overflow = false;
    uint32_t seen = 0u;  // lanes whose own point an exact entry held
    if (lane == 0) stk[w][0] = root;
    int sp = 1;
    while (sp > 0) {
      __syncwarp();
      const int take = sp > kWalkStack - 200 ? 1 : (sp < 32 ? sp : 32);
      const bool has = lane < take;
      const int v = has ? stk[w][sp - take + lane] : 0;
      sp -= take;
      int kind = 0;  // 1 accept, 2 exact, 3 open
      float4 A = make_float4(0.f, 0.f, 0.f, 0.f);
      int4 B = make_int4(0, 0, 0, 0);
      const bool vok = !has || (v < 0 ? TS_IN(~v, 0, n, &sched->flags) : TS_IN(v, 0, n - 1, &sched->flags));
      if (has && vok) {
        if (v < 0) {
          const float2 q = ys[~v];
          A = make_float4(q.x, q.y, 0.f, 1.f);
          B = make_int4(-1, -1, ~v, ~v);
        } else {
          A = nodeA[v];
          B = nodeB[v];
        }
        const float dx = fmaxf(fmaxf(__fsub_rn(gx0, A.x), __fsub_rn(A.x, gx1)), 0.0f);
        const float dy = fmaxf(fmaxf(__fsub_rn(gy0, A.y), __fsub_rn(A.y, gy1)), 0.0f);
        const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        kind = A.z < __fmul_rn(theta2, d2) ? 1 : (B.w - B.z + 1 <= kTreeBucket ? 2 : 3);
      }
      const uint32_t mo = __ballot_sync(0xffffffffu, kind == 3);
      // list offsets: exclusive scan of the items per lane
      const int cnt = kind == 1 ? 1 : (kind == 2 ? B.w - B.z + 1 : 0);
      int off = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += u;
      }
      const int ni = __shfl_sync(0xffffffffu, off, 31);
      off -= cnt;
      if (kind == 1 && TS_IN(off, 0, kWalkList, &sched->flags)) {
        lnx[w][off] = -A.x;
        lny[w][off] = -A.y;
        lc[w][off] = A.w;
      }
      uint32_t cover = 0u;
      if (kind == 2) {
#pragma unroll
        for (int u = 0; u < kTreeBucket; ++u)
          if (u < cnt && TS_IN(B.z + u, 0, n, &sched->flags) && TS_IN(off + u, 0, kWalkList, &sched->flags)) {
            const float2 q = ys[B.z + u];
            lnx[w][off + u] = -q.x;
            lny[w][off + u] = -q.y;
            lc[w][off + u] = 1.0f;
          }
        const int lo = max(B.z, k0) - k0, hi = min(B.w, k1 - 1) - k0;  // lanes whose points it holds
        if (lo <= hi) cover = ((1u << (hi - lo + 1)) - 1u) << lo;  // hi - lo < kTreeBucket
      }
      seen |= __reduce_or_sync(0xffffffffu, cover);
      if (lane == 0 && (ni & 1) && TS_IN(ni, 0, kWalkList, &sched->flags)) {  // pad to a whole pair with a zero-weight item
        lnx[w][ni] = 0.f;
        lny[w][ni] = 0.f;
        lc[w][ni] = 0.f;
      }
      __syncwarp();  // every lane has read its entry before the pushes reuse the slots
      const int npush = 2 * __popc(mo);
      if (sp + npush <= kWalkStack) {
        if (kind == 3 && TS_IN(sp + 2 * __popc(mo & lt) + 1, 0, kWalkStack, &sched->flags)) {
          const int slot = sp + 2 * __popc(mo & lt);
          stk[w][slot] = B.y;  // right below, left on top
          stk[w][slot + 1] = B.x;
        }
        sp += npush;
      } else {
        overflow = true;  // excluded by the bound above; recorded, never written past
      }
      __syncwarp();
      u64 Z = 0ull;
      for (int t = 0; t < ni && TS_IN(t + 1, 0, kWalkList, &sched->flags); t += 2)
        interact2(PX, PY, *reinterpret_cast<const u64*>(&lnx[w][t]), *reinterpret_cast<const u64*>(&lny[w][t]),
                  *reinterpret_cast<const u64*>(&lc[w][t]), FX, FY, Z);
      float z0, z1;
      upk(Z, z0, z1);
      zd += (double)z0 + (double)z1;
    }
    if ((seen >> lane) & 1u) zd -= (double)rcp_approx(1.0f);  // the lane's own term out
    if (!act) zd = 0.0;                                          // idle lanes add nothing
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zd += __shfl_xor_sync(0xffffffffu, zd, o);
    if (lane == 0) {
      zgroup[g] = zd;
      if (overflow) atomicOr(&sched->flags, kFlagTreeOverflow);
    }
    if (act) {
      float fx0, fx1, fy0, fy1;
      upk(FX, fx0, fx1);
      upk(FY, fy0, fy1);
      if (TS_IN(perm[k], 0, n, &sched->flags)) frep[perm[k]] = make_float2(fx0 + fx1, fy0 + fy1);
    }
  }
  if (arrive_last(&st->walk_done)) {
    const double total = sum_partials(zgroup, ngroups);
    if (threadIdx.x == 0) {
      st->next_group = 0u;
      if (stalled)
        atomicOr(&sched->flags, kFlagWaitTimeout);
      else {
        sched->Z = total;
        sched->inv_z = (float)(1.0 / total);
      }
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
  if (n >= (1 << 30)) {
    last_msg() = "the tree code takes fewer than 2^30 points";
    return TSGNE_ERR_INVALID_ARG;
  }
  ntiles = (n + kSortTile - 1) / kSortTile;
  box_blocks = grid_for(n, 256, 2 * sm_count);
  keys_blocks = grid_for(n, 1024, sm_count);
  int per_sm = 0;
  TS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tree_walk, 32 * kWalkWarps, 0));
  walk_blocks = sm_count * (per_sm > 0 ? per_sm : 1);
  const size_t nn = (size_t)(n > 1 ? n - 1 : 1);
  TS_TRY(keys[0].alloc((size_t)n));
  TS_TRY(keys[1].alloc((size_t)n));
  TS_TRY(vals[0].alloc((size_t)n));
  TS_TRY(vals[1].alloc((size_t)n));
  TS_TRY(ys.alloc((size_t)n));
  TS_TRY(sortmem.alloc(sort_words()));
  TS_TRY(scan_scr.alloc(scan_scratch_bytes(n) / sizeof(int64_t)));
  TS_TRY(is_start.alloc((size_t)n));
  TS_TRY(gscan.alloc((size_t)n + 1));
  TS_TRY(gstart.alloc((size_t)n + 1));
  TS_TRY(nodeA.alloc(nn));
  TS_TRY(nodeB.alloc(nn));
  TS_TRY(box.alloc(nn));
  TS_TRY(sum.alloc(nn));
  TS_TRY(slot.alloc(nn));
  TS_TRY(boxpart.alloc((size_t)box_blocks));
  TS_TRY(zgroup.alloc((size_t)n));
  TS_TRY(state.alloc(1));
  TS_CUDA(cudaMemsetAsync(slot.get(), 0xff, sizeof(unsigned long long) * nn, s));  // every slot empty
  TS_CUDA(cudaMemsetAsync(state.get(), 0, sizeof(TreeState), s));
  return TSGNE_OK;
}

tsgne_status launch_tree_build(TreeBufs& tb, const float2* Y, cudaStream_t s) {
  const int n = tb.n;
  TreeState* st = tb.state.get();
  uint32_t* ghist = tb.sortmem.get();
  uint32_t* ctl = ghist + kRadixPasses * kRadixBins;
  uint32_t* status = ctl + kRadixPasses;
  k_tree_box<<<tb.box_blocks, 256, 0, s>>>(Y, n, tb.boxpart.get(), st, tb.sortmem.get(), (int64_t)tb.sort_words(),
                                           tb.is_start.get());
  k_tree_keys<<<tb.keys_blocks, 256, 0, s>>>(Y, n, st, tb.keys[0].get(), tb.vals[0].get(), ghist);
  TS_CUDA(cudaGetLastError());
  for (int pass = 0; pass < kRadixPasses; ++pass) {
    const int in = pass & 1, out = in ^ 1;
    const bool last = pass == kRadixPasses - 1;
    k_radix_onesweep<<<tb.ntiles, kSortThreads, 0, s>>>(tb.keys[in].get(), tb.vals[in].get(), n, pass, ghist, ctl,
                                                        status, tb.ntiles, tb.spin_budget, st, tb.keys[out].get(),
                                                        tb.vals[out].get(), last ? Y : nullptr,
                                                        last ? tb.ys.get() : nullptr);
    TS_CUDA(cudaGetLastError());
  }
  // an even number of passes: sorted keys / permutation are back in slot 0
  static_assert(kRadixPasses % 2 == 0, "sorted keys end in slot 0");
  k_tree_climb<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(n, tb.keys[0].get(), tb.ys.get(), tb.slot.get(),
                                                         tb.box.get(), tb.sum.get(), tb.nodeA.get(), tb.nodeB.get(),
                                                         tb.is_start.get(), st);
  TS_CUDA(cudaGetLastError());
  TS_TRY(scan_i32_to_i64(tb.is_start.get(), tb.gscan.get(), n, tb.scan_scr.get(), s));
  k_tree_group_list<<<grid_for(n, 256, 1 << 30), 256, 0, s>>>(n, st, tb.is_start.get(), tb.gscan.get(),
                                                               tb.gstart.get());
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

tsgne_status launch_tree_walk(TreeBufs& tb, float theta, float2* frep, Sched* sched, int advance, float ee,
                              int ee_iters, float mom0, float mom1, cudaStream_t s) {
  const float theta2 = theta * theta;
  k_tree_walk<<<tb.walk_blocks, 32 * kWalkWarps, 0, s>>>(tb.n, tb.ys.get(), tb.vals[0].get(), tb.nodeA.get(),
                                                         tb.nodeB.get(), tb.gstart.get(), tb.gscan.get(), theta2,
                                                         frep, tb.zgroup.get(), sched, tb.state.get(), advance, ee,
                                                         ee_iters, mom0, mom1);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

}  // namespace tsgne
