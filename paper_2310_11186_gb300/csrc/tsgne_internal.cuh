// Internal declarations shared by the translation units of libtsgne.so.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <new>
#include <string>

#include "tsgne.h"

namespace tsgne {

// Padding point of the repulsion tiles: its squared distance to any real
// point overflows to +inf in FP32, so its Student-t kernel value is exactly 0.
constexpr float kSentinel = 1e30f;

// Fixed-point scale of the exact repulsion's force accumulators: 2^s with
// s = 62 - ceil(log2 n).  Every term w^2 (y_i - y_j) has length r / (1 + r^2)^2
// <= 3 sqrt(3) / 16 < 0.33 (its maximum, at r = 1 / sqrt(3)), so any partial
// or total force component is below n / 2 in magnitude and below 2^61 once
// scaled: no int64 sum can overflow.  Resolution 2^-s (1.1e-13 at 300K points).
inline int fix_shift(int n) {
  int c = 0;
  while (c < 62 && (1LL << c) < (long long)n) ++c;
  return 62 - c;
}
inline float fix_scale(int n) { return ldexpf(1.0f, fix_shift(n)); }
inline float fix_unscale(int n) { return ldexpf(1.0f, -fix_shift(n)); }

// Device-resident scalars of the iteration (one per context).
struct Sched {
  double Z;            // normaliser of the last repulsion pass (ordered pairs, no diagonal)
  float alpha;         // exaggeration for the update that follows that pass
  float mu;            // momentum for the update that follows that pass
  int32_t t;           // index of the next iteration
  uint32_t flags;      // bit 0: non-finite layout seen; bit 1: non-finite P
  uint32_t rep_done;   // last-CTA counter of the repulsion pass
  uint32_t red_done;   // last-CTA counter of the generic reductions
  uint32_t work_next;  // work-queue head of the symmetric repulsion pass
  float inv_z;         // (float)(1 / Z), written with Z: the rows read it instead of dividing in FP64
  double red[4];       // results of the generic reductions
};

constexpr uint32_t kFlagNonfiniteY = 1u;
constexpr uint32_t kFlagNonfiniteP = 2u;
constexpr uint32_t kFlagTreeOverflow = 4u;
constexpr uint32_t kFlagWaitTimeout = 8u;  // a bounded device-side wait ran out (cleared once reported)
constexpr uint32_t kFlagIndexCheck = 16u;  // debug build: an index check failed (cleared once reported)

// Index checks of the debug build (compiled with -DTSGNE_DEBUG into
// libtsgne_debug.so).  TS_IN(v, lo, hi, flags) is true when lo <= v < hi;
// otherwise it records kFlagIndexCheck in the status word *flags (if not
// NULL) and is false, and the caller skips the access it guards.  Nothing
// traps.  In the regular build it is the constant true and compiles away.
#ifdef TSGNE_DEBUG
__device__ __forceinline__ bool ts_in(long long v, long long lo, long long hi, uint32_t* flags) {
  const bool ok = v >= lo && v < hi;
  if (!ok && flags) atomicOr(flags, kFlagIndexCheck);
  return ok;
}
#define TS_IN(v, lo, hi, flags) ::tsgne::ts_in((long long)(v), (long long)(lo), (long long)(hi), (flags))
#else
#define TS_IN(v, lo, hi, flags) true
#endif

// Geometry of one repulsion pass (see repulsion.cu and repulsion_sym.cu).
struct RepShape {
  int grid = 0;      // CTAs (a multiple of the SM count when the work allows)
  int block = 0;     // threads per CTA
  int R = 0;         // i-points per thread
  int jtile = 0;     // j-points staged in shared memory per tile
  int chunks = 0;    // ordered: partial force slots (j-chunks) per point; symmetric: tiles
  int n_pad = 0;     // padded length of Y buffers
  int n_iblk = 0;    // i-blocks of block*R points
  int n_jtiles = 0;  // j-tiles of jtile points
  int units = 0;     // work units of one pass (symmetric: tile pairs a <= b)
  int warps = 0;     // warps per CTA (symmetric)
  size_t smem = 0;   // dynamic shared memory per CTA (symmetric)
};

// Last error message of the calling thread (copied into the context by the API layer).
std::string& last_msg();

// Largest layout of the exact pass: its tile pairs are numbered in 32-bit
// ints, nt (nt + 1) / 2 for nt tiles, and the smallest tile (256 points)
// gives nt = 65,528 here.  An exact iteration at this size takes about a
// minute; the tree code takes up to 2^30 points.
constexpr int kMaxExactPoints = (1 << 24) - 2048;

// Runs f (which returns a status) and turns a failed host allocation into
// TSGNE_ERR_OOM, so that no C++ exception crosses the C ABI or ends a thread
// of the library.
template <class F>
tsgne_status host_guard(F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    last_msg() = "out of host memory";
    return TSGNE_ERR_OOM;
  }
}

// Returns TSGNE_ERR_OOM or TSGNE_ERR_CUDA for e and records a message.
tsgne_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define TS_CUDA(call)                                                   \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) return ::tsgne::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define TS_TRY(call)                        \
  do {                                      \
    tsgne_status s_ = (call);               \
    if (s_ != TSGNE_OK) return s_;          \
  } while (0)

// Process-wide account of the device bytes held by DevBufs, checked against
// an optional limit (tsgne_set_device_memory_limit).  reserve() returns false
// when the allocation would pass the limit; release() gives bytes back.
bool device_bytes_reserve(size_t bytes);
void device_bytes_release(size_t bytes);

// Stream for stream-ordered allocation by the calling thread (NULL: plain
// cudaMalloc / cudaFree).  cudaFree waits for the whole device, so a thread
// that prepares work while kernels of others run (the server's admission
// worker) allocates with cudaMallocAsync / cudaFreeAsync on its own stream.
cudaStream_t& alloc_stream();

// Owning device buffer released with cudaFree (or cudaFreeAsync on the
// stream it was allocated on, if the thread's alloc_stream was set then).
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t as = nullptr;  // stream of a stream-ordered allocation
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n), as(o.as) { o.p = nullptr; o.n = 0; o.as = nullptr; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { reset(); p = o.p; n = o.n; as = o.as; o.p = nullptr; o.n = 0; o.as = nullptr; }
    return *this;
  }
  ~DevBuf() { reset(); }
  void reset() {
    if (p) {
      if (as) cudaFreeAsync(p, as); else cudaFree(p);
      device_bytes_release(n * sizeof(T));
    }
    p = nullptr;
    n = 0;
    as = nullptr;
  }
  tsgne_status alloc(size_t count) {
    reset();
    if (count == 0) count = 1;
    if (!device_bytes_reserve(count * sizeof(T))) {
      last_msg() = "device memory limit reached (tsgne_set_device_memory_limit)";
      return TSGNE_ERR_OOM;
    }
    cudaStream_t s = alloc_stream();
    cudaError_t e = s ? cudaMallocAsync(&p, count * sizeof(T), s) : cudaMalloc(&p, count * sizeof(T));
    if (e == cudaSuccess) as = s;
    if (e != cudaSuccess) {
      p = nullptr;
      device_bytes_release(count * sizeof(T));
      return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    }
    n = count;
    return TSGNE_OK;
  }
  T* get() const { return p; }
};

// ---------------------------------------------------------------- scan
// Exclusive prefix sum of in[0..n) into out[0..n], out[n] = total.
size_t scan_scratch_bytes(int64_t n);
tsgne_status scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, void* scratch, cudaStream_t s);
// The first two phases only: out[k] = exclusive scan of k's block of
// kScanBlock entries, scratch[b] = exclusive scan of the block totals; the
// full exclusive scan at k is out[k] + scratch[k / kScanBlock].
constexpr int64_t kScanBlock = 2048;
tsgne_status scan_i32_to_i64_blocks(const int32_t* in, int64_t* out, int64_t n, void* scratch, cudaStream_t s);

// ------------------------------------------------------------ structure
// Symmetric, sorted, unique, loop-free structure of a validated CSR (device
// pointers).  Allocates *rp_out (n+1), *col_out (nnz) and *tslot_out (nnz).
// Synchronises the stream.  Returns BAD_CSR when the input is malformed.
tsgne_status build_structure(int n, const int64_t* rp_in, const int32_t* col_in, int64_t m, DevBuf<int64_t>& rp_out,
                             DevBuf<int32_t>& col_out, DevBuf<int64_t>& tslot_out, int64_t* nnz_out,
                             Sched* sched, cudaStream_t s);

// Neighbour structure for k_nn: 0 = the graph's edges (build_structure);
// k > 0 = the first k nodes of each node's BFS order (ties by ascending id),
// symmetrised by union (Eq. 7 with k nodes per list).  1 <= k <= 256.
tsgne_status build_neighbor_structure(int n, const int64_t* rp_in, const int32_t* col_in, int64_t m, int k_nn,
                                      DevBuf<int64_t>& rp_out, DevBuf<int32_t>& col_out, DevBuf<int64_t>& tslot_out,
                                      int64_t* nnz_out, cudaStream_t s);

// ------------------------------------------------------------- affinity
// p_{j|i} per entry (Eq. 2 over N(i), bisection of Sec. 2.1) then the joint
// P of Eq. 3 normalised by the total.  Sets kFlagNonfiniteP on NaN / Inf.
tsgne_status build_affinities(int n, const int64_t* rp, const int32_t* col, const int64_t* tslot, int64_t nnz,
                              const float* X, int d, float perplexity, float tol, int max_iter, float* P,
                              Sched* sched, cudaStream_t s);

// Eq. 3 from conditional affinities pcond on a symmetric structure with
// transpose slots: P = (pcond + pcond^T) / total, total into sched->red[0].
// Synchronises the stream.
tsgne_status joint_affinities(int64_t nnz, const float* pcond, const int64_t* tslot, float* P, Sched* sched,
                              cudaStream_t s);

// Random-walk estimate (Eq. 6, random_walk.cu): R walks of L steps from
// every node over the structure (rp, col); allocates the symmetrised
// structure of the walk pairs and its joint P.  Synchronises the stream.
tsgne_status random_walk_affinities(int n, const int64_t* rp, const int32_t* col, int64_t nnz, const float* X, int d,
                                    int R, int L, uint64_t seed, DevBuf<int64_t>& rp_out, DevBuf<int32_t>& col_out,
                                    DevBuf<float>& P_out, int64_t* nnz_out, Sched* sched, cudaStream_t s);

// ------------------------------------------------------ ShortestPath GE
// X (device, n x d float) = BFS distances to the d targets on the symmetric
// structure (rp, col) with nnz entries, capped at l0 + 1 (l0 <= 0: floor(sqrt(nnz/2))).
tsgne_status shortest_path_embedding(int n, const int64_t* rp, const int32_t* col, int64_t nnz,
                                     const int32_t* targets, int d, int l0, float* X, cudaStream_t s);

// ------------------------------------------------------------ repulsion
RepShape repulsion_shape(int n, int sm_count);
size_t repulsion_zpart_count(const RepShape& sh);
// One pass: partial forces frep_part[chunk][n_pad] (float2), Z into sched;
// advance != 0 also sets alpha / mu for iteration sched->t and increments t.
tsgne_status launch_repulsion(const RepShape& sh, int n, const float2* Y, float2* frep_part, double* zpart,
                              Sched* sched, int advance, float ee, int ee_iters, float mom0, float mom1,
                              cudaStream_t s);

// Symmetric pass: every unordered pair once (repulsion_sym.cu).  Adds the
// forces of the n real points into the fixed-point accumulators acc[2 n]
// (int64 pairs at scale fix_scale(n); zero before the pass, read and
// cleared by launch_fix_forces after it); Z and the schedule into sched as
// launch_repulsion does; zpart needs sh.units doubles.
// repulsion_sym_prepare sets kernel attributes (call it outside stream
// capture, once per shape).
RepShape repulsion_shape_sym(int n, int sm_count);
// A given shape: W warps per CTA (1 or 2), RI i-points per lane (8 or 16).
RepShape repulsion_shape_sym_fixed(int n, int sm_count, int W, int RI);
tsgne_status repulsion_sym_prepare(const RepShape& sh);
// Y is float2[n_pad] (y_bf16 = 0) or __nv_bfloat162[n_pad] (y_bf16 = 1).
tsgne_status launch_repulsion_sym(const RepShape& sh, int n, const void* Y, int y_bf16, unsigned long long* acc,
                                  double* zpart, Sched* sched, int advance, float ee, int ee_iters, float mom0,
                                  float mom1, cudaStream_t s);
// A share of the pass for sharding one layout over several GPUs: only units
// [u0, u1) of the sh.units tile pairs (forces into acc, unit partials into
// zpart[u0..u1)); Z and the schedule are left to launch_finalize_z, after
// the caller has summed acc and zpart over the shares.
tsgne_status launch_repulsion_sym_units(const RepShape& sh, int n, const void* Y, int y_bf16,
                                        unsigned long long* acc, double* zpart, Sched* sched, int u0, int u1,
                                        cudaStream_t s);
// Z = fixed-order sum of zpart[0..sh.units) - n and the schedule, as the last
// CTA of a whole pass sets them (same block size, so the same bits).
tsgne_status launch_finalize_z(const RepShape& sh, int n, const double* zpart, Sched* sched, int advance, float ee,
                               int ee_iters, float mom0, float mom1, cudaStream_t s);
// F^r[i] = sum_k part[k * n_pad + i] for k < slots, in slot order (the
// ordered-pair kernel's partial forces).
tsgne_status launch_reduce_slots(int n, const float2* part, int slots, int n_pad, float2* out, cudaStream_t s);
// F^r[i] = acc[2 i .. 2 i + 1] / fix_scale(n) (one FP32 rounding of the exact
// integer sum), and the accumulators back to zero for the next pass.
tsgne_status launch_fix_forces(int n, unsigned long long* acc, float2* out, cudaStream_t s);

// ------------------------------------------------------------ iteration
// Rows with more than kHeavyDeg entries get their attraction from chunks of
// kHeavyChunk entries, one warp per chunk (k_attract_heavy); the update adds a
// row's chunk sums in chunk order.  rows[] is sorted; chunks of heavy row k
// are chunk_off[k] .. chunk_off[k+1]-1.  Rows up to kHeavyDeg entries are
// one 4-entry batch per lane of an 8-lane group, so no group waits on another.
constexpr int kHeavyDeg = 32;
constexpr int kHeavyChunk = 1024;
struct HeavyRows {
  const int32_t* rows = nullptr;       // [count] sorted row ids
  const int32_t* chunk_off = nullptr;  // [count + 1]
  const int32_t* chunk_row = nullptr;  // [chunks]
  const int64_t* chunk_begin = nullptr;  // [chunks] first entry
  const int64_t* chunk_end = nullptr;    // [chunks] one past the last entry
  float2* fa = nullptr;                // [chunks] partial sums
  const int32_t* chunk_heavy = nullptr;  // [chunks] index of the chunk's row in rows
  uint32_t* arrivals = nullptr;        // [count] chunks done this pass (zero between passes)
  int count = 0;
  int chunks = 0;
};
struct HeavyStore {
  DevBuf<int32_t> rows, chunk_off, chunk_row, chunk_heavy;
  DevBuf<int64_t> chunk_begin, chunk_end;
  DevBuf<float2> fa;
  DevBuf<uint32_t> arrivals;
  int count = 0, chunks = 0;
  HeavyRows view() const {
    HeavyRows h;
    h.rows = rows.get();
    h.chunk_off = chunk_off.get();
    h.chunk_row = chunk_row.get();
    h.chunk_begin = chunk_begin.get();
    h.chunk_heavy = chunk_heavy.get();
    h.arrivals = arrivals.get();
    h.chunk_end = chunk_end.get();
    h.fa = fa.get();
    h.count = count;
    h.chunks = chunks;
    return h;
  }
};
tsgne_status find_heavy_rows(int n, const int64_t* rp, HeavyStore& hs, cudaStream_t s);
// L2 prefetch of a buffer (no-op below 1 MB).
tsgne_status launch_prefetch_l2(const void* p, int64_t bytes, cudaStream_t s);

// Attraction + gradient + optimiser update: reads Ycur, writes Ynext.
// Arguments of the attraction / update pass.  P is float[nnz] (p_bf16 = 0)
// or bf16[nnz]; Yr is the layout the forces read: float2 (y_bf16 = 0) or the
// bf16x2 shadow; Ym is the FP32 master layout the update advances into Ynext
// (and, if not NULL, its bf16x2 shadow Ynext16).
struct AttractArgs {
  int n = 0;
  const int64_t* rp = nullptr;
  const int32_t* col = nullptr;
  const void* P = nullptr;
  int p_bf16 = 0;
  const void* Yr = nullptr;
  int y_bf16 = 0;
  const float2* Ym = nullptr;
  float2* Ynext = nullptr;
  void* Ynext16 = nullptr;
  float2* upd = nullptr;
  float2* gains = nullptr;
  const float2* frep = nullptr;
  int chunks = 1;
  int n_pad = 0;
  Sched* sched = nullptr;
  float eta = 0.f;
  float min_gain = 0.f;
  HeavyRows hv;
};
// Schedule of the attraction + update pass fixed when P is installed
// (attract_plan.cu): rows of at most 32 entries in CTAs of 256 consecutive
// rows, rows of 33..128 entries in CTAs of 64 listed rows, their slot chains
// one thread each with coalesced copies of col and P; rows above 128 entries
// one warp per hub chunk.  Same sums, same order as k_attract.
constexpr int kMedDeg = 128;
struct PlanCta {
  int64_t ent;    // first entry of the CTA's chains in colS / PS
  int32_t pair;   // first chain code
  int32_t rows;   // medium CTAs: first index into med_rows
  int32_t nrows;  // rows of the CTA
  int32_t pad_;
  int32_t cnt[4];  // chains of more than k entries, k = 0..3 (cnt[0]: all chains)
};
struct PlanView {
  const PlanCta* med = nullptr;     // [n_med]
  const PlanCta* shorts = nullptr;  // [n_short]
  const uint16_t* code = nullptr;   // chain codes: (row in CTA << 3 | slot) or (<< 5 | slot)
  const int32_t* colS = nullptr;    // col in chain order
  const void* PS = nullptr;         // P in chain order (float, or bf16 with BF16 storage)
  const int32_t* med_rows = nullptr;
  const int32_t* big = nullptr;     // hub chunks of the rows above 128 entries
  int n_med = 0, n_short = 0, n_big = 0;
  int64_t entries = 0, n_codes = 0, n_med_rows = 0;  // array lengths (index checks)
};
struct AttractPlan {
  DevBuf<PlanCta> cta;  // medium CTAs, then short CTAs
  DevBuf<uint16_t> code;
  DevBuf<int32_t> colS, med_rows, big;
  DevBuf<float> PS;
  DevBuf<__nv_bfloat16> PS16;
  int n_med = 0, n_short = 0, n_big = 0;
  int64_t entries = 0, n_codes = 0, n_med_rows = 0;
  bool ready = false;
  PlanView view() const;
};
// Builds the plan for the structure (rp, col) and P (FP32, or its BF16 copy
// when P16 is not NULL); hs must hold the hub rows of the same structure.
// Synchronises the stream.
tsgne_status build_attract_plan(int n, const int64_t* rp, const int32_t* col, const float* P,
                                const __nv_bfloat16* P16, const HeavyStore& hs, AttractPlan& plan, cudaStream_t s);
// The attraction + update pass on the plan (the update mode of
// k_attract: same results, bit for bit).
tsgne_status launch_attract_plan(const AttractArgs& a, const PlanView& pv, cudaStream_t s);
// Gradient export g = 4 (alpha F^a - F^r / Z) without state change.
tsgne_status launch_gradient(const AttractArgs& a, float alpha, float2* g, cudaStream_t s);
// Hub-row chunks for the layout a reads (the update then adds their sums).
tsgne_status launch_attract_heavy(const AttractArgs& a, cudaStream_t s);
// KL terms: sched->red[0] = sum p ln(p / w), sched->red[1] = sum p.
tsgne_status launch_kl(int n, const int64_t* rp, const int32_t* col, const void* P, int p_bf16, const void* Y,
                       int y_bf16, double* partials, int nparts, Sched* sched, cudaStream_t s);
// FP32 -> BF16 copies (round to nearest even); count scalars.
tsgne_status launch_to_bf16(const float* in, void* out, int64_t count, cudaStream_t s);
int kl_partial_count(int sm_count);
// Y0 ~ N(0, sigma^2) from a seed (SplitMix64 counter mode + Box-Muller).
tsgne_status launch_init_Y(int n, uint64_t seed, float sigma, float2* Y, cudaStream_t s);
// ------------------------------------------------- tree-code repulsion
// (repulsion_tree.cu): an opened node of at most this many points is summed
// exactly over its points.
constexpr int kTreeBucket = 4;

struct TreeState {
  double scale;                  // 2^32 / side of the bounding square of the last pass
  float lo_x, lo_y;              // its low corner
  uint32_t box_done, walk_done;  // last-CTA counters
  uint32_t next_group;           // work-queue head of the walk
  uint32_t sort_stall;           // 1: a look-back wait of this pass's sort ran out of its budget
  int32_t root;                  // root of the last tree: an internal node id, or ~0 (one point)
};

// Device buffers of the tree code for n points.
struct TreeBufs {
  int n = 0, ntiles = 0, box_blocks = 0, keys_blocks = 0, walk_blocks = 0;
  long long spin_budget = 2000000000LL;  // clock cycles a look-back wait of the sort may last
  DevBuf<uint64_t> keys[2];
  DevBuf<int32_t> vals[2];    // vals[0] after a build: sorted position -> point
  DevBuf<float2> ys;          // layout in sorted order
  DevBuf<uint32_t> sortmem;   // sort: digit counts [8][256], tile counters [8], tile status [8][ntiles][256]
  DevBuf<int64_t> scan_scr;
  DevBuf<float4> nodeA;       // internal node: centre x, y, r2, count
  DevBuf<int4> nodeB;         // internal node: left, right, first, last
  DevBuf<float4> box;         // internal node: x0, y0, x1, y1
  DevBuf<float2> sum;         // internal node: coordinate sums
  DevBuf<unsigned long long> slot;  // bottom-up exchange slots (kept empty, all ones, between passes)
  DevBuf<float4> boxpart;
  DevBuf<int32_t> is_start;   // 1 where a group begins (sorted positions)
  DevBuf<int64_t> gscan;      // exclusive scan of is_start; gscan[n] = number of groups
  DevBuf<int32_t> gstart;     // first sorted position of each group, then n
  DevBuf<double> zgroup;      // FP64 Z partial per group
  DevBuf<TreeState> state;
  size_t sort_words() const { return (size_t)8 * 256 + 8 + (size_t)8 * ntiles * 256; }
  tsgne_status alloc(int n_points, int sm_count, cudaStream_t s);
};
// Bounding square, keys, sort, tree and summaries of the layout Y[0..n).
tsgne_status launch_tree_build(TreeBufs& tb, const float2* Y, cudaStream_t s);
// Walk with opening angle theta: frep[i] (input order) and sched->Z, then the
// schedule of iteration sched->t as launch_repulsion does.
tsgne_status launch_tree_walk(TreeBufs& tb, float theta, float2* frep, Sched* sched, int advance, float ee,
                              int ee_iters, float mom0, float mom1, cudaStream_t s);

// Fill y[lo..hi) with the sentinel point.
tsgne_status launch_fill_sentinel(float2* Y, int lo, int hi, cudaStream_t s);
// Set every element of a float2 array to (v, v).
tsgne_status launch_fill2(float2* a, int n, float v, cudaStream_t s);

}  // namespace tsgne
