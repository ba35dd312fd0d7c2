// Many layouts per launch: the t-SGNE iteration of every member of a batch
// runs in four launches (five when a member has rows above 32 entries),
// whatever the number and sizes of the members.
//
//   k_batch_repulsion  one global work queue over the tile pairs of all
//                      members (prefix offsets per member); each unit is the
//                      same device code as the single-layout pass (sym_unit)
//                      on that member's buffers, so every member's forces and
//                      Z partials are the same bits as when it runs alone
//   k_batch_finalize   one CTA per member: Z = fixed-order sum of its unit
//                      partials minus n, schedule (alpha, mu) from its own
//                      iteration counter t, t += 1
//   k_batch_reduce     each point's fixed-point force accumulators to F^r,
//                      cleared for the next iteration
//   k_batch_hubs       (members with rows above 32 entries) one warp per
//                      1024-entry chunk of such a row, over all members'
//                      chunks: the single-layout path's chunk sums
//   k_batch_attract    attraction + gradient + optimiser step per row (a hub
//                      row adds its chunk sums in chunk order)
//
// Tree-code members (cfg.repulsion = 1, or per member through
// tsgne_batch_add_ex) take no units of k_batch_repulsion: each runs the
// single-layout tree code's build and walk on its own current layout, as
// its own chain of launches on a branch of the iteration (auxiliary
// streams, forked from and joined back into the batch stream, so in the
// captured graph the members' trees are built and walked concurrently),
// and the walk sets its forces, Z and schedule as k_batch_finalize does for
// the others.  Attraction and update are the shared launches above.
//
// Members keep their P, layout and optimiser state resident on the device
// and may differ in size and in iteration count (each has its own t); the
// current layout of a member is Y[t & 1], so one captured CUDA graph of the
// launches serves every iteration of a given membership.  All members of
// a batch use the same tile size T = 512 W; tsgne_batch_autotune picks W.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "reduce.cuh"
#include "row_update.cuh"
#include "sym_unit.cuh"
#include "tsgne_internal.cuh"

namespace tsgne {

struct GraphDesc {
  const int64_t* rp;
  const int32_t* col;
  const float* P;
  float2* Y[2];
  float2* upd;
  float2* gains;
  unsigned long long* acc;  // fixed-point force accumulators, 2 per point (scale fix_scale(n))
  float2* fsum;
  double* zunit;
  Sched* sched;
  HeavyRows hv;  // rows above kHeavyDeg entries, in kHeavyChunk-entry chunks (as the single-layout path)
  int n, nt, n_pad, units;
  float eta;
  float fscale, funscale;
  int tree;  // 1: tree-code repulsion (no units; forces and Z from its walk)
  int pad_;
};

struct BatchCtr {
  uint32_t work_next;
  uint32_t rep_done;
};

namespace {

constexpr int kMaxT = 2048;  // largest tile (W = 4); member buffers are padded to it
constexpr int kBG = 8;       // lanes per row in the update (as the single-layout kernel: same row sums)

// Largest k with off[k] <= v over off[0..count) (off non-decreasing, off[0] = 0).
__device__ __forceinline__ int find_owner(const int* __restrict__ off, int count, int v) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int W, int RI>
__global__ void __launch_bounds__(W * 32, warps_per_sm(RI) / W)
    k_batch_repulsion(const GraphDesc* __restrict__ descs, const int* __restrict__ unit_off, int members, int U,
                      BatchCtr* ctr) {
  constexpr int T = W * 32 * RI;
  extern __shared__ float4 smem[];
  float4* sj = smem;
  float2* sacc = reinterpret_cast<float2*>(smem + T);
  __shared__ int s_unit, s_g, s_a, s_b;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      const int u = (int)atomicAdd(&ctr->work_next, 1u);
      int g = 0, a = 0, b = 0;
      if (u < U) {
        g = find_owner(unit_off, members, u);
        unit_tiles(u - unit_off[g], descs[g].nt, &a, &b);
      }
      s_unit = u;
      s_g = g;
      s_a = a;
      s_b = b;
    }
    __syncthreads();
    const int u = s_unit, g = s_g, a = s_a, b = s_b;
    if (u >= U) break;
    const GraphDesc& d = descs[g];
    if (!(TS_IN(a, 0, d.nt, &d.sched->flags) && TS_IN(b, a, d.nt, &d.sched->flags))) {  // debug build only
      if (tid == 0) d.zunit[u - unit_off[g]] = 0.0;
      __syncthreads();
      continue;
    }
    const float2* Y = d.Y[d.sched->t & 1];
    const double zt = sym_unit<W, RI>(Y, d.n, d.acc, d.fscale, a, b, sj, sacc);
    const double zb = block_sum_d(zt);
    if (tid == 0) d.zunit[u - unit_off[g]] = zb;
    __syncthreads();
  }
  if (arrive_last(&ctr->rep_done) && tid == 0) ctr->work_next = 0u;
}

__global__ void k_batch_finalize(const GraphDesc* __restrict__ descs, float ee, int ee_iters, float mom0,
                                 float mom1) {
  const GraphDesc& d = descs[blockIdx.x];
  if (d.tree) return;  // its walk set Z and the schedule
  const double total = sum_partials(d.zunit, d.units);
  if (threadIdx.x == 0) {
    Sched* s = d.sched;
    s->Z = total - (double)d.n;
    s->inv_z = (float)(1.0 / s->Z);
    const int t = s->t;
    s->alpha = t < ee_iters ? ee : 1.0f;
    s->mu = t < ee_iters ? mom0 : mom1;
    s->t = t + 1;
  }
}

__global__ void k_batch_reduce(const GraphDesc* __restrict__ descs, const int* __restrict__ row_off, int members,
                               int R) {
  const int stride = gridDim.x * blockDim.x;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += stride) {
    const int g = find_owner(row_off, members, r);
    const GraphDesc& d = descs[g];
    const int i = r - row_off[g];
    if (d.tree) continue;  // its walk wrote F^r
    ulonglong2* a = reinterpret_cast<ulonglong2*>(d.acc) + i;
    const ulonglong2 v = *a;
    d.fsum[i] = make_float2(__ll2float_rn((long long)v.x) * d.funscale, __ll2float_rn((long long)v.y) * d.funscale);
    *a = make_ulonglong2(0ull, 0ull);
  }
}

// A tree member's current layout Y[t & 1] into the buffer its tree build reads.
__global__ void k_member_cur_Y(const float2* __restrict__ Y0, const float2* __restrict__ Y1, const Sched* sched, int n,
                               float2* __restrict__ out) {
  const float2* Y = (sched->t & 1) ? Y1 : Y0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = Y[i];
}

// One warp per chunk of every member's hub rows (global chunk index c over
// the members' chunk offsets), at the layout the update reads: the chunk's
// 32-lane sum, as k_attract_heavy computes it for one layout.
__global__ void __launch_bounds__(256) k_batch_hubs(const GraphDesc* __restrict__ descs,
                                                    const int* __restrict__ chunk_off, int members, int C) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < C; c += warps) {
    const int g = find_owner(chunk_off, members, c);
    const GraphDesc& d = descs[g];
    const int lc = c - chunk_off[g];
    const int64_t i = d.hv.chunk_row[lc];
    const float2* Ycur = d.Y[(d.sched->t - 1) & 1];  // t already advanced by k_batch_finalize
    float ax = 0.f, ay = 0.f;
    attract_entries_pipelined<32>(d.hv.chunk_begin[lc], d.hv.chunk_end[lc], d.col, d.P, Ycur, i, lane, Ycur[i], ax,
                                  ay);
    ax = group_sum<32>(ax);
    ay = group_sum<32>(ay);
    if (lane == 0) d.hv.fa[lc] = make_float2(ax, ay);
  }
}

template <int G>
__global__ void __launch_bounds__(256) k_batch_attract(const GraphDesc* __restrict__ descs,
                                                       const int* __restrict__ row_off, int members, int R,
                                                       float min_gain) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r = gt / G;
  const int lane = (int)(gt % G);
  const bool valid = r < R;
  __shared__ int s_g0;  // owner of the CTA's first row; the CTA's rows span few members
  if (threadIdx.x == 0) {
    const int64_t r0 = (int64_t)blockIdx.x * blockDim.x / G;
    s_g0 = r0 < R ? find_owner(row_off, members, (int)r0) : 0;
  }
  __syncthreads();
  int g = s_g0;
  if (valid)
    while (g + 1 < members && row_off[g + 1] <= (int)r) ++g;
  const GraphDesc& d = descs[g];
  const int64_t i = valid ? r - row_off[g] : 0;
  float ax = 0.f, ay = 0.f;
  float2 yi = make_float2(0.f, 0.f);
  int t = 0;
  if (valid) {
    t = d.sched->t;  // already advanced by k_batch_finalize
    const float2* Ycur = d.Y[(t - 1) & 1];
    yi = Ycur[i];
    if (d.rp[i + 1] - d.rp[i] > kHeavyDeg) {
      if (lane == 0) {  // chunk sums from k_batch_hubs, in chunk order
        int lo = 0, hi = d.hv.count - 1;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (d.hv.rows[mid] < i) lo = mid + 1; else hi = mid;
        }
        for (int c = d.hv.chunk_off[lo]; c < d.hv.chunk_off[lo + 1]; ++c) {
          const float2 f = d.hv.fa[c];
          ax += f.x;
          ay += f.y;
        }
      }
    } else {
      attract_row<G>(d.rp, d.col, d.P, Ycur, i, lane, yi, ax, ay);
    }
  }
  ax = group_sum<G>(ax);
  ay = group_sum<G>(ay);
  if (!valid || lane != 0) return;
  const Sched* s = d.sched;
  const float2 fr = d.fsum[i];
  const float invZ = s->inv_z;
  const float gx = 4.0f * (s->alpha * ax - fr.x * invZ);
  const float gy = 4.0f * (s->alpha * ay - fr.y * invZ);
  float2 u = d.upd[i], gn = d.gains[i];
  const float2 y = optimizer_step(gx, gy, u, gn, s->mu, d.eta, min_gain, yi);
  d.upd[i] = u;
  d.gains[i] = gn;
  d.Y[t & 1][i] = y;
  if (!isfinite(y.x) || !isfinite(y.y)) atomicOr(&d.sched->flags, kFlagNonfiniteY);
}

// The compiled shapes of the batched pass: (warps per CTA, i-points per lane).
constexpr int kShapes[6][2] = {{1, 16}, {2, 16}, {4, 16}, {1, 8}, {2, 8}, {4, 8}};

size_t smem_for(int W, int RI) { return (size_t)(W * 32 * RI) * (sizeof(float4) + sizeof(float2)); }

template <int W, int RI>
tsgne_status prepare_shape() {
  TS_CUDA(cudaFuncSetAttribute(k_batch_repulsion<W, RI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_for(W, RI)));
  return TSGNE_OK;
}

tsgne_status prepare_w(int W, int RI) {
  if (RI == 16) {
    if (W == 4) return prepare_shape<4, 16>();
    if (W == 2) return prepare_shape<2, 16>();
    return prepare_shape<1, 16>();
  }
  if (W == 4) return prepare_shape<4, 8>();
  if (W == 2) return prepare_shape<2, 8>();
  return prepare_shape<1, 8>();
}

// One member: affinities, layout, optimiser state and repulsion scratch.
struct Member {
  int id = -1;
  int n = 0;
  int64_t nnz = 0;
  int n_pad_max = 0;  // buffers sized for T = kMaxT
  float eta = 0.f;
  DevBuf<int64_t> rp;
  DevBuf<int32_t> col;
  DevBuf<float> P;
  DevBuf<float2> Y[2], upd, gains, fsum;
  DevBuf<unsigned long long> acc;  // fixed-point force accumulators (2 per point), zero between iterations
  DevBuf<double> zunit;
  DevBuf<Sched> sched;
  HeavyStore hv;                     // hub rows and their chunks
  int nt = 0, n_pad = 0, units = 0;  // for the batch's current tile
  DevBuf<float2> Y0;                 // initial layout (autotune restores it)
  bool active = true;
  bool tree = false;                 // tree-code repulsion
  TreeBufs tb;                       // its tree (tree members)
  DevBuf<float2> Ytree;              // its current layout, copied for the tree build
};

std::mutex g_cache_mu;
std::map<std::tuple<int, int, int>, int> g_tile_cache;  // (SMs, log2 pairs, log2 members) -> 100 W + RI

}  // namespace
}  // namespace tsgne

using namespace tsgne;

struct tsgne_member {
  std::unique_ptr<tsgne::Member> m;
};

struct tsgne_batch {
  tsgne_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0, sms = 1;
  int W = 1;
  int RI = kRI;  // i-points per lane of the batched pass
  std::string err;
  int next_id = 0;
  std::vector<std::unique_ptr<Member>> members;
  DevBuf<GraphDesc> d_desc;
  DevBuf<int> d_unit_off, d_row_off, d_chunk_off;
  DevBuf<BatchCtr> d_ctr;
  int U = 0, R = 0, G = 0, C = 0;  // of the active members (C: hub-row chunks)
  bool dirty = true;
  cudaGraphExec_t graph = nullptr;
  std::vector<Member*> trees;     // active tree members (refresh)
  std::vector<cudaStream_t> aux;  // branches of the tree members' launches
  std::vector<cudaEvent_t> ev;    // fork event, then one join event per tree member
  ~tsgne_batch() {
    // work still queued may read the members' buffers, and a buffer from the
    // admission worker is freed on the worker's stream, not on these
    if (stream) cudaStreamSynchronize(stream);
    for (auto a : aux) cudaStreamSynchronize(a);
    members.clear();  // stream-ordered frees need their streams
    if (graph) cudaGraphExecDestroy(graph);
    for (auto e : ev) cudaEventDestroy(e);
    for (auto a : aux) cudaStreamDestroy(a);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};

namespace {

tsgne_status bfail(tsgne_batch* b, tsgne_status st, const std::string& msg = std::string()) {
  if (b) b->err = msg.empty() ? last_msg() : msg;
  return st;
}

#define B_TRY(b, call)                             \
  do {                                             \
    tsgne_status s__ = (call);                     \
    if (s__ != TSGNE_OK) return bfail((b), s__);   \
  } while (0)

#define B_CUDA(b, call)                                                                    \
  do {                                                                                     \
    cudaError_t e__ = (call);                                                              \
    if (e__ != cudaSuccess) return bfail((b), cuda_fail(e__, #call, __FILE__, __LINE__));  \
  } while (0)

// The kernels' tile (sym_unit: 32 lanes x RI i-points x W warps); every
// tile size divides kMaxT, so a member's n_pad never exceeds its buffers'.
static_assert(kMaxT % (32 * 8) == 0 && 32 * 16 * 4 <= kMaxT, "tiles of 1, 2 and 4 warps must divide kMaxT");

void shape_member(Member& m, int W, int RI) {
  const int T = 32 * RI * W;
  m.nt = (m.n + T - 1) / T;
  m.n_pad = m.nt * T;
  m.units = m.tree ? 0 : m.nt * (m.nt + 1) / 2;
}

tsgne_status alloc_scratch(Member& m, int W, int RI) {
  shape_member(m, W, RI);
  TS_TRY(m.zunit.alloc((size_t)m.units));
  return TSGNE_OK;
}

void invalidate(tsgne_batch* b) {
  b->dirty = true;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

// Uploads descriptors and prefix offsets for the current membership.
tsgne_status refresh_impl(tsgne_batch* b) {
  if (!b->dirty) return TSGNE_OK;
  std::vector<Member*> act;
  b->trees.clear();
  for (auto& m : b->members)
    if (m->active) {
      act.push_back(m.get());
      if (m->tree) b->trees.push_back(m.get());
    }
  const int G = (int)act.size();
  b->G = G;
  std::vector<GraphDesc> h(G > 0 ? G : 1);
  std::vector<int> uo(G + 1, 0), ro(G + 1, 0), co(G + 1, 0);
  int64_t tu = 0, tr = 0, tc = 0;  // the totals are 32-bit in the kernels
  for (const Member* m : act) {
    tu += m->units;
    tr += m->n;
    tc += m->hv.chunks;
  }
  if (tu > INT32_MAX || tr * kBG > INT32_MAX || tc > INT32_MAX) {
    last_msg() = "the active members' tile pairs, rows or hub chunks exceed the batch's 32-bit counts";
    return TSGNE_ERR_INVALID_ARG;
  }
  for (int k = 0; k < G; ++k) {
    Member& m = *act[k];
    GraphDesc d{};
    d.rp = m.rp.get();
    d.col = m.col.get();
    d.P = m.P.get();
    d.Y[0] = m.Y[0].get();
    d.Y[1] = m.Y[1].get();
    d.upd = m.upd.get();
    d.gains = m.gains.get();
    d.acc = m.acc.get();
    d.fsum = m.fsum.get();
    d.zunit = m.zunit.get();
    d.sched = m.sched.get();
    d.hv = m.hv.view();
    d.n = m.n;
    d.nt = m.nt;
    d.n_pad = m.n_pad;
    d.units = m.units;
    d.eta = m.eta;
    d.fscale = fix_scale(m.n);
    d.funscale = fix_unscale(m.n);
    d.tree = m.tree ? 1 : 0;
    h[k] = d;
    uo[k + 1] = uo[k] + m.units;
    ro[k + 1] = ro[k] + m.n;
    co[k + 1] = co[k] + m.hv.chunks;
  }
  b->U = uo[G];
  b->R = ro[G];
  b->C = co[G];
  TS_TRY(b->d_desc.alloc(h.size()));
  TS_TRY(b->d_unit_off.alloc(uo.size()));
  TS_TRY(b->d_row_off.alloc(ro.size()));
  TS_TRY(b->d_chunk_off.alloc(co.size()));
  TS_CUDA(cudaMemcpyAsync(b->d_desc.get(), h.data(), sizeof(GraphDesc) * h.size(), cudaMemcpyHostToDevice, b->stream));
  TS_CUDA(cudaMemcpyAsync(b->d_unit_off.get(), uo.data(), sizeof(int) * uo.size(), cudaMemcpyHostToDevice, b->stream));
  TS_CUDA(cudaMemcpyAsync(b->d_row_off.get(), ro.data(), sizeof(int) * ro.size(), cudaMemcpyHostToDevice, b->stream));
  TS_CUDA(cudaMemcpyAsync(b->d_chunk_off.get(), co.data(), sizeof(int) * co.size(), cudaMemcpyHostToDevice, b->stream));
  TS_CUDA(cudaStreamSynchronize(b->stream));
  b->dirty = false;
  return TSGNE_OK;
}

tsgne_status refresh(tsgne_batch* b) { return host_guard([&] { return refresh_impl(b); }); }

constexpr int kAuxStreams = 8;

// Streams and events for the tree members' branches (created on first use).
tsgne_status ensure_aux(tsgne_batch* b, int ntree) {
  while ((int)b->aux.size() < std::min(ntree, kAuxStreams)) {
    cudaStream_t st = nullptr;
    TS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    b->aux.push_back(st);
  }
  while ((int)b->ev.size() < ntree + 1) {
    cudaEvent_t e = nullptr;
    TS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    b->ev.push_back(e);
  }
  return TSGNE_OK;
}

tsgne_status enqueue_iteration(tsgne_batch* b) {
  const int G = b->G;
  if (G == 0) return TSGNE_OK;
  const tsgne_config& c = b->cfg;
  // tree members: copy of the current layout, tree build and walk (forces,
  // Z, schedule), each member on a branch forked from the batch stream
  const int ntree = (int)b->trees.size();
  if (ntree > 0) {
    TS_TRY(ensure_aux(b, ntree));
    TS_CUDA(cudaEventRecord(b->ev[0], b->stream));
    for (int k = 0; k < ntree; ++k) {
      Member& m = *b->trees[k];
      cudaStream_t s = b->aux[k % b->aux.size()];
      TS_CUDA(cudaStreamWaitEvent(s, b->ev[0], 0));
      k_member_cur_Y<<<std::max(1, std::min((m.n + 255) / 256, 1024)), 256, 0, s>>>(m.Y[0].get(), m.Y[1].get(),
                                                                                     m.sched.get(), m.n,
                                                                                     m.Ytree.get());
      TS_CUDA(cudaGetLastError());
      TS_TRY(launch_tree_build(m.tb, m.Ytree.get(), s));
      TS_TRY(launch_tree_walk(m.tb, c.theta, m.fsum.get(), m.sched.get(), 1, c.early_exag, c.ee_iters, c.momentum0,
                              c.momentum1, s));
      TS_CUDA(cudaEventRecord(b->ev[1 + k], s));
    }
  }
  const int W = b->W, RI = b->RI;
  const int slots = b->sms * (warps_per_sm(RI) / W);
  const int grid = b->U < slots ? b->U : slots;
  const size_t sm = smem_for(W, RI);
  if (b->U > 0) {
    const GraphDesc* dd = b->d_desc.get();
    const int* uo = b->d_unit_off.get();
    BatchCtr* ctr = b->d_ctr.get();
    if (RI == 16) {
      if (W == 4) k_batch_repulsion<4, 16><<<grid, 128, sm, b->stream>>>(dd, uo, G, b->U, ctr);
      else if (W == 2) k_batch_repulsion<2, 16><<<grid, 64, sm, b->stream>>>(dd, uo, G, b->U, ctr);
      else k_batch_repulsion<1, 16><<<grid, 32, sm, b->stream>>>(dd, uo, G, b->U, ctr);
    } else {
      if (W == 4) k_batch_repulsion<4, 8><<<grid, 128, sm, b->stream>>>(dd, uo, G, b->U, ctr);
      else if (W == 2) k_batch_repulsion<2, 8><<<grid, 64, sm, b->stream>>>(dd, uo, G, b->U, ctr);
      else k_batch_repulsion<1, 8><<<grid, 32, sm, b->stream>>>(dd, uo, G, b->U, ctr);
    }
  }
  // 32 W threads: the same reduction tree as the single-layout pass's last CTA
  k_batch_finalize<<<G, 32 * W, 0, b->stream>>>(b->d_desc.get(), c.early_exag, c.ee_iters, c.momentum0, c.momentum1);
  const int rgrid = std::max(1, std::min((b->R + 255) / 256, b->sms * 16));
  k_batch_reduce<<<rgrid, 256, 0, b->stream>>>(b->d_desc.get(), b->d_row_off.get(), G, b->R);
  for (int k = 0; k < ntree; ++k) TS_CUDA(cudaStreamWaitEvent(b->stream, b->ev[1 + k], 0));  // join
  if (b->C > 0) {
    const int hgrid = std::min((b->C + 7) / 8, 4096);  // one warp per chunk
    k_batch_hubs<<<hgrid, 256, 0, b->stream>>>(b->d_desc.get(), b->d_chunk_off.get(), G, b->C);
  }
  const int64_t threads = (int64_t)b->R * kBG;
  const int agrid = (int)std::max<int64_t>(1, (threads + 255) / 256);
  k_batch_attract<kBG><<<agrid, 256, 0, b->stream>>>(b->d_desc.get(), b->d_row_off.get(), G, b->R, c.min_gain);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

tsgne_status run_iterations(tsgne_batch* b, int n_iter, bool use_graph) {
  TS_TRY(refresh(b));
  if (b->G == 0 || n_iter <= 0) return TSGNE_OK;
  if (use_graph && !b->graph) {
    cudaGraph_t g = nullptr;
    TS_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    tsgne_status st = enqueue_iteration(b);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (st != TSGNE_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
    }
  }
  for (int k = 0; k < n_iter; ++k) {
    if (use_graph) {
      TS_CUDA(cudaGraphLaunch(b->graph, b->stream));
    } else {
      TS_TRY(enqueue_iteration(b));
    }
  }
  return TSGNE_OK;
}

Member* find_member(tsgne_batch* b, int id, size_t* pos = nullptr) {
  for (size_t k = 0; k < b->members.size(); ++k)
    if (b->members[k]->id == id) {
      if (pos) *pos = k;
      return b->members[k].get();
    }
  return nullptr;
}

tsgne_status reset_member_state(Member& m, cudaStream_t s) {
  TS_CUDA(cudaMemcpyAsync(m.Y[0].get(), m.Y0.get(), sizeof(float2) * m.n, cudaMemcpyDeviceToDevice, s));
  TS_TRY(launch_fill2(m.upd.get(), m.n_pad_max, 0.f, s));
  TS_TRY(launch_fill2(m.gains.get(), m.n_pad_max, 1.f, s));
  Sched h{};
  TS_CUDA(cudaMemcpyAsync(m.sched.get(), &h, sizeof(Sched), cudaMemcpyHostToDevice, s));
  return TSGNE_OK;
}

// A member built from its inputs on stream s: structure, P, hub rows, its
// layout buffers and state (and its tree, repulsion = 1); everything but the
// per-tile scratch, which depends on the batch's tile (attach_member).
// Touches no batch state, so it may run on another thread while the batch
// runs.  Synchronises s.
tsgne_status prepare_member(const tsgne_config& cfg, int sms, int32_t n, const int64_t* row_ptr,
                            const int32_t* col_idx, const float* X, int32_t d, const float* Y0, int32_t ptr_kind,
                            int32_t repulsion, cudaStream_t s, std::unique_ptr<Member>& out) {
  auto fail_ = [](tsgne_status st, const char* m) {
    last_msg() = m;
    return st;
  };
  if (!(repulsion == 0 || repulsion == 1)) return fail_(TSGNE_ERR_INVALID_ARG, "repulsion must be 0 or 1");
  if (n < 2 || d < 1 || !row_ptr || !X || !(ptr_kind == TSGNE_PTR_HOST || ptr_kind == TSGNE_PTR_DEVICE))
    return fail_(TSGNE_ERR_INVALID_ARG, "need n >= 2, d >= 1, row_ptr, X and a valid ptr_kind");
  if (repulsion == 0 && n > kMaxExactPoints)
    return fail_(TSGNE_ERR_INVALID_ARG, "an exact member takes at most 2^24 - 2048 points (repulsion = 1: the tree code)");
  if (repulsion == 1 && n >= (1 << 30)) return fail_(TSGNE_ERR_INVALID_ARG, "the tree code takes fewer than 2^30 points");
  const cudaMemcpyKind kin = ptr_kind == TSGNE_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  int64_t first = 0, m = 0;
  if (ptr_kind == TSGNE_PTR_HOST) {
    first = row_ptr[0];
    m = row_ptr[n];
  } else {
    TS_CUDA(cudaMemcpyAsync(&first, row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaMemcpyAsync(&m, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TS_CUDA(cudaStreamSynchronize(s));
  }
  if (first != 0 || m < 0) return fail_(TSGNE_ERR_BAD_CSR, "row_ptr[0] must be 0 and row_ptr[n] >= 0");
  if (m > 0 && !col_idx) return fail_(TSGNE_ERR_INVALID_ARG, "col_idx is NULL");
  auto mem = std::make_unique<Member>();
  Member& mb = *mem;
  mb.n = n;
  DevBuf<int64_t> rp_in, tslot;
  DevBuf<int32_t> col_in;
  DevBuf<float> X_in;
  TS_TRY(rp_in.alloc((size_t)n + 1));
  TS_TRY(col_in.alloc((size_t)m));
  TS_TRY(X_in.alloc((size_t)n * d));
  TS_CUDA(cudaMemcpyAsync(rp_in.get(), row_ptr, sizeof(int64_t) * ((size_t)n + 1), kin, s));
  if (m > 0) TS_CUDA(cudaMemcpyAsync(col_in.get(), col_idx, sizeof(int32_t) * (size_t)m, kin, s));
  TS_CUDA(cudaMemcpyAsync(X_in.get(), X, sizeof(float) * (size_t)n * d, kin, s));
  TS_TRY(mb.sched.alloc(1));
  TS_CUDA(cudaMemsetAsync(mb.sched.get(), 0, sizeof(Sched), s));
  TS_TRY(build_neighbor_structure(n, rp_in.get(), col_in.get(), m, cfg.k_nn, mb.rp, mb.col, tslot, &mb.nnz,
                                    s));
  TS_TRY(find_heavy_rows(n, mb.rp.get(), mb.hv, s));
  TS_TRY(mb.P.alloc((size_t)mb.nnz));
  TS_TRY(build_affinities(n, mb.rp.get(), mb.col.get(), tslot.get(), mb.nnz, X_in.get(), d, cfg.perplexity,
                            cfg.bisect_tol, cfg.bisect_max_iter, mb.P.get(), mb.sched.get(), s));
  Sched hs;
  TS_CUDA(cudaMemcpyAsync(&hs, mb.sched.get(), sizeof(Sched), cudaMemcpyDeviceToHost, s));
  TS_CUDA(cudaStreamSynchronize(s));
  if (hs.flags & kFlagNonfiniteP) return fail_(TSGNE_ERR_NONFINITE, "non-finite affinity (check X)");
  mb.n_pad_max = ((n + kMaxT - 1) / kMaxT) * kMaxT;
  const size_t np = (size_t)mb.n_pad_max;
  TS_TRY(mb.Y[0].alloc(np));
  TS_TRY(mb.Y[1].alloc(np));
  TS_TRY(mb.upd.alloc(np));
  TS_TRY(mb.gains.alloc(np));
  TS_TRY(mb.fsum.alloc(np));
  TS_TRY(mb.acc.alloc(2 * (size_t)n));
  TS_CUDA(cudaMemsetAsync(mb.acc.get(), 0, 2 * (size_t)n * sizeof(unsigned long long), s));
  TS_TRY(mb.Y0.alloc((size_t)n));
  TS_TRY(launch_fill_sentinel(mb.Y[0].get(), 0, (int)np, s));
  TS_TRY(launch_fill_sentinel(mb.Y[1].get(), 0, (int)np, s));
  if (Y0) {
    TS_CUDA(cudaMemcpyAsync(mb.Y0.get(), Y0, sizeof(float2) * (size_t)n, kin, s));
  } else {
    TS_TRY(launch_init_Y(n, cfg.seed, 1e-4f, mb.Y0.get(), s));
  }
  mb.tree = repulsion == 1;
  if (mb.tree) {
    TS_TRY(mb.tb.alloc(n, sms, s));
    mb.tb.spin_budget = cfg.spin_budget_cycles;
    TS_TRY(mb.Ytree.alloc((size_t)n));
  }
  TS_TRY(reset_member_state(mb, s));
  const float ee = cfg.early_exag > 0.f ? cfg.early_exag : 1.f;
  mb.eta = cfg.learning_rate > 0.f ? cfg.learning_rate : std::fmax((float)n / ee / 4.0f, 50.0f);
  TS_CUDA(cudaStreamSynchronize(s));
  out = std::move(mem);
  return TSGNE_OK;
}

// Adds a prepared member to the batch (its per-tile scratch for the current
// tile); the membership changes at the next run.
tsgne_status attach_member(tsgne_batch* b, std::unique_ptr<Member> mem, int32_t* id_out) {
  TS_TRY(alloc_scratch(*mem, b->W, b->RI));
  mem->id = b->next_id++;
  if (id_out) *id_out = mem->id;
  b->members.push_back(std::move(mem));
  invalidate(b);
  return TSGNE_OK;
}


bool capturable_stream(cudaStream_t s) { return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread; }

}  // namespace

extern "C" {

tsgne_status tsgne_batch_create(tsgne_batch** out, const tsgne_config* cfg, int32_t tile_warps, void* cuda_stream) {
  if (!out) return TSGNE_ERR_INVALID_ARG;
  *out = nullptr;
  tsgne_config c;
  if (cfg) c = *cfg; else tsgne_config_default(&c);
  if (!(c.perplexity > 1.f) || c.k_nn < 0 || c.k_nn > 256 || c.precision != 0 || c.ee_iters < 0 ||
      !(c.repulsion == 0 || c.repulsion == 1) || !(c.theta >= 0.f && c.theta <= 1.f) || c.spin_budget_cycles < 1)
    return TSGNE_ERR_INVALID_ARG;
  if (!(tile_warps == 0 || tile_warps == 1 || tile_warps == 2 || tile_warps == 4))
    return TSGNE_ERR_INVALID_ARG;
  tsgne_batch* b = new (std::nothrow) tsgne_batch();
  if (!b) return TSGNE_ERR_OOM;
  b->cfg = c;
  b->W = tile_warps ? tile_warps : 1;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess) {
    if (cuda_stream) {
      b->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
      e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
      b->own_stream = (e == cudaSuccess);
    }
  }
  tsgne_status st = e == cudaSuccess ? TSGNE_OK : cuda_fail(e, "tsgne_batch_create", __FILE__, __LINE__);
  if (st == TSGNE_OK) st = b->d_ctr.alloc(1);
  if (st == TSGNE_OK && cudaMemsetAsync(b->d_ctr.get(), 0, sizeof(BatchCtr), b->stream) != cudaSuccess)
    st = TSGNE_ERR_CUDA;
  for (const auto& sh : kShapes)
    if (st == TSGNE_OK) st = prepare_w(sh[0], sh[1]);
  if (st == TSGNE_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) st = TSGNE_ERR_CUDA;
  if (st != TSGNE_OK) {
    delete b;
    return st;
  }
  *out = b;
  return TSGNE_OK;
}

void tsgne_batch_destroy(tsgne_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  delete b;
}

const char* tsgne_batch_last_error(const tsgne_batch* b) { return b ? b->err.c_str() : ""; }

tsgne_status tsgne_batch_add(tsgne_batch* b, int32_t n, const int64_t* row_ptr, const int32_t* col_idx, const float* X,
                             int32_t d, const float* Y0, int32_t ptr_kind, int32_t* id_out) {
  if (!b) return TSGNE_ERR_INVALID_ARG;
  return tsgne_batch_add_ex(b, n, row_ptr, col_idx, X, d, Y0, ptr_kind, b->cfg.repulsion, id_out);
}

tsgne_status tsgne_batch_add_ex(tsgne_batch* b, int32_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                const float* X, int32_t d, const float* Y0, int32_t ptr_kind, int32_t repulsion,
                                int32_t* id_out) {
  if (!b) return TSGNE_ERR_INVALID_ARG;
  b->err.clear();
  last_msg().clear();
  std::unique_ptr<Member> mem;
  B_TRY(b, host_guard([&] {
          return prepare_member(b->cfg, b->sms, n, row_ptr, col_idx, X, d, Y0, ptr_kind, repulsion, b->stream, mem);
        }));
  B_TRY(b, attach_member(b, std::move(mem), id_out));
  return TSGNE_OK;
}

tsgne_status tsgne_batch_prepare(tsgne_batch* b, int32_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                 const float* X, int32_t d, const float* Y0, int32_t ptr_kind, int32_t repulsion,
                                 void* cuda_stream, tsgne_member** out) {
  if (!b || !out || !cuda_stream) return TSGNE_ERR_INVALID_ARG;
  *out = nullptr;
  last_msg().clear();
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  TS_CUDA(cudaGetDevice(&dev));
  if (dev != b->device) TS_CUDA(cudaSetDevice(b->device));
  cudaStream_t& as = alloc_stream();
  const cudaStream_t saved = as;
  as = s;  // stream-ordered allocations: no device-wide wait in cudaFree
  std::unique_ptr<Member> mem;
  const tsgne_status st = host_guard(
      [&] { return prepare_member(b->cfg, b->sms, n, row_ptr, col_idx, X, d, Y0, ptr_kind, repulsion, s, mem); });
  as = saved;
  if (st != TSGNE_OK) return st;
  tsgne_member* h = new (std::nothrow) tsgne_member();
  if (!h) return TSGNE_ERR_OOM;
  h->m = std::move(mem);
  *out = h;
  return TSGNE_OK;
}

tsgne_status tsgne_batch_attach(tsgne_batch* b, tsgne_member* m, int32_t* id_out) {
  if (!b || !m || !m->m) return TSGNE_ERR_INVALID_ARG;
  b->err.clear();
  last_msg().clear();
  B_TRY(b, attach_member(b, std::move(m->m), id_out));
  delete m;
  return TSGNE_OK;
}

void tsgne_batch_discard(tsgne_member* m) { delete m; }

tsgne_status tsgne_batch_remove(tsgne_batch* b, int32_t id) {
  if (!b) return TSGNE_ERR_INVALID_ARG;
  b->err.clear();
  size_t pos = 0;
  if (!find_member(b, id, &pos)) return bfail(b, TSGNE_ERR_INVALID_ARG, "unknown member id");
  B_CUDA(b, cudaStreamSynchronize(b->stream));
  b->members.erase(b->members.begin() + (long)pos);
  invalidate(b);
  return TSGNE_OK;
}

tsgne_status tsgne_batch_size(tsgne_batch* b, int32_t* members, int32_t* tile_warps, int64_t* units) {
  if (!b) return TSGNE_ERR_INVALID_ARG;
  B_TRY(b, refresh(b));
  if (members) *members = (int32_t)b->members.size();
  if (tile_warps) *tile_warps = b->W;
  if (units) *units = b->U;
  return TSGNE_OK;
}

tsgne_status tsgne_batch_run(tsgne_batch* b, int32_t n_iter) {
  if (!b) return TSGNE_ERR_INVALID_ARG;
  b->err.clear();
  if (n_iter < 0) return bfail(b, TSGNE_ERR_INVALID_ARG, "n_iter < 0");
  B_TRY(b, run_iterations(b, n_iter, capturable_stream(b->stream)));
  B_CUDA(b, cudaStreamSynchronize(b->stream));
  for (auto& m : b->members) {
    Sched h;
    B_CUDA(b, cudaMemcpyAsync(&h, m->sched.get(), sizeof(Sched), cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    if (h.flags & kFlagNonfiniteY) return bfail(b, TSGNE_ERR_NONFINITE, "a member's layout became non-finite");
  }
  return TSGNE_OK;
}

tsgne_status tsgne_batch_get_Y(tsgne_batch* b, int32_t id, float* Y_out, int32_t* iter, int32_t ptr_kind) {
  if (!b || !Y_out) return TSGNE_ERR_INVALID_ARG;
  b->err.clear();
  Member* m = find_member(b, id);
  if (!m) return bfail(b, TSGNE_ERR_INVALID_ARG, "unknown member id");
  Sched h;
  B_CUDA(b, cudaMemcpyAsync(&h, m->sched.get(), sizeof(Sched), cudaMemcpyDeviceToHost, b->stream));
  B_CUDA(b, cudaStreamSynchronize(b->stream));
  B_CUDA(b, cudaMemcpyAsync(Y_out, m->Y[h.t & 1].get(), sizeof(float2) * (size_t)m->n,
                            ptr_kind == TSGNE_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, b->stream));
  B_CUDA(b, cudaStreamSynchronize(b->stream));
  if (iter) *iter = h.t;
  return TSGNE_OK;
}

tsgne_status tsgne_batch_set_active(tsgne_batch* b, int32_t id, int32_t active) {
  if (!b) return TSGNE_ERR_INVALID_ARG;
  b->err.clear();
  Member* m = find_member(b, id);
  if (!m) return bfail(b, TSGNE_ERR_INVALID_ARG, "unknown member id");
  if (m->active != (active != 0)) {
    m->active = active != 0;
    invalidate(b);
  }
  return TSGNE_OK;
}

tsgne_status tsgne_batch_set_shape(tsgne_batch* b, int32_t tile_warps, int32_t i_per_lane) {
  if (!b) return TSGNE_ERR_INVALID_ARG;
  if (!(tile_warps == 1 || tile_warps == 2 || tile_warps == 4) || !(i_per_lane == 8 || i_per_lane == 16))
    return bfail(b, TSGNE_ERR_INVALID_ARG, "tile_warps must be 1, 2 or 4 and i_per_lane 8 or 16");
  if (tile_warps == b->W && i_per_lane == b->RI) return TSGNE_OK;
  B_CUDA(b, cudaStreamSynchronize(b->stream));
  for (auto& m : b->members) B_TRY(b, alloc_scratch(*m, tile_warps, i_per_lane));
  b->W = tile_warps;
  b->RI = i_per_lane;
  invalidate(b);
  return TSGNE_OK;
}

tsgne_status tsgne_batch_set_tile(tsgne_batch* b, int32_t tile_warps) {
  if (!b) return TSGNE_ERR_INVALID_ARG;
  return tsgne_batch_set_shape(b, tile_warps, b->RI);
}

tsgne_status tsgne_batch_shape(tsgne_batch* b, int32_t* tile_warps, int32_t* i_per_lane) {
  if (!b) return TSGNE_ERR_INVALID_ARG;
  if (tile_warps) *tile_warps = b->W;
  if (i_per_lane) *i_per_lane = b->RI;
  return TSGNE_OK;
}

tsgne_status tsgne_batch_reset(tsgne_batch* b) {
  if (!b) return TSGNE_ERR_INVALID_ARG;
  for (auto& m : b->members) B_TRY(b, reset_member_state(*m, b->stream));
  B_CUDA(b, cudaStreamSynchronize(b->stream));
  return TSGNE_OK;
}

namespace {
// Times trial_iters iterations of each candidate shape from the members'
// initial state, keeps the fastest (the members are reset to their initial
// state afterwards) and caches it per (SM count, log2 pairs, log2 members).
tsgne_status autotune(tsgne_batch* b, int32_t trial_iters, const int (*cand)[2], int ncand, float* ms_out,
                      int* best_w, int* best_ri) {
  TS_TRY(refresh(b));
  double pairs = 0.0;
  for (auto& m : b->members) pairs += 0.5 * (double)m->n * (double)m->n;
  const auto key = std::make_tuple(b->sms, (int)std::log2(pairs + 1.0), (int)std::log2((double)b->members.size() + 1.0));
  int bw = -1, bri = -1;
  float best_ms = 0.f;
  cudaEvent_t e0, e1;
  TS_CUDA(cudaEventCreate(&e0));
  TS_CUDA(cudaEventCreate(&e1));
  tsgne_status st = TSGNE_OK;
  for (int k = 0; k < ncand && st == TSGNE_OK; ++k) {
    st = tsgne_batch_set_shape(b, cand[k][0], cand[k][1]);
    if (st == TSGNE_OK) st = run_iterations(b, 1, false);  // warm-up
    if (st == TSGNE_OK) st = cudaEventRecord(e0, b->stream) == cudaSuccess ? TSGNE_OK : TSGNE_ERR_CUDA;
    if (st == TSGNE_OK) st = run_iterations(b, trial_iters, false);
    if (st == TSGNE_OK) st = cudaEventRecord(e1, b->stream) == cudaSuccess ? TSGNE_OK : TSGNE_ERR_CUDA;
    if (st == TSGNE_OK) st = cudaEventSynchronize(e1) == cudaSuccess ? TSGNE_OK : TSGNE_ERR_CUDA;
    float ms = 0.f;
    if (st == TSGNE_OK) st = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess ? TSGNE_OK : TSGNE_ERR_CUDA;
    if (st != TSGNE_OK) break;
    ms /= (float)trial_iters;
    if (ms_out) ms_out[k] = ms;
    if (bw < 0 || ms < best_ms) {
      bw = cand[k][0];
      bri = cand[k][1];
      best_ms = ms;
    }
    st = tsgne_batch_reset(b);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TS_TRY(st);
  TS_TRY(tsgne_batch_set_shape(b, bw, bri));
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_tile_cache[key] = 100 * bw + bri;
  }
  *best_w = bw;
  *best_ri = bri;
  return TSGNE_OK;
}
}  // namespace

tsgne_status tsgne_batch_autotune(tsgne_batch* b, int32_t trial_iters, int32_t* chosen, float* ms_per_iter) {
  if (!b || trial_iters < 1) return TSGNE_ERR_INVALID_ARG;
  b->err.clear();
  const int cand[3][2] = {{1, 16}, {2, 16}, {4, 16}};
  int w = 0, ri = 0;
  B_TRY(b, autotune(b, trial_iters, cand, 3, ms_per_iter, &w, &ri));
  if (chosen) *chosen = w;
  return TSGNE_OK;
}

tsgne_status tsgne_batch_autotune_shapes(tsgne_batch* b, int32_t trial_iters, int32_t* tile_warps,
                                         int32_t* i_per_lane, float* ms_per_iter) {
  if (!b || trial_iters < 1) return TSGNE_ERR_INVALID_ARG;
  b->err.clear();
  int w = 0, ri = 0;
  B_TRY(b, autotune(b, trial_iters, kShapes, 6, ms_per_iter, &w, &ri));
  if (tile_warps) *tile_warps = w;
  if (i_per_lane) *i_per_lane = ri;
  return TSGNE_OK;
}

tsgne_status tsgne_batch_cached_tile(tsgne_batch* b, int32_t* tile_warps) {
  if (!b || !tile_warps) return TSGNE_ERR_INVALID_ARG;
  double pairs = 0.0;
  for (auto& m : b->members) pairs += 0.5 * (double)m->n * (double)m->n;
  const auto key = std::make_tuple(b->sms, (int)std::log2(pairs + 1.0), (int)std::log2((double)b->members.size() + 1.0));
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto it = g_tile_cache.find(key);
  *tile_warps = it == g_tile_cache.end() ? 0 : it->second / 100;
  return TSGNE_OK;
}

}  // extern "C"
