// C ABI of libtsgne.so (declared in include/tsgne.h): context ownership,
// argument validation, host/device copies, CUDA-graph replay of iterations
// and per-kernel CUDA-event profiling.  All arithmetic runs in the kernels of
// structure.cu, affinity.cu, repulsion.cu and iterate.cu.
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <cstddef>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "storage.cuh"
#include "tsgne_internal.cuh"

namespace tsgne {

std::string& last_msg() {
  thread_local std::string m;
  return m;
}

cudaStream_t& alloc_stream() {
  thread_local cudaStream_t s = nullptr;
  return s;
}

namespace {
std::atomic<int64_t> g_dev_bytes{0};
std::atomic<int64_t> g_dev_limit{0};  // 0: no limit
}  // namespace

bool device_bytes_reserve(size_t bytes) {
  const int64_t b = (int64_t)bytes;
  const int64_t lim = g_dev_limit.load();
  int64_t cur = g_dev_bytes.load();
  do {
    if (lim > 0 && cur + b > lim) return false;
  } while (!g_dev_bytes.compare_exchange_weak(cur, cur + b));
  return true;
}

void device_bytes_release(size_t bytes) { g_dev_bytes.fetch_sub((int64_t)bytes); }

tsgne_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  std::string s = std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" + std::to_string(line) + ")";
  last_msg() = s;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // not sticky: clear it
    return TSGNE_ERR_OOM;
  }
  return TSGNE_ERR_CUDA;
}

namespace {

__global__ void k_cmp_i64(const int64_t* a, const int64_t* b, int64_t n, uint32_t* neq) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    if (a[k] != b[k]) atomicOr(neq, 1u);
}
__global__ void k_cmp_i32(const int32_t* a, const int32_t* b, int64_t n, uint32_t* neq) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    if (a[k] != b[k]) atomicOr(neq, 1u);
}

constexpr int kClasses = 8;  // repulsion, attraction+update, gradient, KL, build, force conversion, hub rows, tree build

struct ProfRec {
  int cls;
  cudaEvent_t a, b;
};

}  // namespace
}  // namespace tsgne

using namespace tsgne;

struct tsgne_ctx {
  tsgne_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  int sms = 1;
  std::string err;

  int n = 0;
  int64_t nnz = 0;
  bool have_P = false;
  bool have_Y = false;
  bool poisoned = false;
  float eta = 0.f;
  RepShape shape;

  DevBuf<int64_t> rp;
  DevBuf<int32_t> col;
  DevBuf<float> P;
  DevBuf<float2> Y[2];
  int cur = 0;
  DevBuf<float2> upd, gains, fsum, grad;
  DevBuf<unsigned long long> facc;  // exact repulsion: fixed-point force accumulators (2 per point)
  // BF16 storage (cfg.precision = 1): P and a shadow of the layout, read by
  // every force kernel; the FP32 master layout is what the update advances
  bool bf16 = false;
  DevBuf<tsgne::bf16> P16;
  DevBuf<tsgne::bf162> Y16[2];
  const void* Pread() const { return bf16 ? (const void*)P16.get() : (const void*)P.get(); }
  const void* Yread(int k) const { return bf16 ? (const void*)Y16[k].get() : (const void*)Y[k].get(); }
  // tree-code repulsion (cfg.repulsion = 1): reads the FP32 master layout
  bool use_tree = false;
  TreeBufs tree;
  HeavyStore hub;
  HeavyRows heavy() const { return hub.view(); }
  AttractPlan plan;  // schedule of the attraction + update pass (fixed with P)
  DevBuf<double> zpart, klpart;
  DevBuf<Sched> sched;
  // sharding of the exact repulsion over several contexts (tsgne_shard_*):
  // this context evaluates tile-pair units [shard_u0, shard_u1)
  // shape of the exact pass: symmetric (shape) or the ordered-pair kernel
  // (oshape, its per-chunk partial forces in oslots); tsgne_autotune picks
  bool ordered = false;
  RepShape oshape;
  DevBuf<float2> oslots;
  int n_pad_alloc = 0;
  int shard_rank = 0, shard_world = 1;
  int shard_u0 = 0, shard_u1 = 0;
  bool shard_pending = false;  // a share was enqueued and awaits its finish call

  cudaGraphExec_t g2[2] = {nullptr, nullptr};  // two iterations starting from buffer 0 / 1

  std::vector<ProfRec> pending;
  std::vector<cudaEvent_t> spare;
  double prof_ms[kClasses] = {0, 0, 0, 0, 0, 0, 0, 0};
  int64_t prof_n[kClasses] = {0, 0, 0, 0, 0, 0, 0, 0};

  ~tsgne_ctx() {
    reset_graphs();
    for (auto& r : pending) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : spare) cudaEventDestroy(e);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
  void reset_graphs() {
    for (auto& g : g2)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
  }
};

namespace {

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int now = -1;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
  }
};

tsgne_status fail(tsgne_ctx* ctx, tsgne_status st, const std::string& msg = std::string()) {
  if (ctx) {
    ctx->err = msg.empty() ? last_msg() : msg;
    if (st == TSGNE_ERR_CUDA) ctx->poisoned = true;
  }
  return st;
}

#define API_TRY(ctx, call)                        \
  do {                                            \
    tsgne_status s__ = (call);                    \
    if (s__ != TSGNE_OK) return fail((ctx), s__); \
  } while (0)

#define API_CUDA(ctx, call)                                                          \
  do {                                                                               \
    cudaError_t e__ = (call);                                                        \
    if (e__ != cudaSuccess) return fail((ctx), cuda_fail(e__, #call, __FILE__, __LINE__)); \
  } while (0)

tsgne_status enter(tsgne_ctx* ctx) {
  if (!ctx) return TSGNE_ERR_INVALID_ARG;
  ctx->err.clear();
  last_msg().clear();
  if (ctx->poisoned) return fail(ctx, TSGNE_ERR_CUDA, "context is unusable after an earlier CUDA error");
  return TSGNE_OK;
}

// Copies count elements from src (host or device) into a new device buffer.
template <class T>
tsgne_status to_device(const T* src, size_t count, int ptr_kind, DevBuf<T>& dst, cudaStream_t s) {
  TS_TRY(dst.alloc(count));
  if (count == 0) return TSGNE_OK;
  TS_CUDA(cudaMemcpyAsync(dst.get(), src, count * sizeof(T),
                          ptr_kind == TSGNE_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  return TSGNE_OK;
}

tsgne_status copy_out(void* dst, const void* src, size_t bytes, int ptr_kind, cudaStream_t s) {
  if (bytes == 0) return TSGNE_OK;
  TS_CUDA(cudaMemcpyAsync(dst, src, bytes, ptr_kind == TSGNE_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                          s));
  return TSGNE_OK;
}

tsgne_status copy_in(void* dst, const void* src, size_t bytes, int ptr_kind, cudaStream_t s) {
  if (bytes == 0) return TSGNE_OK;
  TS_CUDA(cudaMemcpyAsync(dst, src, bytes, ptr_kind == TSGNE_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                          s));
  return TSGNE_OK;
}

bool valid_kind(int k) { return k == TSGNE_PTR_HOST || k == TSGNE_PTR_DEVICE; }

// ---------------------------------------------------------------- profiling

tsgne_status prof_begin(tsgne_ctx* ctx, int cls, ProfRec* rec) {
  rec->cls = cls;
  rec->a = rec->b = nullptr;
  if (!ctx->cfg.profile) return TSGNE_OK;
  for (cudaEvent_t* e : {&rec->a, &rec->b}) {
    if (!ctx->spare.empty()) {
      *e = ctx->spare.back();
      ctx->spare.pop_back();
    } else {
      TS_CUDA(cudaEventCreate(e));
    }
  }
  TS_CUDA(cudaEventRecord(rec->a, ctx->stream));
  return TSGNE_OK;
}

tsgne_status prof_collect(tsgne_ctx* ctx) {
  if (ctx->pending.empty()) return TSGNE_OK;
  TS_CUDA(cudaStreamSynchronize(ctx->stream));
  for (auto& r : ctx->pending) {
    float ms = 0.f;
    TS_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    ctx->prof_ms[r.cls] += ms;
    ctx->prof_n[r.cls] += 1;
    ctx->spare.push_back(r.a);
    ctx->spare.push_back(r.b);
  }
  ctx->pending.clear();
  return TSGNE_OK;
}

tsgne_status prof_end(tsgne_ctx* ctx, ProfRec* rec) {
  if (!ctx->cfg.profile) return TSGNE_OK;
  TS_CUDA(cudaEventRecord(rec->b, ctx->stream));
  ctx->pending.push_back(*rec);
  if (ctx->pending.size() >= 8192) TS_TRY(prof_collect(ctx));
  return TSGNE_OK;
}

// ------------------------------------------------------------- iteration

tsgne_status enqueue_repulsion(tsgne_ctx* ctx, int advance) {
  const tsgne_config& c = ctx->cfg;
  ProfRec pr;
  if (ctx->use_tree) {
    ProfRec pb;
    TS_TRY(prof_begin(ctx, 7, &pb));
    TS_TRY(launch_tree_build(ctx->tree, ctx->Y[ctx->cur].get(), ctx->stream));
    TS_TRY(prof_end(ctx, &pb));
    TS_TRY(prof_begin(ctx, 0, &pr));
    TS_TRY(launch_tree_walk(ctx->tree, c.theta, ctx->fsum.get(), ctx->sched.get(), advance, c.early_exag,
                            c.ee_iters, c.momentum0, c.momentum1, ctx->stream));
    return prof_end(ctx, &pr);
  }
  TS_TRY(prof_begin(ctx, 0, &pr));
  if (ctx->ordered) {  // every ordered pair, partial forces per j-chunk
    TS_TRY(launch_repulsion(ctx->oshape, ctx->n, ctx->Y[ctx->cur].get(), ctx->oslots.get(), ctx->zpart.get(),
                            ctx->sched.get(), advance, c.early_exag, c.ee_iters, c.momentum0, c.momentum1,
                            ctx->stream));
    TS_TRY(prof_end(ctx, &pr));
    ProfRec pr2;
    TS_TRY(prof_begin(ctx, 5, &pr2));
    TS_TRY(launch_reduce_slots(ctx->n, ctx->oslots.get(), ctx->oshape.chunks, ctx->oshape.n_pad, ctx->fsum.get(),
                               ctx->stream));
    return prof_end(ctx, &pr2);
  }
  TS_TRY(launch_repulsion_sym(ctx->shape, ctx->n, ctx->Yread(ctx->cur), ctx->bf16 ? 1 : 0, ctx->facc.get(),
                              ctx->zpart.get(), ctx->sched.get(), advance, c.early_exag, c.ee_iters, c.momentum0,
                              c.momentum1, ctx->stream));
  TS_TRY(prof_end(ctx, &pr));
  ProfRec pr2;
  TS_TRY(prof_begin(ctx, 5, &pr2));
  TS_TRY(launch_fix_forces(ctx->n, ctx->facc.get(), ctx->fsum.get(), ctx->stream));
  return prof_end(ctx, &pr2);
}

// Reads of the current layout / P for the force kernels of the context.
AttractArgs attract_args(tsgne_ctx* ctx) {
  AttractArgs a;
  a.n = ctx->n;
  a.rp = ctx->rp.get();
  a.col = ctx->col.get();
  a.P = ctx->Pread();
  a.p_bf16 = ctx->bf16 ? 1 : 0;
  a.Yr = ctx->Yread(ctx->cur);
  a.y_bf16 = ctx->bf16 ? 1 : 0;
  a.Ym = ctx->Y[ctx->cur].get();
  a.frep = ctx->fsum.get();
  a.chunks = 1;
  a.n_pad = ctx->shape.n_pad;
  a.sched = ctx->sched.get();
  a.hv = ctx->heavy();
  return a;
}

// Refreshes the BF16 shadow of Y[k] (all n_pad points, sentinels included).
tsgne_status sync_shadow(tsgne_ctx* ctx, int k) {
  if (!ctx->bf16) return TSGNE_OK;
  return launch_to_bf16(reinterpret_cast<const float*>(ctx->Y[k].get()), ctx->Y16[k].get(),
                        2 * (int64_t)ctx->n_pad_alloc, ctx->stream);
}

// Attraction + update of every row from the forces of the last repulsion
// pass, into the other layout buffer.
tsgne_status enqueue_update(tsgne_ctx* ctx) {
  ProfRec pr;
  // the layout is pulled into L2 before the gathers
  const int nxt = ctx->cur ^ 1;
  AttractArgs a = attract_args(ctx);
  a.Ynext = ctx->Y[nxt].get();
  a.Ynext16 = ctx->bf16 ? (void*)ctx->Y16[nxt].get() : nullptr;
  a.upd = ctx->upd.get();
  a.gains = ctx->gains.get();
  a.eta = ctx->eta;
  a.min_gain = ctx->cfg.min_gain;
  const int64_t ybytes = (int64_t)ctx->n * (ctx->bf16 ? 4 : 8);
  TS_TRY(prof_begin(ctx, 1, &pr));
  TS_TRY(launch_prefetch_l2(a.Yr, ybytes, ctx->stream));
  TS_TRY(launch_attract_plan(a, ctx->plan.view(), ctx->stream));  // hub-row chunks included (one launch)
  TS_TRY(prof_end(ctx, &pr));
  ctx->cur = nxt;
  return TSGNE_OK;
}

tsgne_status enqueue_step(tsgne_ctx* ctx) {
  TS_TRY(enqueue_repulsion(ctx, 1));
  return enqueue_update(ctx);
}

tsgne_status read_sched(tsgne_ctx* ctx, Sched* h) {
  TS_CUDA(cudaMemcpyAsync(h, ctx->sched.get(), sizeof(Sched), cudaMemcpyDeviceToHost, ctx->stream));
  TS_CUDA(cudaStreamSynchronize(ctx->stream));
  return TSGNE_OK;
}

// Errors of the tree code's passes (stack overflow, a sort wait that ran out)
// in a status word already read into h.
tsgne_status check_tree_flags(tsgne_ctx* ctx, const Sched& h) {
  if (h.flags & kFlagIndexCheck) {  // debug build only; reported once
    const uint32_t rest = h.flags & ~kFlagIndexCheck;
    TS_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(ctx->sched.get()) + offsetof(Sched, flags), &rest,
                            sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream));
    TS_CUDA(cudaStreamSynchronize(ctx->stream));
    last_msg() = "an index check of the debug build failed and its access was skipped; the pass is not valid";
    return TSGNE_ERR_INDEX;
  }
  if (h.flags & kFlagTreeOverflow) {
    last_msg() = "tree walk stack overflow (results of the pass are incomplete)";
    return TSGNE_ERR_CUDA;
  }
  if (h.flags & kFlagWaitTimeout) {
    // reported once: the next pass rebuilds the tree from scratch
    const uint32_t rest = h.flags & ~kFlagWaitTimeout;
    TS_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(ctx->sched.get()) + offsetof(Sched, flags), &rest,
                            sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream));
    TS_CUDA(cudaStreamSynchronize(ctx->stream));
    last_msg() = "a device-side wait ran out of spin_budget_cycles (tree sort); the pass's forces are zero";
    return TSGNE_ERR_TIMEOUT;
  }
  return TSGNE_OK;
}

tsgne_status check_flags(tsgne_ctx* ctx) {
  Sched h;
  TS_TRY(read_sched(ctx, &h));
  if (h.flags & kFlagNonfiniteY) {
    last_msg() = "the layout became non-finite";
    return TSGNE_ERR_NONFINITE;
  }
  TS_TRY(check_tree_flags(ctx, h));
  return TSGNE_OK;
}

bool capturable(cudaStream_t s) { return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread; }

tsgne_status ensure_graph(tsgne_ctx* ctx, int start) {
  if (ctx->g2[start]) return TSGNE_OK;
  const int saved = ctx->cur;
  ctx->cur = start;
  cudaGraph_t g = nullptr;
  TS_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  tsgne_status st = enqueue_step(ctx);
  if (st == TSGNE_OK) st = enqueue_step(ctx);
  cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
  ctx->cur = saved;
  if (st != TSGNE_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  e = cudaGraphInstantiate(&ctx->g2[start], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    ctx->g2[start] = nullptr;
    return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
  }
  return TSGNE_OK;
}

// Allocates the per-layout buffers for n points (after P is known).
tsgne_status alloc_layout(tsgne_ctx* ctx) {
  if (ctx->cfg.repulsion == 0 && ctx->n > kMaxExactPoints) {
    last_msg() = "the exact repulsion takes at most 2^24 - 2048 points (cfg.repulsion = 1: the tree code)";
    return TSGNE_ERR_INVALID_ARG;
  }
  ctx->shape = repulsion_shape_sym(ctx->n, ctx->sms);
  ctx->ordered = false;
  TS_TRY(repulsion_sym_prepare(ctx->shape));
  // padded for every shape of the exact pass (tiles of 256 ... 2048 points)
  const size_t np = (size_t)((ctx->n + 2047) / 2048) * 2048;
  ctx->n_pad_alloc = (int)np;
  TS_TRY(ctx->Y[0].alloc(np));
  TS_TRY(ctx->Y[1].alloc(np));
  TS_TRY(ctx->upd.alloc(np));
  TS_TRY(ctx->gains.alloc(np));
  TS_TRY(ctx->grad.alloc(np));
  TS_TRY(ctx->fsum.alloc(np));
  ctx->use_tree = ctx->cfg.repulsion == 1;
  if (ctx->use_tree) {
    ctx->facc = DevBuf<unsigned long long>();
    ctx->zpart = DevBuf<double>();
    TS_TRY(ctx->tree.alloc(ctx->n, ctx->sms, ctx->stream));
    ctx->tree.spin_budget = ctx->cfg.spin_budget_cycles;
  } else {
    ctx->tree = TreeBufs();
    TS_TRY(ctx->facc.alloc(2 * np));
    TS_CUDA(cudaMemsetAsync(ctx->facc.get(), 0, 2 * np * sizeof(unsigned long long), ctx->stream));
    TS_TRY(ctx->zpart.alloc((size_t)ctx->shape.units));
  }
  TS_TRY(ctx->klpart.alloc(2 * (size_t)kl_partial_count(ctx->sms)));
  TS_TRY(launch_fill_sentinel(ctx->Y[0].get(), 0, (int)np, ctx->stream));
  TS_TRY(launch_fill_sentinel(ctx->Y[1].get(), 0, (int)np, ctx->stream));
  ctx->bf16 = ctx->cfg.precision == 1;
  if (ctx->bf16) {
    TS_TRY(ctx->Y16[0].alloc(np));
    TS_TRY(ctx->Y16[1].alloc(np));
    TS_TRY(sync_shadow(ctx, 0));
    TS_TRY(sync_shadow(ctx, 1));
  } else {
    ctx->Y16[0] = DevBuf<tsgne::bf162>();
    ctx->Y16[1] = DevBuf<tsgne::bf162>();
  }
  const float ee = ctx->cfg.early_exag > 0.f ? ctx->cfg.early_exag : 1.f;
  ctx->eta = ctx->cfg.learning_rate > 0.f ? ctx->cfg.learning_rate : std::fmax((float)ctx->n / ee / 4.0f, 50.0f);
  return TSGNE_OK;
}

// Installs a built structure + P into the context (commit point of build / set).
tsgne_status install(tsgne_ctx* ctx, int n, int64_t nnz, DevBuf<int64_t>& rp, DevBuf<int32_t>& col, DevBuf<float>& P) {
  ctx->reset_graphs();
  ctx->have_P = false;
  ctx->have_Y = false;
  ctx->n = n;
  ctx->nnz = nnz;
  ctx->rp = std::move(rp);
  ctx->col = std::move(col);
  ctx->P = std::move(P);
  TS_TRY(alloc_layout(ctx));
  if (ctx->bf16) {
    TS_TRY(ctx->P16.alloc((size_t)nnz));
    TS_TRY(launch_to_bf16(ctx->P.get(), ctx->P16.get(), nnz, ctx->stream));
  } else {
    ctx->P16 = DevBuf<tsgne::bf16>();
  }
  TS_TRY(host_guard([&] { return find_heavy_rows(n, ctx->rp.get(), ctx->hub, ctx->stream); }));
  TS_TRY(host_guard([&] {
    return build_attract_plan(n, ctx->rp.get(), ctx->col.get(), ctx->P.get(), ctx->bf16 ? ctx->P16.get() : nullptr,
                              ctx->hub, ctx->plan, ctx->stream);
  }));
  ctx->have_P = true;
  return TSGNE_OK;
}

tsgne_status reset_optimizer(tsgne_ctx* ctx, int32_t t) {
  TS_TRY(launch_fill2(ctx->upd.get(), ctx->n_pad_alloc, 0.f, ctx->stream));
  TS_TRY(launch_fill2(ctx->gains.get(), ctx->n_pad_alloc, 1.f, ctx->stream));
  Sched h{};
  h.t = t;
  TS_CUDA(cudaMemcpyAsync(ctx->sched.get(), &h, sizeof(Sched), cudaMemcpyHostToDevice, ctx->stream));
  return TSGNE_OK;
}

tsgne_status read_ends(const int64_t* rp, int32_t n, int ptr_kind, cudaStream_t s, int64_t* first, int64_t* last) {
  if (ptr_kind == TSGNE_PTR_HOST) {
    *first = rp[0];
    *last = rp[n];
    return TSGNE_OK;
  }
  TS_CUDA(cudaMemcpyAsync(first, rp, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TS_CUDA(cudaMemcpyAsync(last, rp + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TS_CUDA(cudaStreamSynchronize(s));
  return TSGNE_OK;
}

}  // namespace

extern "C" {

void tsgne_config_default(tsgne_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->perplexity = 30.f;
  cfg->k_nn = 0;
  cfg->early_exag = 12.f;
  cfg->ee_iters = 250;
  cfg->momentum0 = 0.5f;
  cfg->momentum1 = 0.8f;
  cfg->learning_rate = 0.f;
  cfg->min_gain = 0.01f;
  cfg->bisect_tol = 1e-5f;
  cfg->bisect_max_iter = 100;
  cfg->seed = 0;
  cfg->precision = 0;
  cfg->profile = 0;
  cfg->spin_budget_cycles = 2000000000LL;
  cfg->repulsion = 0;
  cfg->theta = 0.5f;
  cfg->p_walks = 0;
  cfg->p_walk_length = 3;
}

const char* tsgne_status_string(tsgne_status s) {
  switch (s) {
    case TSGNE_OK: return "TSGNE_OK";
    case TSGNE_ERR_INVALID_ARG: return "TSGNE_ERR_INVALID_ARG";
    case TSGNE_ERR_BAD_CSR: return "TSGNE_ERR_BAD_CSR";
    case TSGNE_ERR_OOM: return "TSGNE_ERR_OOM";
    case TSGNE_ERR_CUDA: return "TSGNE_ERR_CUDA";
    case TSGNE_ERR_NOT_BUILT: return "TSGNE_ERR_NOT_BUILT";
    case TSGNE_ERR_NONFINITE: return "TSGNE_ERR_NONFINITE";
    case TSGNE_ERR_TIMEOUT: return "TSGNE_ERR_TIMEOUT";
    case TSGNE_ERR_CANCELLED: return "TSGNE_ERR_CANCELLED";
    case TSGNE_ERR_INDEX: return "TSGNE_ERR_INDEX";
  }
  return "TSGNE_ERR_UNKNOWN";
}

tsgne_status tsgne_create(tsgne_ctx** out, const tsgne_config* cfg, void* cuda_stream) {
  if (!out) return TSGNE_ERR_INVALID_ARG;
  *out = nullptr;
  tsgne_config c;
  if (cfg) c = *cfg; else tsgne_config_default(&c);
  if (!(c.perplexity > 1.f) || c.k_nn < 0 || c.k_nn > 256 || (c.precision != 0 && c.precision != 1) ||
      c.ee_iters < 0 || !(c.min_gain >= 0.f) || !(c.bisect_tol > 0.f) || c.bisect_max_iter < 1 ||
      !std::isfinite(c.early_exag) || !std::isfinite(c.momentum0) || !std::isfinite(c.momentum1) ||
      (c.repulsion != 0 && c.repulsion != 1) || !(c.theta >= 0.f && c.theta <= 1.f) || c.p_walks < 0 ||
      c.p_walks > 512 || c.p_walk_length < 1 || c.p_walk_length > 64 || c.spin_budget_cycles <= 0) {
    last_msg() =
        "invalid configuration (perplexity must exceed 1; k_nn in [0, 256]; precision 0 or 1; repulsion 0 or 1; "
        "theta in [0, 1]; p_walks in [0, 512]; p_walk_length in [1, 64]; spin_budget_cycles > 0)";
    return TSGNE_ERR_INVALID_ARG;
  }
  tsgne_ctx* ctx = new (std::nothrow) tsgne_ctx();
  if (!ctx) return TSGNE_ERR_OOM;
  ctx->cfg = c;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) {
    if (cuda_stream) {
      ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
      e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
      ctx->own_stream = (e == cudaSuccess);
    }
  }
  tsgne_status st = TSGNE_OK;
  if (e != cudaSuccess) st = cuda_fail(e, "tsgne_create", __FILE__, __LINE__);
  if (st == TSGNE_OK) st = ctx->sched.alloc(1);
  if (st == TSGNE_OK) {
    e = cudaMemsetAsync(ctx->sched.get(), 0, sizeof(Sched), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "tsgne_create", __FILE__, __LINE__);
  }
  if (st != TSGNE_OK) {
    delete ctx;
    return st;
  }
  *out = ctx;
  return TSGNE_OK;
}

void tsgne_destroy(tsgne_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  delete ctx;
}

const char* tsgne_last_error(const tsgne_ctx* ctx) { return ctx ? ctx->err.c_str() : last_msg().c_str(); }

tsgne_status tsgne_build_P(tsgne_ctx* ctx, int32_t n, const int64_t* row_ptr, const int32_t* col_idx, const float* X,
                           int32_t d, int32_t ptr_kind) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (n < 2 || d < 1 || !row_ptr || !X || !valid_kind(ptr_kind))
    return fail(ctx, TSGNE_ERR_INVALID_ARG, "need n >= 2, d >= 1, non-NULL row_ptr and X, a valid ptr_kind");
  int64_t first = 0, m = 0;
  API_TRY(ctx, read_ends(row_ptr, n, ptr_kind, ctx->stream, &first, &m));
  if (first != 0 || m < 0) return fail(ctx, TSGNE_ERR_BAD_CSR, "row_ptr[0] must be 0 and row_ptr[n] >= 0");
  if (m > 0 && !col_idx) return fail(ctx, TSGNE_ERR_INVALID_ARG, "col_idx is NULL");
  if (m > (int64_t)1 << 30) return fail(ctx, TSGNE_ERR_INVALID_ARG, "more than 2^30 input entries");
  ProfRec pr;
  API_TRY(ctx, prof_begin(ctx, 4, &pr));
  DevBuf<int64_t> rp_in;
  DevBuf<int32_t> col_in;
  DevBuf<float> X_in;
  const int64_t* rp_d = row_ptr;
  const int32_t* col_d = col_idx;
  const float* X_d = X;
  if (ptr_kind == TSGNE_PTR_HOST) {
    API_TRY(ctx, to_device(row_ptr, (size_t)n + 1, ptr_kind, rp_in, ctx->stream));
    API_TRY(ctx, to_device(col_idx, (size_t)m, ptr_kind, col_in, ctx->stream));
    API_TRY(ctx, to_device(X, (size_t)n * (size_t)d, ptr_kind, X_in, ctx->stream));
    rp_d = rp_in.get();
    col_d = col_in.get();
    X_d = X_in.get();
  }
  DevBuf<int64_t> rp, tslot;
  DevBuf<int32_t> col;
  DevBuf<float> P;
  int64_t nnz = 0;
  API_TRY(ctx, build_neighbor_structure(n, rp_d, col_d, m, ctx->cfg.k_nn, rp, col, tslot, &nnz, ctx->stream));
  API_CUDA(ctx, cudaMemsetAsync(ctx->sched.get(), 0, sizeof(Sched), ctx->stream));
  if (ctx->cfg.p_walks > 0) {  // Eq. 6: the structure becomes that of the walk pairs
    DevBuf<int64_t> wrp;
    DevBuf<int32_t> wcol;
    int64_t wnnz = 0;
    API_TRY(ctx, random_walk_affinities(n, rp.get(), col.get(), nnz, X_d, d, ctx->cfg.p_walks,
                                        ctx->cfg.p_walk_length, ctx->cfg.seed, wrp, wcol, P, &wnnz, ctx->sched.get(),
                                        ctx->stream));
    rp = std::move(wrp);
    col = std::move(wcol);
    nnz = wnnz;
  } else {
    API_TRY(ctx, P.alloc((size_t)nnz));
    API_TRY(ctx, build_affinities(n, rp.get(), col.get(), tslot.get(), nnz, X_d, d, ctx->cfg.perplexity,
                                  ctx->cfg.bisect_tol, ctx->cfg.bisect_max_iter, P.get(), ctx->sched.get(),
                                  ctx->stream));
  }
  API_TRY(ctx, prof_end(ctx, &pr));
  Sched h;
  API_TRY(ctx, read_sched(ctx, &h));
  if (h.flags & kFlagNonfiniteP) return fail(ctx, TSGNE_ERR_NONFINITE, "non-finite affinity (check X)");
  API_TRY(ctx, install(ctx, n, nnz, rp, col, P));
  API_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return TSGNE_OK;
}

tsgne_status tsgne_build_P_shortest_path(tsgne_ctx* ctx, int32_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                         const int32_t* targets, int32_t d, int32_t l0, int32_t ptr_kind) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (n < 2 || d < 1 || d > 1024 || !row_ptr || !targets || !valid_kind(ptr_kind))
    return fail(ctx, TSGNE_ERR_INVALID_ARG, "need n >= 2, 1 <= d <= 1024, row_ptr, targets, a valid ptr_kind");
  int64_t first = 0, m = 0;
  API_TRY(ctx, read_ends(row_ptr, n, ptr_kind, ctx->stream, &first, &m));
  if (first != 0 || m < 0) return fail(ctx, TSGNE_ERR_BAD_CSR, "row_ptr[0] must be 0 and row_ptr[n] >= 0");
  DevBuf<int64_t> rp_in;
  DevBuf<int32_t> col_in, tg;
  DevBuf<float> X;
  API_TRY(ctx, to_device(row_ptr, (size_t)n + 1, ptr_kind, rp_in, ctx->stream));
  API_TRY(ctx, to_device(col_idx, (size_t)m, ptr_kind, col_in, ctx->stream));
  API_TRY(ctx, to_device(targets, (size_t)d, ptr_kind, tg, ctx->stream));
  API_TRY(ctx, X.alloc((size_t)n * d));
  const tsgne_status st = tsgne_shortest_path_embedding(n, rp_in.get(), col_in.get(), tg.get(), d, l0, X.get(),
                                                        TSGNE_PTR_DEVICE, ctx->stream);
  if (st != TSGNE_OK) return fail(ctx, st, last_msg().empty() ? "ShortestPath embedding failed" : last_msg());
  return tsgne_build_P(ctx, n, rp_in.get(), col_in.get(), X.get(), d, TSGNE_PTR_DEVICE);
}

tsgne_status tsgne_set_P(tsgne_ctx* ctx, int32_t n, const int64_t* row_ptr, const int32_t* col_idx, const float* Pv,
                         int32_t ptr_kind) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (n < 2 || !row_ptr || !valid_kind(ptr_kind)) return fail(ctx, TSGNE_ERR_INVALID_ARG, "need n >= 2 and row_ptr");
  int64_t first = 0, m = 0;
  API_TRY(ctx, read_ends(row_ptr, n, ptr_kind, ctx->stream, &first, &m));
  if (first != 0 || m < 0) return fail(ctx, TSGNE_ERR_BAD_CSR, "row_ptr[0] must be 0 and row_ptr[n] >= 0");
  if (m > 0 && (!col_idx || !Pv)) return fail(ctx, TSGNE_ERR_INVALID_ARG, "col_idx or P is NULL");
  DevBuf<int64_t> rp_in, rp, tslot;
  DevBuf<int32_t> col_in, col;
  DevBuf<float> P;
  API_TRY(ctx, to_device(row_ptr, (size_t)n + 1, ptr_kind, rp_in, ctx->stream));
  API_TRY(ctx, to_device(col_idx, (size_t)m, ptr_kind, col_in, ctx->stream));
  API_TRY(ctx, to_device(Pv, (size_t)m, ptr_kind, P, ctx->stream));
  int64_t nnz = 0;
  API_TRY(ctx, build_structure(n, rp_in.get(), col_in.get(), m, rp, col, tslot, &nnz, ctx->sched.get(), ctx->stream));
  if (nnz != m) return fail(ctx, TSGNE_ERR_BAD_CSR, "structure is not symmetric, sorted, unique and loop-free");
  DevBuf<uint32_t> neq;
  API_TRY(ctx, neq.alloc(1));
  API_CUDA(ctx, cudaMemsetAsync(neq.get(), 0, sizeof(uint32_t), ctx->stream));
  k_cmp_i64<<<64, 256, 0, ctx->stream>>>(rp.get(), rp_in.get(), (int64_t)n + 1, neq.get());
  if (m > 0) k_cmp_i32<<<256, 256, 0, ctx->stream>>>(col.get(), col_in.get(), m, neq.get());
  API_CUDA(ctx, cudaGetLastError());
  uint32_t hneq = 0;
  API_CUDA(ctx, cudaMemcpyAsync(&hneq, neq.get(), sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
  API_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hneq) return fail(ctx, TSGNE_ERR_BAD_CSR, "structure is not symmetric, sorted, unique and loop-free");
  API_CUDA(ctx, cudaMemsetAsync(ctx->sched.get(), 0, sizeof(Sched), ctx->stream));
  API_TRY(ctx, install(ctx, n, nnz, rp, col, P));
  API_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return TSGNE_OK;
}

tsgne_status tsgne_get_sizes(tsgne_ctx* ctx, int32_t* n, int64_t* nnz) {
  TS_TRY(enter(ctx));
  if (!ctx->have_P) return fail(ctx, TSGNE_ERR_NOT_BUILT, "no affinities yet");
  if (n) *n = ctx->n;
  if (nnz) *nnz = ctx->nnz;
  return TSGNE_OK;
}

tsgne_status tsgne_get_P(tsgne_ctx* ctx, int64_t* row_ptr, int32_t* col, float* val, int32_t ptr_kind) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (!valid_kind(ptr_kind)) return fail(ctx, TSGNE_ERR_INVALID_ARG, "bad ptr_kind");
  if (!ctx->have_P) return fail(ctx, TSGNE_ERR_NOT_BUILT, "no affinities yet");
  if (row_ptr) API_TRY(ctx, copy_out(row_ptr, ctx->rp.get(), sizeof(int64_t) * ((size_t)ctx->n + 1), ptr_kind, ctx->stream));
  if (col) API_TRY(ctx, copy_out(col, ctx->col.get(), sizeof(int32_t) * (size_t)ctx->nnz, ptr_kind, ctx->stream));
  if (val) API_TRY(ctx, copy_out(val, ctx->P.get(), sizeof(float) * (size_t)ctx->nnz, ptr_kind, ctx->stream));
  API_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return TSGNE_OK;
}

tsgne_status tsgne_init_Y(tsgne_ctx* ctx, const float* Y0, int32_t ptr_kind) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (!valid_kind(ptr_kind)) return fail(ctx, TSGNE_ERR_INVALID_ARG, "bad ptr_kind");
  if (!ctx->have_P) return fail(ctx, TSGNE_ERR_NOT_BUILT, "build P first");
  ctx->cur = 0;
  if (Y0) {
    API_TRY(ctx, copy_in(ctx->Y[0].get(), Y0, sizeof(float2) * (size_t)ctx->n, ptr_kind, ctx->stream));
  } else {
    API_TRY(ctx, launch_init_Y(ctx->n, ctx->cfg.seed, 1e-4f, ctx->Y[0].get(), ctx->stream));
  }
  API_TRY(ctx, sync_shadow(ctx, 0));
  API_TRY(ctx, reset_optimizer(ctx, 0));
  API_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->have_Y = true;
  return TSGNE_OK;
}

tsgne_status tsgne_step(tsgne_ctx* ctx) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (!ctx->have_P || !ctx->have_Y) return fail(ctx, TSGNE_ERR_NOT_BUILT, "build P and set Y first");
  API_TRY(ctx, enqueue_step(ctx));
  return TSGNE_OK;
}

tsgne_status tsgne_run(tsgne_ctx* ctx, int32_t n_iter) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (n_iter < 0) return fail(ctx, TSGNE_ERR_INVALID_ARG, "n_iter < 0");
  if (!ctx->have_P || !ctx->have_Y) return fail(ctx, TSGNE_ERR_NOT_BUILT, "build P and set Y first");
  int32_t k = 0;
  if (!ctx->cfg.profile && capturable(ctx->stream) && n_iter >= 2) {
    API_TRY(ctx, ensure_graph(ctx, ctx->cur));
    for (; k + 2 <= n_iter; k += 2) API_CUDA(ctx, cudaGraphLaunch(ctx->g2[ctx->cur], ctx->stream));
  }
  for (; k < n_iter; ++k) API_TRY(ctx, enqueue_step(ctx));
  API_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  API_TRY(ctx, check_flags(ctx));
  return TSGNE_OK;
}

tsgne_status tsgne_sync(tsgne_ctx* ctx) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  API_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->have_P) API_TRY(ctx, check_flags(ctx));
  return TSGNE_OK;
}

tsgne_status tsgne_kl(tsgne_ctx* ctx, double* kl_out) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (!kl_out) return fail(ctx, TSGNE_ERR_INVALID_ARG, "kl_out is NULL");
  if (!ctx->have_P || !ctx->have_Y) return fail(ctx, TSGNE_ERR_NOT_BUILT, "build P and set Y first");
  API_TRY(ctx, enqueue_repulsion(ctx, 0));
  ProfRec pr;
  API_TRY(ctx, prof_begin(ctx, 3, &pr));
  API_TRY(ctx, launch_kl(ctx->n, ctx->rp.get(), ctx->col.get(), ctx->Pread(), ctx->bf16 ? 1 : 0,
                         ctx->Yread(ctx->cur), ctx->bf16 ? 1 : 0, ctx->klpart.get(), kl_partial_count(ctx->sms),
                         ctx->sched.get(), ctx->stream));
  API_TRY(ctx, prof_end(ctx, &pr));
  Sched h;
  API_TRY(ctx, read_sched(ctx, &h));
  API_TRY(ctx, check_tree_flags(ctx, h));
  *kl_out = h.red[0] + h.red[1] * std::log(h.Z);
  if (!std::isfinite(*kl_out)) return fail(ctx, TSGNE_ERR_NONFINITE, "KL is not finite");
  return TSGNE_OK;
}

tsgne_status tsgne_gradient(tsgne_ctx* ctx, float alpha, float* g_out, double* z_out, int32_t ptr_kind) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (!g_out || !valid_kind(ptr_kind)) return fail(ctx, TSGNE_ERR_INVALID_ARG, "g_out is NULL or bad ptr_kind");
  if (!ctx->have_P || !ctx->have_Y) return fail(ctx, TSGNE_ERR_NOT_BUILT, "build P and set Y first");
  API_TRY(ctx, enqueue_repulsion(ctx, 0));
  ProfRec pr;
  API_TRY(ctx, prof_begin(ctx, 2, &pr));
  API_TRY(ctx, launch_gradient(attract_args(ctx), alpha, ctx->grad.get(), ctx->stream));
  API_TRY(ctx, prof_end(ctx, &pr));
  API_TRY(ctx, copy_out(g_out, ctx->grad.get(), sizeof(float2) * (size_t)ctx->n, ptr_kind, ctx->stream));
  Sched h;
  API_TRY(ctx, read_sched(ctx, &h));
  API_TRY(ctx, check_tree_flags(ctx, h));
  if (z_out) *z_out = h.Z;
  return TSGNE_OK;
}

tsgne_status tsgne_get_Y(tsgne_ctx* ctx, float* Y_out, int32_t ptr_kind) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (!Y_out || !valid_kind(ptr_kind)) return fail(ctx, TSGNE_ERR_INVALID_ARG, "Y_out is NULL or bad ptr_kind");
  if (!ctx->have_Y) return fail(ctx, TSGNE_ERR_NOT_BUILT, "no layout yet");
  API_TRY(ctx, copy_out(Y_out, ctx->Y[ctx->cur].get(), sizeof(float2) * (size_t)ctx->n, ptr_kind, ctx->stream));
  API_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return TSGNE_OK;
}

tsgne_status tsgne_get_state(tsgne_ctx* ctx, float* Y, float* update, float* gains, int32_t* iter, int32_t ptr_kind) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (!valid_kind(ptr_kind)) return fail(ctx, TSGNE_ERR_INVALID_ARG, "bad ptr_kind");
  if (!ctx->have_Y) return fail(ctx, TSGNE_ERR_NOT_BUILT, "no layout yet");
  const size_t bytes = sizeof(float2) * (size_t)ctx->n;
  if (Y) API_TRY(ctx, copy_out(Y, ctx->Y[ctx->cur].get(), bytes, ptr_kind, ctx->stream));
  if (update) API_TRY(ctx, copy_out(update, ctx->upd.get(), bytes, ptr_kind, ctx->stream));
  if (gains) API_TRY(ctx, copy_out(gains, ctx->gains.get(), bytes, ptr_kind, ctx->stream));
  Sched h;
  API_TRY(ctx, read_sched(ctx, &h));
  if (iter) *iter = h.t;
  return TSGNE_OK;
}

tsgne_status tsgne_set_state(tsgne_ctx* ctx, const float* Y, const float* update, const float* gains, int32_t iter,
                             int32_t ptr_kind) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (!valid_kind(ptr_kind) || iter < 0 || !Y) return fail(ctx, TSGNE_ERR_INVALID_ARG, "need Y, iter >= 0, ptr_kind");
  if (!ctx->have_P) return fail(ctx, TSGNE_ERR_NOT_BUILT, "build P first");
  const size_t bytes = sizeof(float2) * (size_t)ctx->n;
  ctx->cur = 0;
  API_TRY(ctx, reset_optimizer(ctx, iter));
  API_TRY(ctx, copy_in(ctx->Y[0].get(), Y, bytes, ptr_kind, ctx->stream));
  API_TRY(ctx, sync_shadow(ctx, 0));
  if (update) API_TRY(ctx, copy_in(ctx->upd.get(), update, bytes, ptr_kind, ctx->stream));
  if (gains) API_TRY(ctx, copy_in(ctx->gains.get(), gains, bytes, ptr_kind, ctx->stream));
  API_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->have_Y = true;
  return TSGNE_OK;
}

tsgne_status tsgne_kernel_times(tsgne_ctx* ctx, double* ms, int64_t* launches, int32_t n, int32_t reset) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (n < 0 || n > kClasses) return fail(ctx, TSGNE_ERR_INVALID_ARG, "n outside [0, 8]");
  API_TRY(ctx, prof_collect(ctx));
  for (int k = 0; k < n; ++k) {
    if (ms) ms[k] = ctx->prof_ms[k];
    if (launches) launches[k] = ctx->prof_n[k];
  }
  if (reset)
    for (int k = 0; k < kClasses; ++k) {
      ctx->prof_ms[k] = 0.0;
      ctx->prof_n[k] = 0;
    }
  return TSGNE_OK;
}

void tsgne_set_device_memory_limit(int64_t bytes) { tsgne::g_dev_limit.store(bytes > 0 ? bytes : 0); }

int64_t tsgne_device_memory_in_use(void) { return tsgne::g_dev_bytes.load(); }

tsgne_status tsgne_repulsion_shape(tsgne_ctx* ctx, int32_t* grid, int32_t* block, int32_t* i_per_thread,
                                   int32_t* j_tile, int32_t* j_chunks, int32_t* n_pad) {
  TS_TRY(enter(ctx));
  if (!ctx->have_P) return fail(ctx, TSGNE_ERR_NOT_BUILT, "build P first");
  const RepShape& sh = ctx->ordered ? ctx->oshape : ctx->shape;
  if (grid) *grid = sh.grid;
  if (block) *block = sh.block;
  if (i_per_thread) *i_per_thread = sh.R;
  if (j_tile) *j_tile = sh.jtile;
  if (j_chunks) *j_chunks = sh.chunks;
  if (n_pad) *n_pad = sh.n_pad;
  return TSGNE_OK;
}

namespace {
std::mutex g_shape_mu;
std::map<std::tuple<int, int, int>, int> g_shape_cache;  // (SMs, ceil log2 n, bf16) -> candidate index

// Candidate shapes of the exact pass: (warps per CTA, i-points per lane,
// symmetric); the last is the ordered-pair kernel (FP32 storage only).
constexpr int kCtxShapes[5][3] = {{2, 16, 1}, {1, 16, 1}, {2, 8, 1}, {1, 8, 1}, {0, 0, 0}};

tsgne_status set_shape(tsgne_ctx* ctx, int warps, int ri, int symmetric) {
  if (symmetric) {
    if (!((warps == 1 || warps == 2) && (ri == 8 || ri == 16))) {
      last_msg() = "symmetric shapes: warps 1 or 2, i_per_lane 8 or 16";
      return TSGNE_ERR_INVALID_ARG;
    }
    const RepShape sh = repulsion_shape_sym_fixed(ctx->n, ctx->sms, warps, ri);
    TS_TRY(repulsion_sym_prepare(sh));
    if ((size_t)sh.units > ctx->zpart.n) TS_TRY(ctx->zpart.alloc((size_t)sh.units));
    ctx->shape = sh;
    ctx->ordered = false;
    ctx->oslots = DevBuf<float2>();
  } else {
    if (ctx->bf16) {
      last_msg() = "the ordered-pair kernel reads FP32 layouts only";
      return TSGNE_ERR_INVALID_ARG;
    }
    const RepShape sh = repulsion_shape(ctx->n, ctx->sms);
    if (sh.n_pad > ctx->n_pad_alloc) {
      last_msg() = "ordered shape exceeds the layout padding";
      return TSGNE_ERR_INVALID_ARG;
    }
    TS_TRY(ctx->oslots.alloc((size_t)sh.chunks * (size_t)sh.n_pad));
    if (repulsion_zpart_count(sh) > ctx->zpart.n) TS_TRY(ctx->zpart.alloc(repulsion_zpart_count(sh)));
    ctx->oshape = sh;
    ctx->ordered = true;
  }
  ctx->reset_graphs();
  return TSGNE_OK;
}
}  // namespace

tsgne_status tsgne_set_repulsion_shape(tsgne_ctx* ctx, int32_t tile_warps, int32_t i_per_lane, int32_t symmetric) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (!ctx->have_P) return fail(ctx, TSGNE_ERR_NOT_BUILT, "build P first");
  if (ctx->use_tree) return fail(ctx, TSGNE_ERR_INVALID_ARG, "the tree code has no exact-pass shape");
  if (ctx->shard_pending) return fail(ctx, TSGNE_ERR_INVALID_ARG, "a share is awaiting its finish call");
  API_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  API_TRY(ctx, set_shape(ctx, tile_warps, i_per_lane, symmetric ? 1 : 0));
  return TSGNE_OK;
}

tsgne_status tsgne_autotune(tsgne_ctx* ctx, int32_t trial_passes, int32_t* tile_warps, int32_t* i_per_lane,
                            int32_t* symmetric, float* ms_per_pass) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (trial_passes < 1) return fail(ctx, TSGNE_ERR_INVALID_ARG, "trial_passes < 1");
  if (!ctx->have_P || !ctx->have_Y) return fail(ctx, TSGNE_ERR_NOT_BUILT, "build P and set Y first");
  if (ctx->use_tree) return fail(ctx, TSGNE_ERR_INVALID_ARG, "the tree code has no exact-pass shape");
  if (ctx->shard_pending) return fail(ctx, TSGNE_ERR_INVALID_ARG, "a share is awaiting its finish call");
  int lg = 0;
  while ((1LL << lg) < (long long)ctx->n) ++lg;
  const auto key = std::make_tuple(ctx->sms, lg, ctx->bf16 ? 1 : 0);
  const bool prof = ctx->cfg.profile != 0;
  ctx->cfg.profile = 0;  // candidate passes are timed here, not by the kernel profile
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  API_CUDA(ctx, cudaEventCreate(&e0));
  API_CUDA(ctx, cudaEventCreate(&e1));
  int best = -1;
  float best_ms = 0.f;
  tsgne_status st = TSGNE_OK;
  for (int k = 0; k < 5 && st == TSGNE_OK; ++k) {
    const int* c = kCtxShapes[k];
    float ms = -1.f;
    if (!c[2] && ctx->bf16) {
      if (ms_per_pass) ms_per_pass[k] = ms;  // not a candidate with BF16 storage
      continue;
    }
    st = cudaStreamSynchronize(ctx->stream) == cudaSuccess ? TSGNE_OK : TSGNE_ERR_CUDA;
    if (st == TSGNE_OK) st = set_shape(ctx, c[0], c[1], c[2]);
    if (st == TSGNE_OK) st = enqueue_repulsion(ctx, 0);  // warm-up; passes do not advance the iteration
    if (st == TSGNE_OK) st = cudaEventRecord(e0, ctx->stream) == cudaSuccess ? TSGNE_OK : TSGNE_ERR_CUDA;
    for (int t = 0; t < trial_passes && st == TSGNE_OK; ++t) st = enqueue_repulsion(ctx, 0);
    if (st == TSGNE_OK) st = cudaEventRecord(e1, ctx->stream) == cudaSuccess ? TSGNE_OK : TSGNE_ERR_CUDA;
    if (st == TSGNE_OK) st = cudaEventSynchronize(e1) == cudaSuccess ? TSGNE_OK : TSGNE_ERR_CUDA;
    if (st == TSGNE_OK) st = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess ? TSGNE_OK : TSGNE_ERR_CUDA;
    if (st != TSGNE_OK) break;
    ms /= (float)trial_passes;
    if (ms_per_pass) ms_per_pass[k] = ms;
    if (best < 0 || ms < best_ms) {
      best = k;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->cfg.profile = prof ? 1 : 0;
  if (st != TSGNE_OK) return fail(ctx, st);
  API_TRY(ctx, set_shape(ctx, kCtxShapes[best][0], kCtxShapes[best][1], kCtxShapes[best][2]));
  {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_shape_cache[key] = best;
  }
  if (tile_warps) *tile_warps = kCtxShapes[best][0];
  if (i_per_lane) *i_per_lane = kCtxShapes[best][1];
  if (symmetric) *symmetric = kCtxShapes[best][2];
  return TSGNE_OK;
}

// ------------------------------------------------------------- sharding

tsgne_status tsgne_shard_set(tsgne_ctx* ctx, int32_t rank, int32_t world) {
  TS_TRY(enter(ctx));
  if (world < 1 || rank < 0 || rank >= world)
    return fail(ctx, TSGNE_ERR_INVALID_ARG, "need 0 <= rank < world");
  if (ctx->cfg.repulsion != 0)
    return fail(ctx, TSGNE_ERR_INVALID_ARG, "sharding applies to the exact repulsion (cfg.repulsion = 0)");
  if (ctx->shard_pending) return fail(ctx, TSGNE_ERR_INVALID_ARG, "a share is awaiting its finish call");
  ctx->shard_rank = rank;
  ctx->shard_world = world;
  return TSGNE_OK;
}

tsgne_status tsgne_shard_repulsion(tsgne_ctx* ctx, int64_t* units, int32_t* u0, int32_t* u1, void** acc,
                                   int64_t* acc_count, void** zunit) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (!ctx->have_P || !ctx->have_Y) return fail(ctx, TSGNE_ERR_NOT_BUILT, "build P and set Y first");
  if (ctx->use_tree || ctx->ordered)
    return fail(ctx, TSGNE_ERR_INVALID_ARG, "sharding applies to the symmetric exact repulsion");
  if (ctx->shard_pending) return fail(ctx, TSGNE_ERR_INVALID_ARG, "the previous share has not been finished");
  const int64_t U = ctx->shape.units;
  ctx->shard_u0 = (int)(U * ctx->shard_rank / ctx->shard_world);
  ctx->shard_u1 = (int)(U * (ctx->shard_rank + 1) / ctx->shard_world);
  // units of the other shares contribute 0 here, so the sum over the
  // shares holds every unit's partial exactly once
  API_CUDA(ctx, cudaMemsetAsync(ctx->zpart.get(), 0, sizeof(double) * (size_t)U, ctx->stream));
  ProfRec pr;
  API_TRY(ctx, prof_begin(ctx, 0, &pr));
  API_TRY(ctx, launch_repulsion_sym_units(ctx->shape, ctx->n, ctx->Yread(ctx->cur), ctx->bf16 ? 1 : 0,
                                          ctx->facc.get(), ctx->zpart.get(), ctx->sched.get(), ctx->shard_u0,
                                          ctx->shard_u1, ctx->stream));
  API_TRY(ctx, prof_end(ctx, &pr));
  ctx->shard_pending = true;
  if (units) *units = U;
  if (u0) *u0 = ctx->shard_u0;
  if (u1) *u1 = ctx->shard_u1;
  if (acc) *acc = ctx->facc.get();
  if (acc_count) *acc_count = 2 * (int64_t)ctx->n;
  if (zunit) *zunit = ctx->zpart.get();
  return TSGNE_OK;
}

namespace {
// Z, schedule and F^r after the shares were summed (advance: an iteration).
tsgne_status shard_close(tsgne_ctx* ctx, int advance) {
  const tsgne_config& c = ctx->cfg;
  TS_TRY(launch_finalize_z(ctx->shape, ctx->n, ctx->zpart.get(), ctx->sched.get(), advance, c.early_exag, c.ee_iters,
                           c.momentum0, c.momentum1, ctx->stream));
  ProfRec pr;
  TS_TRY(prof_begin(ctx, 5, &pr));
  TS_TRY(launch_fix_forces(ctx->n, ctx->facc.get(), ctx->fsum.get(), ctx->stream));
  TS_TRY(prof_end(ctx, &pr));
  ctx->shard_pending = false;
  return TSGNE_OK;
}
}  // namespace

tsgne_status tsgne_shard_step_finish(tsgne_ctx* ctx) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (!ctx->shard_pending) return fail(ctx, TSGNE_ERR_INVALID_ARG, "no share awaits its finish call");
  API_TRY(ctx, shard_close(ctx, 1));
  API_TRY(ctx, enqueue_update(ctx));
  return TSGNE_OK;
}

tsgne_status tsgne_shard_gradient_finish(tsgne_ctx* ctx, float alpha, float* g_out, double* z_out,
                                         int32_t ptr_kind) {
  TS_TRY(enter(ctx));
  DeviceGuard dg(ctx->device);
  if (!g_out || !valid_kind(ptr_kind)) return fail(ctx, TSGNE_ERR_INVALID_ARG, "g_out is NULL or bad ptr_kind");
  if (!ctx->shard_pending) return fail(ctx, TSGNE_ERR_INVALID_ARG, "no share awaits its finish call");
  API_TRY(ctx, shard_close(ctx, 0));
  API_TRY(ctx, launch_gradient(attract_args(ctx), alpha, ctx->grad.get(), ctx->stream));
  API_TRY(ctx, copy_out(g_out, ctx->grad.get(), sizeof(float2) * (size_t)ctx->n, ptr_kind, ctx->stream));
  Sched h;
  API_TRY(ctx, read_sched(ctx, &h));
  if (z_out) *z_out = h.Z;
  return TSGNE_OK;
}

tsgne_status tsgne_stream(tsgne_ctx* ctx, void** cuda_stream) {
  if (!ctx || !cuda_stream) return TSGNE_ERR_INVALID_ARG;
  *cuda_stream = ctx->stream;
  return TSGNE_OK;
}

}  // extern "C"
