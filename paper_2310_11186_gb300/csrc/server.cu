// Continuous-batching layout server (host scheduler over the batch engine).
//
// A request is a graph (CSR + embedding, optional Y0) to lay out for a fixed
// number of iterations.  Submitted requests wait in a FIFO queue; every tick
//   1. admits queued requests in order while the estimated device bytes of
//      all resident layouts stay within the budget and below the free device
//      memory (the first request is admitted whatever its size when nothing
//      is resident, so no request starves);
//   2. selects the resident layouts to advance: all of them (policy 0), or
//      (policy 1, shortest remaining work first with aging) first the
//      layouts left out of aging_ticks ticks in a row, longest waiting
//      first, then those with the least remaining iterations x n^2, until
//      their pairs per iteration reach fill_pairs, enough tile pairs to keep
//      every SM busy (without aging a stream of small requests could hold
//      a large one back indefinitely);
//   3. runs tick_iters iterations of the selected layouts in one batched call
//      (requests of at least tree_min_n points are tree-code members, whose
//      trees are built and walked concurrently within each iteration);
//   4. retires the layouts that reached their iterations: the layout is
//      copied to server-owned host memory and the member's device memory is
//      freed.
// Admission overlaps with the running iterations: an admitted request is
// handed to a worker thread that builds its member (structure, P, buffers,
// tree) with tsgne_batch_prepare on the worker's own stream, with
// stream-ordered allocations (cudaFree would wait for the whole device),
// while the tick launches the resident layouts' iterations; prepared members
// are attached at the start of the next tick.  A tick with nothing resident
// waits for all admitted requests to be prepared instead of running nothing.
// Every member's arithmetic is independent of the others (batch.cu), so a
// request's layout is the same whatever else is resident.  Cancelling a
// queued or resident request frees it at once; its result reports
// TSGNE_ERR_CANCELLED.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "tsgne.h"

namespace {

// kPreparing (admitted, its member being built by the worker) is reported
// as queued.
enum ReqState : int32_t { kQueued = 0, kResident = 1, kDone = 2, kCancelled = 3, kPreparing = 4 };

struct Req {
  int64_t id = 0;
  int32_t n = 0, d = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> col;
  std::vector<float> X, Y0, Y;
  int32_t state = kQueued;
  int32_t iters = 0;
  int32_t member = -1;
  int64_t bytes = 0;
  int32_t waited = 0;  // ticks in a row this resident layout was not advanced
  int32_t repulsion = 0;  // 0 exact, 1 tree code
};

// Work of one iteration in exact-pass pairs: n^2 / 2 for the exact pass; for
// the tree code about 250 n log2 n (measured: 300K points take 1/35 of the
// exact pass's time).  Only orders requests and sizes a tick.
double iter_pairs(const Req& r) {
  const double n = (double)r.n;
  return r.repulsion ? 250.0 * n * std::log2(n > 2.0 ? n : 2.0) : 0.5 * n * n;
}

// Device bytes of a tree-code member's tree (TreeBufs) and layout copy.
int64_t tree_bytes(int64_t n) { return 144 * n + 4096; }

}  // namespace

struct tsgne_server {
  tsgne_server_config cfg{};
  tsgne_batch* batch = nullptr;
  std::map<int64_t, Req> reqs;  // inserted / erased under mu (the worker looks requests up)
  std::deque<int64_t> queue;
  std::vector<int64_t> finished;  // retired since the last tsgne_server_finished
  int64_t next_id = 1;
  int64_t used = 0;
  std::string msg;
  // admission worker
  int device = 0;
  cudaStream_t prep = nullptr;  // the worker's stream (its members' memory is ordered on it)
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_ready;
  std::deque<int64_t> prep_q;                                // admitted, to prepare (under mu)
  std::vector<std::pair<int64_t, tsgne_member*>> ready;      // prepared (under mu)
  std::vector<std::pair<int64_t, std::string>> failed;      // prepare errors (under mu)
  bool stop = false;                                         // (under mu)
  int32_t preparing = 0;                                     // admitted, not yet attached
};

namespace {

tsgne_status sfail(tsgne_server* s, tsgne_status st, const std::string& m) {
  s->msg = m;
  return st;
}

tsgne_status batch_fail(tsgne_server* s, tsgne_status st) {
  s->msg = tsgne_batch_last_error(s->batch);
  return st;
}

int64_t free_device_bytes(int64_t fallback) {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return fallback;
  return (int64_t)fr;
}

tsgne_status admit(tsgne_server* s) {
  int32_t members = s->preparing;
  for (const auto& kv : s->reqs) members += kv.second.state == kResident;
  while (!s->queue.empty()) {
    Req& r = s->reqs[s->queue.front()];
    r.repulsion = (s->cfg.tree_min_n > 0 && r.n >= s->cfg.tree_min_n) ? 1 : 0;
    const int64_t need =
        tsgne_server_estimate_bytes(r.n, 2 * r.rp[r.n], s->cfg.tile_warps) + (r.repulsion ? tree_bytes(r.n) : 0);
    if (members > 0 && (members >= s->cfg.max_members || s->used + need > s->cfg.budget_bytes ||
                        need > free_device_bytes(s->cfg.budget_bytes)))
      break;
    r.state = kPreparing;
    r.bytes = need;
    s->used += need;
    ++members;
    ++s->preparing;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->prep_q.push_back(r.id);
    }
    s->cv_work.notify_one();
    s->queue.pop_front();
  }
  return TSGNE_OK;
}

// Prepares admitted requests' members while the ticks run.
void worker_main(tsgne_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    Req* r = nullptr;
    int64_t id = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [s] { return s->stop || !s->prep_q.empty(); });
      if (s->stop) return;
      id = s->prep_q.front();
      s->prep_q.pop_front();
      r = &s->reqs.find(id)->second;  // present and not erased while preparing; its inputs are not touched by the ticks
    }
    tsgne_member* m = nullptr;
    const tsgne_status st = tsgne_batch_prepare(s->batch, r->n, r->rp.data(), r->col.empty() ? nullptr : r->col.data(),
                                                r->X.data(), r->d, r->Y0.empty() ? nullptr : r->Y0.data(),
                                                TSGNE_PTR_HOST, r->repulsion, s->prep, &m);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (st == TSGNE_OK)
        s->ready.emplace_back(id, m);
      else
        s->failed.emplace_back(id, std::string(tsgne_status_string(st)) + ": " + tsgne_last_error(nullptr));
    }
    s->cv_ready.notify_all();
  }
}

// Attaches the members the worker has prepared.  wait_all: first wait until
// every admitted request has come back (used when nothing is resident: the
// GPU has nothing else to do, and the selection then sees every admitted
// request, as it would without the worker).
tsgne_status attach_ready(tsgne_server* s, bool wait_all) {
  std::vector<std::pair<int64_t, tsgne_member*>> got;
  std::vector<std::pair<int64_t, std::string>> bad;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    if (wait_all) {
      const size_t want = (size_t)s->preparing;
      s->cv_ready.wait(lk, [s, want] { return s->ready.size() + s->failed.size() >= want; });
    }
    got.swap(s->ready);
    bad.swap(s->failed);
  }
  tsgne_status first_err = TSGNE_OK;
  for (auto& f : bad) {
    Req& r = s->reqs[f.first];
    --s->preparing;
    s->used -= r.bytes;
    const bool was_cancelled = r.state == kCancelled;
    r.state = kCancelled;  // its result reports CANCELLED; the tick reports why
    if (!was_cancelled && first_err == TSGNE_OK) {
      s->msg = "building request " + std::to_string(f.first) + " failed: " + f.second;
      first_err = TSGNE_ERR_CUDA;
    }
  }
  for (auto& g : got) {
    Req& r = s->reqs[g.first];
    --s->preparing;
    if (r.state == kCancelled) {  // cancelled while it was being prepared
      tsgne_batch_discard(g.second);
      s->used -= r.bytes;
      continue;
    }
    int32_t mid = -1;
    const tsgne_status st = tsgne_batch_attach(s->batch, g.second, &mid);
    if (st != TSGNE_OK) return batch_fail(s, st);
    r.member = mid;
    r.state = kResident;
    std::vector<int64_t>().swap(r.rp);  // the batch holds its own copy now
    std::vector<int32_t>().swap(r.col);
    std::vector<float>().swap(r.X);
    std::vector<float>().swap(r.Y0);
  }
  return first_err;
}

}  // namespace

extern "C" {

void tsgne_server_config_default(tsgne_server_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->budget_bytes = (int64_t)80 << 30;
  c->iters = 500;
  c->tick_iters = 10;
  c->max_members = 256;
  c->tile_warps = 2;
  c->policy = 1;
  c->aging_ticks = 20;
  c->fill_pairs = 4e9;
  c->tree_min_n = 0;
}

int64_t tsgne_server_estimate_bytes(int32_t n, int64_t nnz, int32_t tile_warps) {
  if (n < 1 || nnz < 0 || tile_warps < 1) return -1;
  const int64_t T = 512 * (int64_t)tile_warps;  // the batch tile: 32 lanes x 16 i-points per warp
  const int64_t n_pad_max = (n + 2047) / 2048 * 2048;
  const int64_t nt = (n + T - 1) / T;
  const int64_t units = nt * (nt + 1) / 2;
  // hub rows (more than 32 entries: at most nnz / 33 of them) and their
  // 1024-entry chunks: 12 B per row, 32 B per chunk
  const int64_t hub_rows = nnz / 33 + 1, hub_chunks = nnz / 1024 + hub_rows;
  // row_ptr, col + P, Y x 2 / update / gains / F^r (n_pad_max float2 each),
  // the initial layout, the fixed-point force accumulators (16 B per
  // point), the unit Z partials, the hub-row chunk lists
  return 8 * ((int64_t)n + 1) + 8 * nnz + 5 * 8 * n_pad_max + 8 * (int64_t)n + 16 * (int64_t)n + 8 * units +
         12 * hub_rows + 32 * hub_chunks + 256;
}

tsgne_status tsgne_server_create(tsgne_server** out, const tsgne_server_config* scfg, const tsgne_config* cfg,
                                 void* cuda_stream) {
  if (!out) return TSGNE_ERR_INVALID_ARG;
  *out = nullptr;
  tsgne_server_config c;
  if (scfg) c = *scfg; else tsgne_server_config_default(&c);
  if (c.iters < 1 || c.tick_iters < 1 || c.iters % c.tick_iters != 0 || c.max_members < 1 || c.budget_bytes < 1 ||
      !(c.tile_warps == 1 || c.tile_warps == 2 || c.tile_warps == 4) ||
      !(c.policy == 0 || c.policy == 1) || c.aging_ticks < 0 || !(c.fill_pairs > 0.0) || c.tree_min_n < 0)
    return TSGNE_ERR_INVALID_ARG;
  tsgne_server* s = new (std::nothrow) tsgne_server();
  if (!s) return TSGNE_ERR_OOM;
  s->cfg = c;
  const tsgne_status st = tsgne_batch_create(&s->batch, cfg, c.tile_warps, cuda_stream);
  if (st != TSGNE_OK) {
    delete s;
    return st;
  }
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->prep, cudaStreamNonBlocking) != cudaSuccess) {
    tsgne_batch_destroy(s->batch);
    delete s;
    return TSGNE_ERR_CUDA;
  }
  try {
    s->worker = std::thread(worker_main, s);
  } catch (...) {
    tsgne_batch_destroy(s->batch);
    cudaStreamDestroy(s->prep);
    delete s;
    return TSGNE_ERR_OOM;
  }
  *out = s;
  return TSGNE_OK;
}

void tsgne_server_destroy(tsgne_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& g : s->ready) tsgne_batch_discard(g.second);
  tsgne_batch_destroy(s->batch);  // frees members whose memory is ordered on prep
  if (s->prep) {
    cudaStreamSynchronize(s->prep);
    cudaStreamDestroy(s->prep);
  }
  delete s;
}

const char* tsgne_server_last_error(const tsgne_server* s) { return s ? s->msg.c_str() : ""; }

tsgne_status tsgne_server_submit(tsgne_server* s, int32_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                 const float* X, int32_t d, const float* Y0, int64_t* request_id) {
  if (!s) return TSGNE_ERR_INVALID_ARG;
  if (n < 2 || d < 1 || !row_ptr || !X || !request_id)
    return sfail(s, TSGNE_ERR_INVALID_ARG, "need n >= 2, d >= 1, row_ptr, X and request_id");
  const int64_t m = row_ptr[n];
  if (row_ptr[0] != 0 || m < 0) return sfail(s, TSGNE_ERR_BAD_CSR, "row_ptr[0] must be 0 and row_ptr[n] >= 0");
  for (int32_t i = 0; i < n; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return sfail(s, TSGNE_ERR_BAD_CSR, "row_ptr decreases");
  if (m > 0 && !col_idx) return sfail(s, TSGNE_ERR_INVALID_ARG, "col_idx is NULL");
  for (int64_t e = 0; e < m; ++e)
    if (col_idx[e] < 0 || col_idx[e] >= n) return sfail(s, TSGNE_ERR_BAD_CSR, "column outside [0, n)");
  Req r;
  r.id = s->next_id++;
  r.n = n;
  r.d = d;
  try {
    r.rp.assign(row_ptr, row_ptr + n + 1);
    if (m > 0) r.col.assign(col_idx, col_idx + m);
    r.X.assign(X, X + (size_t)n * d);
    if (Y0) r.Y0.assign(Y0, Y0 + 2 * (size_t)n);
    std::lock_guard<std::mutex> lk(s->mu);
    s->queue.push_back(r.id);
    s->reqs.emplace(r.id, std::move(r));
  } catch (const std::bad_alloc&) {
    return sfail(s, TSGNE_ERR_OOM, "host memory for the request");
  }
  *request_id = s->next_id - 1;
  return TSGNE_OK;
}

tsgne_status tsgne_server_tick(tsgne_server* s, int32_t* resident, int32_t* queued, int32_t* retired) {
  if (!s) return TSGNE_ERR_INVALID_ARG;
  {
    tsgne_status st = attach_ready(s, false);
    if (st == TSGNE_OK) st = admit(s);
    if (st != TSGNE_OK) return st;
    int32_t nres = 0;
    for (const auto& kv : s->reqs) nres += kv.second.state == kResident;
    if (nres == 0 && s->preparing > 0) st = attach_ready(s, true);  // nothing else to run meanwhile
    if (st != TSGNE_OK) return st;
  }
  // (aged first, -ticks waited, remaining work, id): the overdue layouts
  // longest waiting first, then shortest remaining work first
  std::vector<std::pair<std::tuple<int, int, double>, int64_t>> order;
  const int aging = s->cfg.aging_ticks;
  for (const auto& kv : s->reqs)
    if (kv.second.state == kResident) {
      const Req& r = kv.second;
      const bool overdue = aging > 0 && r.waited >= aging;
      order.push_back({std::make_tuple(overdue ? 0 : 1, overdue ? -r.waited : 0,
                                       (double)(s->cfg.iters - r.iters) * iter_pairs(r)),
                       kv.first});
    }
  std::vector<std::pair<double, int64_t>> res;  // selection order
  int32_t done_now = 0;
  if (!order.empty()) {
    std::sort(order.begin(), order.end());
    for (const auto& o : order) res.emplace_back(std::get<2>(o.first), o.second);
    std::vector<int64_t> chosen;
    double pairs = 0.0;
    for (const auto& w : res) {
      chosen.push_back(w.second);
      pairs += iter_pairs(s->reqs[w.second]);
      if (s->cfg.policy == 1 && pairs >= s->cfg.fill_pairs) break;
    }
    for (const auto& w : res) {
      const bool want = std::find(chosen.begin(), chosen.end(), w.second) != chosen.end();
      Req& r = s->reqs[w.second];
      r.waited = want ? 0 : r.waited + 1;
      const tsgne_status st = tsgne_batch_set_active(s->batch, r.member, want ? 1 : 0);
      if (st != TSGNE_OK) return batch_fail(s, st);
    }
    tsgne_status st = tsgne_batch_run(s->batch, s->cfg.tick_iters);
    if (st != TSGNE_OK) return batch_fail(s, st);
    for (int64_t id : chosen) {
      Req& r = s->reqs[id];
      r.iters += s->cfg.tick_iters;
      if (r.iters < s->cfg.iters) continue;
      try {
        r.Y.resize(2 * (size_t)r.n);
      } catch (const std::bad_alloc&) {
        return sfail(s, TSGNE_ERR_OOM, "host memory for a result");
      }
      int32_t it = 0;
      st = tsgne_batch_get_Y(s->batch, r.member, r.Y.data(), &it, TSGNE_PTR_HOST);
      if (st != TSGNE_OK) return batch_fail(s, st);
      r.iters = it;  // the member's own device counter
      st = tsgne_batch_remove(s->batch, r.member);
      if (st != TSGNE_OK) return batch_fail(s, st);
      r.state = kDone;
      r.member = -1;
      s->used -= r.bytes;
      s->finished.push_back(id);
      ++done_now;
    }
  }
  int32_t nres = 0;
  for (const auto& kv : s->reqs) nres += kv.second.state == kResident;
  if (resident) *resident = nres;
  if (queued) *queued = (int32_t)s->queue.size() + s->preparing;
  if (retired) *retired = done_now;
  return TSGNE_OK;
}

tsgne_status tsgne_server_finished(tsgne_server* s, int64_t* ids, int32_t capacity, int32_t* count) {
  if (!s || !count || capacity < 0 || (capacity > 0 && !ids)) return TSGNE_ERR_INVALID_ARG;
  const int32_t k = std::min<int32_t>(capacity, (int32_t)s->finished.size());
  for (int32_t i = 0; i < k; ++i) ids[i] = s->finished[i];
  s->finished.erase(s->finished.begin(), s->finished.begin() + k);
  *count = k;
  return TSGNE_OK;
}

tsgne_status tsgne_server_status(tsgne_server* s, int64_t request_id, int32_t* state, int32_t* iterations) {
  if (!s) return TSGNE_ERR_INVALID_ARG;
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return sfail(s, TSGNE_ERR_INVALID_ARG, "unknown request id");
  if (state) *state = it->second.state == kPreparing ? kQueued : it->second.state;
  if (iterations) *iterations = it->second.iters;
  return TSGNE_OK;
}

tsgne_status tsgne_server_result(tsgne_server* s, int64_t request_id, float* Y_out) {
  if (!s) return TSGNE_ERR_INVALID_ARG;
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return sfail(s, TSGNE_ERR_INVALID_ARG, "unknown request id");
  Req& r = it->second;
  if (r.state == kCancelled) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->reqs.erase(it);
    return sfail(s, TSGNE_ERR_CANCELLED, "the request was cancelled");
  }
  if (r.state != kDone) return sfail(s, TSGNE_ERR_NOT_BUILT, "the request has not finished");
  if (!Y_out) return sfail(s, TSGNE_ERR_INVALID_ARG, "Y_out is NULL");
  std::memcpy(Y_out, r.Y.data(), sizeof(float) * r.Y.size());
  std::lock_guard<std::mutex> lk(s->mu);
  s->reqs.erase(it);
  return TSGNE_OK;
}

tsgne_status tsgne_server_cancel(tsgne_server* s, int64_t request_id) {
  if (!s) return TSGNE_ERR_INVALID_ARG;
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return sfail(s, TSGNE_ERR_INVALID_ARG, "unknown request id");
  Req& r = it->second;
  if (r.state == kQueued) {
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), request_id));
  } else if (r.state == kPreparing) {
    // the worker may be building it: its member is discarded (and its bytes
    // returned) when it comes back, or now if the worker has not taken it
    std::lock_guard<std::mutex> lk(s->mu);
    auto q = std::find(s->prep_q.begin(), s->prep_q.end(), request_id);
    if (q != s->prep_q.end()) {
      s->prep_q.erase(q);
      --s->preparing;
      s->used -= r.bytes;
    }
    r.state = kCancelled;
    return TSGNE_OK;
  } else if (r.state == kResident) {
    const tsgne_status st = tsgne_batch_remove(s->batch, r.member);
    if (st != TSGNE_OK) return batch_fail(s, st);
    s->used -= r.bytes;
    r.member = -1;
  } else {
    return sfail(s, TSGNE_ERR_INVALID_ARG, "the request has already finished or been cancelled");
  }
  r.state = kCancelled;
  std::vector<int64_t>().swap(r.rp);
  std::vector<int32_t>().swap(r.col);
  std::vector<float>().swap(r.X);
  std::vector<float>().swap(r.Y0);
  return TSGNE_OK;
}

tsgne_status tsgne_server_usage(tsgne_server* s, int64_t* used_bytes, int32_t* resident, int32_t* queued) {
  if (!s) return TSGNE_ERR_INVALID_ARG;
  int32_t nres = 0;
  for (const auto& kv : s->reqs) nres += kv.second.state == kResident;
  if (used_bytes) *used_bytes = s->used;
  if (resident) *resident = nres;
  if (queued) *queued = (int32_t)s->queue.size() + s->preparing;
  return TSGNE_OK;
}

}  // extern "C"
