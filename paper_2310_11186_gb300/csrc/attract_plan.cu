// Attraction + update (S3 + S5 fused) on a schedule fixed when P is
// installed.  The terms and the order in which each row adds them are those
// of k_attract (iterate.cu) -- the definition the gradient export, the batch
// engine and the oracle parity tests share -- so the results are the same
// bits; what changes is how the work is laid out over threads.
//
// The order of a row's sum, by degree d:
//   d <= 32:   8 slot chains, slot s adding entries s, s + 8, ... in order
//              (at most 4), then the 8 slots in xor-butterfly order;
//   d > 32:    chunks of 1024 entries; within a chunk 32 lane chains, lane l
//              adding entries l, l + 32, ... in order, then the 32 lanes in
//              xor-butterfly order; the chunk sums in chunk order.
// A row of 33 to 128 entries is one chunk whose lane chains hold at most 4
// entries.  One warp per such row leaves most lanes with one or two entries
// and pays the warp's fixed costs per row; R-MAT 2^21 has 122,000 of them.
// So rows up to 128 entries are cut into their chains ("pairs" of row and
// slot: 8 per row up to 32 entries, 32 per row above), one thread per chain,
// and rows above 128 entries keep one warp per chunk.
//
// The schedule (built on the host from row_ptr, once per P):
//   short CTAs  rows [256 c, 256 c + 256): the chains of their rows of at most
//               32 entries; then one thread per row adds its 8 slots and
//               updates the row (rows above 32 entries are left to the others;
//               rows without entries get F^a = 0);
//   medium CTAs up to 64 rows of 33..128 entries (listed): their 32 chains
//               each; then one warp per row adds the 32 chains with the same
//               shuffle butterfly the chunk warps use, and one thread per row
//               updates it;
//   big CTAs    one warp per 1024-entry chunk of the rows above 128 entries,
//               as k_attract's fused hub branch.
// Within a CTA the chains are sorted by length (longest first), so the chains
// still running at level k are a prefix [0, cnt[k]) of the list and entry k
// of chain q sits at ent + off[k] + q in copies of col and P made in that
// order: every level's loads are coalesced, and each thread issues the loads
// of all entries of its chain before the first gather returns.  A CTA starts
// by prefetching into L2 the streams it reads (chain codes, col and P in chain
// order, its rows' optimiser state; a hub chunk's col and P).
#include <algorithm>
#include <cstring>
#include <vector>

#include "row_update.cuh"
#include "storage.cuh"
#include "tsgne_internal.cuh"

namespace tsgne {

namespace {

constexpr int kPlanThreads = 256;
constexpr int kShortRowsPerCta = 256;
constexpr int kMedRowsPerCta = 64;
constexpr int kSlotsShort = 8;
constexpr int kSlotsMed = 32;
static_assert(kShortRowsPerCta * kSlotsShort == kMedRowsPerCta * kSlotsMed, "one shared partial array");
constexpr int kPartials = kShortRowsPerCta * kSlotsShort;  // 2048

// L2 prefetch of the 128-byte lines of [lo, hi), spread over nt threads; every
// address touched lies inside the range.  A hint: the CTA's streams (chain
// codes, col and P in chain order, the rows' optimiser state; a hub chunk's
// col and P) are on their way from DRAM while its first gathers run.
template <class T>
__device__ __forceinline__ void prefetch_range(const T* lo, const T* hi, int t, int nt) {
  const uintptr_t a = (uintptr_t)lo, b = (uintptr_t)hi;
  for (uintptr_t q = (a & ~(uintptr_t)127) + (uintptr_t)t * 128; q < b; q += (uintptr_t)nt * 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(q < a ? a : q));
}

// One entry's term of F^a, as attract_entries adds it.
template <class PT, class YT>
__device__ __forceinline__ void add_term(float2 yi, float2 yj, float p, float& ax, float& ay) {
  const float dx = yi.x - yj.x, dy = yi.y - yj.y;
  const float w = 1.0f / fmaf(dy, dy, fmaf(dx, dx, 1.0f));
  const float pw = p * w;
  ax = fmaf(pw, dx, ax);
  ay = fmaf(pw, dy, ay);
}

template <class PT, class YT>
__global__ void __launch_bounds__(kPlanThreads, 6)
    k_attract_plan(AttractArgs a, PlanView pv, int big_blocks) {
  __shared__ float2 spart[kPartials];
  __shared__ float2 sfa[kMedRowsPerCta];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const PT* __restrict__ P = static_cast<const PT*>(a.P);
  const YT* __restrict__ Y = static_cast<const YT*>(a.Yr);
  bf162* Ynext16 = static_cast<bf162*>(a.Ynext16);
  uint32_t* dbg = &a.sched->flags;  // index checks of the debug build
  (void)dbg;

  if ((int)blockIdx.x < big_blocks) {  // one warp per chunk of a row above 128 entries
    const HeavyRows& hv = a.hv;
    const int stride = big_blocks * (kPlanThreads / 32);
    for (int k = blockIdx.x * (kPlanThreads / 32) + warp; k < pv.n_big; k += stride) {
      const int c = pv.big[k];
      if (!TS_IN(c, 0, hv.chunks, dbg)) continue;
      const int64_t i = hv.chunk_row[c];
      if (!TS_IN(i, 0, a.n, dbg)) continue;
      prefetch_range(a.col + hv.chunk_begin[c], a.col + hv.chunk_end[c], lane, 32);
      prefetch_range(P + hv.chunk_begin[c], P + hv.chunk_end[c], lane, 32);
      float ax = 0.f, ay = 0.f;
      attract_entries<32, PT, YT>(hv.chunk_begin[c], hv.chunk_end[c], a.col, P, Y, i, lane, ld_y(Y, i), ax, ay,
                                  a.n, dbg);
      ax = group_sum<32>(ax);
      ay = group_sum<32>(ay);
      if (lane == 0) {
        hv.fa[c] = make_float2(ax, ay);
        const int h = hv.chunk_heavy[c];
        const int c0 = hv.chunk_off[h], c1 = hv.chunk_off[h + 1];
        if (atom_add_acq_rel_u32(&hv.arrivals[h], 1u) == (unsigned)(c1 - c0 - 1)) {  // last chunk of the row
          hv.arrivals[h] = 0u;
          float sx = 0.f, sy = 0.f;
          for (int q = c0; q < c1; ++q) {
            const float2 f = __ldcg(hv.fa + q);
            sx += f.x;
            sy += f.y;
          }
          finish_row<false>(i, make_float2(sx, sy), a.frep, a.chunks, a.n_pad, a.sched, 0.f, nullptr, a.Ym,
                            a.Ynext, Ynext16, a.upd, a.gains, a.eta, a.min_gain);
        }
      }
    }
    return;
  }

  const int cb = (int)blockIdx.x - big_blocks;
  const bool med = cb < pv.n_med;
  const PlanCta m = med ? pv.med[cb] : pv.shorts[cb - pv.n_med];
  const int shift = med ? 5 : 3;
  const int64_t row0 = med ? 0 : (int64_t)(cb - pv.n_med) * kShortRowsPerCta;
  {
    const int64_t tot = (int64_t)m.cnt[0] + m.cnt[1] + m.cnt[2] + m.cnt[3];
    prefetch_range(pv.code + m.pair, pv.code + m.pair + m.cnt[0], tid, kPlanThreads);
    prefetch_range(pv.colS + m.ent, pv.colS + m.ent + tot, tid, kPlanThreads);
    const PT* PS = static_cast<const PT*>(pv.PS);
    prefetch_range(PS + m.ent, PS + m.ent + tot, tid, kPlanThreads);
  }
  if (!med) {
    const int64_t r1 = row0 + kShortRowsPerCta < a.n ? row0 + kShortRowsPerCta : a.n;
    prefetch_range(a.rp + row0, a.rp + r1 + 1, tid, kPlanThreads);
    prefetch_range(a.frep + row0, a.frep + r1, tid, kPlanThreads);
    prefetch_range(a.upd + row0, a.upd + r1, tid, kPlanThreads);
    prefetch_range(a.gains + row0, a.gains + r1, tid, kPlanThreads);
    prefetch_range(a.Ym + row0, a.Ym + r1, tid, kPlanThreads);
  }
  for (int k = tid; k < kPartials; k += kPlanThreads) spart[k] = make_float2(0.f, 0.f);
  __syncthreads();

  // the chains: thread per chain, every entry's loads issued up front
  const int64_t off1 = m.cnt[0], off2 = off1 + m.cnt[1], off3 = off2 + m.cnt[2];
  for (int q = tid; q < m.cnt[0]; q += kPlanThreads) {
    if (!TS_IN(m.pair + q, 0, pv.n_codes, dbg)) continue;
    const int code = pv.code[m.pair + q];
    const int r = code >> shift, s = code & ((1 << shift) - 1);
    if (!TS_IN(r, 0, m.nrows, dbg) || (med && !TS_IN(m.rows + r, 0, pv.n_med_rows, dbg))) continue;
    const int64_t i = med ? (int64_t)pv.med_rows[m.rows + r] : row0 + r;
    if (!TS_IN(i, 0, a.n, dbg)) continue;
    const int depth = 1 + (q < m.cnt[1]) + (q < m.cnt[2]) + (q < m.cnt[3]);
    const int64_t e[4] = {m.ent + q, m.ent + off1 + q, m.ent + off2 + q, m.ent + off3 + q};
    int32_t j[4];
    float p[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool ld = k < depth && TS_IN(e[k], 0, pv.entries, dbg);
      j[k] = ld ? pv.colS[e[k]] : (int32_t)i;
      p[k] = ld ? ld_p(static_cast<const PT*>(pv.PS), e[k]) : 0.f;
      if (!TS_IN(j[k], 0, a.n, dbg)) j[k] = (int32_t)i;
    }
    const float2 yi = ld_y(Y, i);
    float2 yj[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) yj[k] = ld_y(Y, j[k]);
    float ax = 0.f, ay = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < depth) add_term<PT, YT>(yi, yj[k], p[k], ax, ay);
    spart[(r << shift) + s] = make_float2(ax, ay);
  }
  __syncthreads();

  if (!med) {  // one thread per row of at most 32 entries: slots in butterfly order, then the update
    const int64_t i = row0 + tid;
    if (i >= a.n) return;
    if (a.rp[i + 1] - a.rp[i] > kHeavyDeg) return;  // a medium or big CTA updates it
    const float2* sp = spart + tid * kSlotsShort;
    float2 a0 = sp[0], a1 = sp[1], t = sp[4];
    a0 = make_float2(a0.x + t.x, a0.y + t.y);  // o = 4
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
    finish_row<false>(i, fa, a.frep, a.chunks, a.n_pad, a.sched, 0.f, nullptr, a.Ym, a.Ynext, Ynext16, a.upd,
                      a.gains, a.eta, a.min_gain);
    return;
  }
  // medium rows: the 32 chains of a row with the chunk warps' shuffle
  // butterfly, then (one chunk) its sum starting from 0 as the chunk-sum loop
  for (int r = warp; r < m.nrows; r += kPlanThreads / 32) {
    const float2 v = spart[r * kSlotsMed + lane];
    const float ax = group_sum<32>(v.x), ay = group_sum<32>(v.y);
    if (lane == 0) sfa[r] = make_float2(0.f + ax, 0.f + ay);
  }
  __syncthreads();
  if (tid < m.nrows && TS_IN(m.rows + tid, 0, pv.n_med_rows, dbg))
    finish_row<false>(pv.med_rows[m.rows + tid], sfa[tid], a.frep, a.chunks, a.n_pad, a.sched, 0.f, nullptr, a.Ym,
                      a.Ynext, Ynext16, a.upd, a.gains, a.eta, a.min_gain);
}

template <class PT>
__global__ void k_plan_gather(int64_t count, const int64_t* __restrict__ perm, const int32_t* __restrict__ col,
                              const PT* __restrict__ P, int32_t* __restrict__ colS, PT* __restrict__ PS) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) {
    const int64_t e = perm[k];
    colS[k] = col[e];
    PS[k] = P[e];
  }
}

// Chains of one CTA's rows: codes sorted longest first, per-level counts, and
// the entry positions of level k, chain q (in that order) appended to perm.
void plan_cta(const std::vector<int64_t>& rp, const std::vector<int64_t>& rows, int slots, int shift,
              std::vector<uint16_t>& code, std::vector<int64_t>& perm, PlanCta& pc) {
  std::vector<uint16_t> by[4];
  std::vector<int64_t> first[4];
  for (size_t r = 0; r < rows.size(); ++r) {
    const int64_t i = rows[r];
    if (i < 0) continue;
    const int64_t d = rp[i + 1] - rp[i];
    for (int s = 0; s < slots && s < d; ++s) {
      const int depth = (int)((d - s + slots - 1) / slots);  // 1..4
      by[depth - 1].push_back((uint16_t)((r << shift) | (size_t)s));
      first[depth - 1].push_back(rp[i] + s);
    }
  }
  pc.pair = (int32_t)code.size();
  pc.ent = (int64_t)perm.size();
  std::vector<int64_t> start;
  for (int dep = 3; dep >= 0; --dep) {
    code.insert(code.end(), by[dep].begin(), by[dep].end());
    start.insert(start.end(), first[dep].begin(), first[dep].end());
  }
  const int64_t total = (int64_t)start.size();
  pc.cnt[0] = (int32_t)total;
  for (int k = 1; k < 4; ++k) {
    int64_t c = 0;
    for (int dep = k; dep < 4; ++dep) c += (int64_t)by[dep].size();
    pc.cnt[k] = (int32_t)c;
  }
  for (int k = 0; k < 4; ++k)
    for (int32_t q = 0; q < pc.cnt[k]; ++q) perm.push_back(start[q] + (int64_t)slots * k);
}

}  // namespace

tsgne_status build_attract_plan(int n, const int64_t* rp_dev, const int32_t* col_dev, const float* P_dev,
                                const bf16* P16_dev, const HeavyStore& hs, AttractPlan& plan, cudaStream_t s) {
  plan = AttractPlan();
  std::vector<int64_t> rp((size_t)n + 1);
  TS_CUDA(cudaMemcpyAsync(rp.data(), rp_dev, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost, s));
  TS_CUDA(cudaStreamSynchronize(s));
  std::vector<uint16_t> code;
  std::vector<int64_t> perm;
  std::vector<PlanCta> med, shorts;
  std::vector<int32_t> med_rows, big;
  // medium rows (33..128 entries), 64 per CTA; big rows' chunks
  int32_t chunk = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t d = rp[i + 1] - rp[i];
    if (d <= kHeavyDeg) continue;
    const int32_t nch = (int32_t)((d + kHeavyChunk - 1) / kHeavyChunk);
    if (d <= kMedDeg) {
      med_rows.push_back((int32_t)i);
    } else {
      for (int32_t k = 0; k < nch; ++k) big.push_back(chunk + k);
    }
    chunk += nch;
  }
  if (chunk != hs.chunks) {
    last_msg() = "attraction plan: chunk count differs from the hub-row store";
    return TSGNE_ERR_CUDA;
  }
  for (size_t r0 = 0; r0 < med_rows.size(); r0 += kMedRowsPerCta) {
    const size_t r1 = std::min(med_rows.size(), r0 + kMedRowsPerCta);
    std::vector<int64_t> rows(med_rows.begin() + (long)r0, med_rows.begin() + (long)r1);
    PlanCta pc{};
    plan_cta(rp, rows, kSlotsMed, 5, code, perm, pc);
    pc.rows = (int32_t)r0;
    pc.nrows = (int32_t)(r1 - r0);
    med.push_back(pc);
  }
  for (int64_t r0 = 0; r0 < n; r0 += kShortRowsPerCta) {
    std::vector<int64_t> rows;
    for (int64_t i = r0; i < std::min<int64_t>(n, r0 + kShortRowsPerCta); ++i)
      rows.push_back(rp[i + 1] - rp[i] <= kHeavyDeg ? i : -1);
    PlanCta pc{};
    plan_cta(rp, rows, kSlotsShort, 3, code, perm, pc);
    pc.nrows = (int32_t)rows.size();
    shorts.push_back(pc);
  }
  plan.n_med = (int)med.size();
  plan.n_short = (int)shorts.size();
  plan.n_big = (int)big.size();
  plan.entries = (int64_t)perm.size();
  plan.n_codes = (int64_t)code.size();
  plan.n_med_rows = (int64_t)med_rows.size();
  std::vector<PlanCta> ctas(med);
  ctas.insert(ctas.end(), shorts.begin(), shorts.end());
  TS_TRY(plan.cta.alloc(ctas.size()));
  TS_TRY(plan.code.alloc(code.size()));
  TS_TRY(plan.med_rows.alloc(med_rows.size()));
  TS_TRY(plan.big.alloc(big.size()));
  TS_TRY(plan.colS.alloc((size_t)plan.entries));
  DevBuf<int64_t> dperm;
  TS_TRY(dperm.alloc((size_t)plan.entries));
  TS_CUDA(cudaMemcpyAsync(plan.cta.get(), ctas.data(), sizeof(PlanCta) * ctas.size(), cudaMemcpyHostToDevice, s));
  if (!code.empty())
    TS_CUDA(cudaMemcpyAsync(plan.code.get(), code.data(), sizeof(uint16_t) * code.size(), cudaMemcpyHostToDevice, s));
  if (!med_rows.empty())
    TS_CUDA(cudaMemcpyAsync(plan.med_rows.get(), med_rows.data(), sizeof(int32_t) * med_rows.size(),
                            cudaMemcpyHostToDevice, s));
  if (!big.empty())
    TS_CUDA(cudaMemcpyAsync(plan.big.get(), big.data(), sizeof(int32_t) * big.size(), cudaMemcpyHostToDevice, s));
  if (plan.entries > 0)
    TS_CUDA(cudaMemcpyAsync(dperm.get(), perm.data(), sizeof(int64_t) * perm.size(), cudaMemcpyHostToDevice, s));
  const int g = (int)std::min<int64_t>(8192, std::max<int64_t>(1, (plan.entries + 255) / 256));
  if (P16_dev) {
    TS_TRY(plan.PS16.alloc((size_t)plan.entries));
    if (plan.entries > 0)
      k_plan_gather<bf16><<<g, 256, 0, s>>>(plan.entries, dperm.get(), col_dev, P16_dev, plan.colS.get(),
                                            plan.PS16.get());
  } else {
    TS_TRY(plan.PS.alloc((size_t)plan.entries));
    if (plan.entries > 0)
      k_plan_gather<float><<<g, 256, 0, s>>>(plan.entries, dperm.get(), col_dev, P_dev, plan.colS.get(),
                                             plan.PS.get());
  }
  TS_CUDA(cudaGetLastError());
  TS_CUDA(cudaStreamSynchronize(s));  // dperm is freed on return
  plan.ready = true;
  return TSGNE_OK;
}

PlanView AttractPlan::view() const {
  PlanView v;
  v.med = cta.get();
  v.shorts = cta.get() + n_med;
  v.code = code.get();
  v.colS = colS.get();
  v.PS = PS16.get() ? (const void*)PS16.get() : (const void*)PS.get();
  v.med_rows = med_rows.get();
  v.big = big.get();
  v.n_med = n_med;
  v.n_short = n_short;
  v.n_big = n_big;
  v.entries = entries;
  v.n_codes = n_codes;
  v.n_med_rows = n_med_rows;
  return v;
}

tsgne_status launch_attract_plan(const AttractArgs& a, const PlanView& pv, cudaStream_t s) {
  int big_blocks = (pv.n_big + kPlanThreads / 32 - 1) / (kPlanThreads / 32);
  if (big_blocks > 4096) big_blocks = 4096;
  const int grid = big_blocks + pv.n_med + pv.n_short;
  if (grid <= 0) return TSGNE_OK;
  if (a.p_bf16 && a.y_bf16)
    k_attract_plan<bf16, bf162><<<grid, kPlanThreads, 0, s>>>(a, pv, big_blocks);
  else if (!a.p_bf16 && !a.y_bf16)
    k_attract_plan<float, float2><<<grid, kPlanThreads, 0, s>>>(a, pv, big_blocks);
  else {
    last_msg() = "P and Y must share a storage precision";
    return TSGNE_ERR_INVALID_ARG;
  }
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

}  // namespace tsgne
