// Symmetric exact repulsion (Sec. 2.1, Eq. 4): each unordered pair {i, j} is
// evaluated once and its force is applied to both points,
//   w = (1 + ||y_i - y_j||^2)^-1,  F^r_i += w^2 (y_i - y_j),  F^r_j -= w^2 (y_i - y_j),
//   Z += 2 w  (Z sums ordered pairs k != l).
// Per unordered pair this is 10 FP32 lane-ops and one MUFU reciprocal, i.e.
// 5 lane-ops and half a reciprocal per ordered pair (the ordered kernel in
// repulsion.cu spends 8 and 1).  Forces go to per-point fixed-point
// accumulators with integer atomics (sym_unit.cuh), so the pass needs 16
// bytes per point whatever the number of tiles, and its result does not
// depend on the order in which units finish.
//
// Decomposition.  Points are padded to n_pad = nt * T (T = 512 W) with the
// sentinel point.  A unit of work is a tile pair (a, b), a <= b; the units
// are enumerated row by row and taken from a global work queue by a
// persistent grid (8 warps per SM; 2-warp CTAs once there are enough units,
// else 1-warp CTAs).  Sixteen i-points per lane and few warps beat eight
// i-points and 24 warps per SM on GB300: the longer independent chains per
// lane hide the reciprocal latency better than more warps do.  Unit (a, b),
// a < b, adds the forces of tile a's points and of tile b's points into
// their accumulators; the diagonal unit (t, t) evaluates its ordered pairs
// with the i-side only.  Each unit also writes its own FP64 Z partial; the
// last CTA adds them in unit order, removes the n self terms w_ii = 1 and
// sets the iteration schedule.
//
// Inside a unit (a < b).  Each of the W warps holds 512 points of tile a in
// registers (16 per lane, as eight FP32x2 pairs).  Tile b sits in shared
// memory as {-x, -x, -y, -y} plus an FP32 force accumulator per point, cut
// into 8W groups of 64 points.  In phase p warp w works on group (w + p) mod
// 8W, so no two warps touch the same accumulators at once and no atomics are
// needed.  Within a warp, lane l starts with the accumulators of the group's
// points 2l and 2l+1; each of 32 steps evaluates the lane's 16 i-points
// against those 2 j-points, then passes the j accumulators one lane down the
// ring (shuffle); after 32 steps every j has met all 512 i of the warp and
// its accumulators are back home.  Only sentinel points lie in the last tile,
// and a < b means tile a never holds any, so sentinel-sentinel pairs (w = 1)
// occur only in the diagonal unit, where they are masked out of Z.
#include "f32x2.cuh"
#include "reduce.cuh"
#include "sym_unit.cuh"
#include "tsgne_internal.cuh"

namespace tsgne {

namespace {

// Z and the schedule of the iteration from the unit partials: the fixed-order
// sum of zunit[0..units) minus the n self terms; alpha / mu for iteration
// sched->t, which advance != 0 increments.  Called by every thread of one CTA
// (the last one of the pass, or the finalize launch of a sharded pass: with
// the same block size both give the same bits).
__device__ __forceinline__ void finalize_z(const double* zunit, int units, int n, Sched* sched, int advance,
                                           float ee, int ee_iters, float mom0, float mom1) {
  const double total = sum_partials(zunit, units);
  if (threadIdx.x == 0) {
    sched->work_next = 0u;
    sched->Z = total - (double)n;
    sched->inv_z = (float)(1.0 / sched->Z);
    const int t = sched->t;
    sched->alpha = t < ee_iters ? ee : 1.0f;
    sched->mu = t < ee_iters ? mom0 : mom1;
    if (advance) sched->t = t + 1;
  }
}

// Units [u0, u1) of the nt (nt + 1) / 2 tile pairs (all of them on one GPU;
// one rank's share when the pass is sharded).  finalize != 0: the last CTA
// also sets Z and the schedule (one GPU); else the caller sums the unit
// partials over the ranks and launches k_finalize_z.
template <int W, int RI, class YT>
__global__ void __launch_bounds__(W * 32, warps_per_sm(RI) / W)
    k_repulsion_sym(const YT* __restrict__ Y, int n, int nt, unsigned long long* __restrict__ acc, float fscale,
                    double* __restrict__ zunit, Sched* sched, int u0, int u1, int finalize, int advance, float ee,
                    int ee_iters, float mom0, float mom1) {
  constexpr int T = W * 32 * RI;
  extern __shared__ float4 smem[];
  float4* sj = smem;                                   // T x {-x, -x, -y, -y}
  float2* sacc = reinterpret_cast<float2*>(smem + T);  // T x force accumulator
  __shared__ int s_unit, s_a, s_b;
  const int tid = threadIdx.x;
  const int units = nt * (nt + 1) / 2;

  for (;;) {
    if (tid == 0) {
      const int u = u0 + (int)atomicAdd(&sched->work_next, 1u);
      int a = 0, b = 0;
      if (u < u1) unit_tiles(u, nt, &a, &b);
      s_unit = u;
      s_a = a;
      s_b = b;
    }
    __syncthreads();
    const int u = s_unit, a = s_a, b = s_b;
    if (u >= u1) break;
    if (!(TS_IN(a, 0, nt, &sched->flags) && TS_IN(b, a, nt, &sched->flags))) {  // debug build only
      if (tid == 0) zunit[u] = 0.0;
      __syncthreads();
      continue;
    }
    const double zt = sym_unit<W, RI, YT>(Y, n, acc, fscale, a, b, sj, sacc);
    const double zb = block_sum_d(zt);
    if (tid == 0) zunit[u] = zb;
    __syncthreads();  // shared tiles are rewritten by the next unit
  }

  if (arrive_last(&sched->rep_done)) {
    if (finalize)
      finalize_z(zunit, units, n, sched, advance, ee, ee_iters, mom0, mom1);
    else if (tid == 0)
      sched->work_next = 0u;
  }
}

__global__ void k_finalize_z(const double* __restrict__ zunit, int units, int n, Sched* sched, int advance, float ee,
                             int ee_iters, float mom0, float mom1) {
  finalize_z(zunit, units, n, sched, advance, ee, ee_iters, mom0, mom1);
}

template <int W, int RI>
size_t smem_bytes() {
  constexpr int T = W * 32 * RI;
  return (size_t)T * (sizeof(float4) + sizeof(float2));
}

template <int W, int RI>
tsgne_status prepare() {
  TS_CUDA(cudaFuncSetAttribute(k_repulsion_sym<W, RI, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_bytes<W, RI>()));
  TS_CUDA(cudaFuncSetAttribute(k_repulsion_sym<W, RI, bf162>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_bytes<W, RI>()));
  return TSGNE_OK;
}

template <int W, int RI>
tsgne_status launch(const RepShape& sh, int grid, int n, const void* Y, int y_bf16, unsigned long long* acc,
                    double* zunit, Sched* sched, int u0, int u1, int finalize, int advance, float ee, int ee_iters,
                    float mom0, float mom1, cudaStream_t s) {
  const float fs = fix_scale(n);
  if (y_bf16)
    k_repulsion_sym<W, RI, bf162><<<grid, W * 32, sh.smem, s>>>(static_cast<const bf162*>(Y), n, sh.chunks, acc, fs,
                                                                zunit, sched, u0, u1, finalize, advance, ee,
                                                                ee_iters, mom0, mom1);
  else
    k_repulsion_sym<W, RI, float2><<<grid, W * 32, sh.smem, s>>>(static_cast<const float2*>(Y), n, sh.chunks, acc,
                                                                 fs, zunit, sched, u0, u1, finalize, advance, ee,
                                                                 ee_iters, mom0, mom1);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

// The four compiled shapes: (warps per CTA, i-points per lane).
tsgne_status dispatch(const RepShape& sh, int grid, int n, const void* Y, int y_bf16, unsigned long long* acc,
                      double* zunit, Sched* sched, int u0, int u1, int finalize, int advance, float ee, int ee_iters,
                      float mom0, float mom1, cudaStream_t s) {
  if (sh.warps == 2 && sh.R == 16)
    return launch<2, 16>(sh, grid, n, Y, y_bf16, acc, zunit, sched, u0, u1, finalize, advance, ee, ee_iters, mom0,
                         mom1, s);
  if (sh.warps == 1 && sh.R == 16)
    return launch<1, 16>(sh, grid, n, Y, y_bf16, acc, zunit, sched, u0, u1, finalize, advance, ee, ee_iters, mom0,
                         mom1, s);
  if (sh.warps == 2 && sh.R == 8)
    return launch<2, 8>(sh, grid, n, Y, y_bf16, acc, zunit, sched, u0, u1, finalize, advance, ee, ee_iters, mom0,
                        mom1, s);
  if (sh.warps == 1 && sh.R == 8)
    return launch<1, 8>(sh, grid, n, Y, y_bf16, acc, zunit, sched, u0, u1, finalize, advance, ee, ee_iters, mom0,
                        mom1, s);
  last_msg() = "no compiled repulsion shape with these warps / i-points per lane";
  return TSGNE_ERR_INVALID_ARG;
}

}  // namespace

RepShape repulsion_shape_sym_fixed(int n, int sm_count, int W, int RI) {
  RepShape sh;
  const int T = 32 * RI * W;
  const int nt = (n + T - 1) / T;
  sh.warps = W;
  sh.block = 32 * W;
  sh.R = RI;
  sh.jtile = T;
  sh.chunks = nt;
  sh.n_pad = nt * T;
  sh.n_iblk = nt;
  sh.n_jtiles = nt;
  sh.units = nt * (nt + 1) / 2;
  const int slots = sm_count * (warps_per_sm(RI) / W);
  sh.grid = sh.units < slots ? sh.units : slots;
  sh.smem = (size_t)T * (sizeof(float4) + sizeof(float2));
  return sh;
}

RepShape repulsion_shape_sym(int n, int sm_count) {
  int W = 2;
  for (int w : {2, 1}) {  // 2-warp CTAs once the units fill 4 waves of the grid
    W = w;
    const long T = 32L * kRI * w;
    const long nt = (n + T - 1) / T;
    const long units = nt * (nt + 1) / 2;
    const long slots = (long)sm_count * (kWarpsPerSm / w);
    if (units >= 4 * slots) break;
  }
  return repulsion_shape_sym_fixed(n, sm_count, W, kRI);
}

tsgne_status repulsion_sym_prepare(const RepShape& sh) {
  if (sh.warps == 2 && sh.R == 16) return prepare<2, 16>();
  if (sh.warps == 1 && sh.R == 16) return prepare<1, 16>();
  if (sh.warps == 2 && sh.R == 8) return prepare<2, 8>();
  if (sh.warps == 1 && sh.R == 8) return prepare<1, 8>();
  last_msg() = "no compiled repulsion shape with these warps / i-points per lane";
  return TSGNE_ERR_INVALID_ARG;
}

tsgne_status launch_repulsion_sym(const RepShape& sh, int n, const void* Y, int y_bf16, unsigned long long* acc,
                                  double* zpart, Sched* sched, int advance, float ee, int ee_iters, float mom0,
                                  float mom1, cudaStream_t s) {
  return dispatch(sh, sh.grid, n, Y, y_bf16, acc, zpart, sched, 0, sh.units, 1, advance, ee, ee_iters, mom0, mom1,
                  s);
}

tsgne_status launch_repulsion_sym_units(const RepShape& sh, int n, const void* Y, int y_bf16,
                                        unsigned long long* acc, double* zpart, Sched* sched, int u0, int u1,
                                        cudaStream_t s) {
  if (u1 <= u0) return TSGNE_OK;
  const int slots = sh.grid > 0 ? sh.grid : 1;  // persistent grid of the full pass: one CTA per slot
  const int grid = (u1 - u0) < slots ? (u1 - u0) : slots;
  return dispatch(sh, grid, n, Y, y_bf16, acc, zpart, sched, u0, u1, 0, 0, 1.f, 0, 0.f, 0.f, s);
}

tsgne_status launch_finalize_z(const RepShape& sh, int n, const double* zpart, Sched* sched, int advance, float ee,
                               int ee_iters, float mom0, float mom1, cudaStream_t s) {
  k_finalize_z<<<1, sh.block, 0, s>>>(zpart, sh.units, n, sched, advance, ee, ee_iters, mom0, mom1);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

}  // namespace tsgne
