// Affinities of t-SGNE on the neighbour structure.
//
// K1  conditional affinities (Eq. 2 with the denominator over N(i)):
//     p_{j|i} = exp(-beta_i (d_ij - m_i)) / S_i,  d_ij = ||x_i - x_j||^2,
//     m_i = min_j d_ij (the shift leaves p unchanged and keeps exp in range),
//     beta_i = 1 / (2 sigma_i^2) chosen by binary search so that the row
//     entropy H_i = ln S_i + beta_i E_p[d - m_i] equals ln(perplexity)
//     (Sec. 2.1: Perp = 2^H with H in bits).  One warp per row: lanes stride
//     the embedding dimension with float4 loads for the distances and the
//     row entries for the entropy sums; every lane reaches the same sums
//     (xor butterfly), so all branch decisions are warp-uniform.
//     Search: beta = 1, doubled / halved until the target is bracketed, then
//     midpoints; stop when |H - ln perp| <= tol or after max_iter entropy
//     evaluations; p is taken at the last evaluated beta.  A row with
//     |N(i)| <= perplexity cannot reach ln(perp) (its maximum entropy is
//     ln |N(i)|) and is set uniform.
//     Precision: the whole row computation (distances, exp, entropy sums,
//     bisection) runs in FP64 and only p is rounded to FP32.  The build runs
//     once per layout, and FP32 here turns the rounding of d ~ 10^2 into
//     ~1e-4 relative errors in p at small perplexities (large beta) and can
//     flip bisection decisions near the stopping tolerance.
// K2  joint affinities (Eq. 3): p_ij = (p_{j|i} + p_{i|j}) / T with T the
//     FP64 total of all numerators (T = 2n without isolated nodes), so that
//     sum P = 1; the total is a fixed-order reduction.
#include <cmath>

#include "reduce.cuh"
#include "tsgne_internal.cuh"

namespace tsgne {

namespace {

constexpr int kAffCta = 256;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_min_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <bool VEC4>
__global__ void __launch_bounds__(kAffCta) k_cond_affinity(int n, const int64_t* __restrict__ rp,
                                                           const int32_t* __restrict__ col,
                                                           const float* __restrict__ X, int d, float perp,
                                                           double Hstar, double tol, int max_iter,
                                                           double* __restrict__ dist, float* __restrict__ pcond) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const int64_t a = rp[i], b = rp[i + 1];
    const int64_t k = b - a;
    if (k == 0) continue;
    if ((float)k <= perp) {  // saturated row: uniform, no distances needed
      const float u = 1.0f / (float)k;
      for (int64_t e = a + lane; e < b; e += 32) pcond[e] = u;
      continue;
    }
    // squared distances in R^d, one neighbour at a time across the warp
    for (int64_t e = a; e < b; ++e) {
      const int64_t j = col[e];
      double s = 0.0;
      if (VEC4) {
        const float4* xi = reinterpret_cast<const float4*>(X + i * d);
        const float4* xj = reinterpret_cast<const float4*>(X + j * d);
        for (int c = lane; c < (d >> 2); c += 32) {
          const float4 u = xi[c], v = xj[c];
          const double t0 = (double)u.x - v.x, t1 = (double)u.y - v.y;
          const double t2 = (double)u.z - v.z, t3 = (double)u.w - v.w;
          s = fma(t0, t0, s);
          s = fma(t1, t1, s);
          s = fma(t2, t2, s);
          s = fma(t3, t3, s);
        }
      } else {
        for (int c = lane; c < d; c += 32) {
          const double t = (double)X[i * d + c] - (double)X[j * d + c];
          s = fma(t, t, s);
        }
      }
      s = warp_sum_d(s);
      if (lane == 0) dist[e] = s;
    }
    __syncwarp();
    double m = INFINITY;
    for (int64_t e = a + lane; e < b; e += 32) m = fmin(m, dist[e]);
    m = warp_min_d(m);
    double beta = 1.0, lo = -INFINITY, hi = INFINITY, S = 1.0;
    for (int it = 0; it < max_iter; ++it) {
      double s = 0.0, E = 0.0;
      for (int64_t e = a + lane; e < b; e += 32) {
        const double delta = dist[e] - m;
        const double w = exp(-beta * delta);
        s += w;
        E += delta * w;
      }
      S = warp_sum_d(s);
      E = warp_sum_d(E);
      const double H = log(S) + beta * E / S;
      if (fabs(H - Hstar) <= tol || it == max_iter - 1) break;
      if (H > Hstar) {
        lo = beta;
        beta = isinf(hi) ? 2.0 * beta : 0.5 * (beta + hi);
      } else {
        hi = beta;
        beta = isinf(lo) ? 0.5 * beta : 0.5 * (beta + lo);
      }
    }
    for (int64_t e = a + lane; e < b; e += 32) pcond[e] = (float)(exp(-beta * (dist[e] - m)) / S);
  }
}

// Total of the Eq. 3 numerators (FP64, fixed order) into sched->red[0].
__global__ void __launch_bounds__(kAffCta) k_joint_total(int64_t nnz, const float* __restrict__ pcond,
                                                         const int64_t* __restrict__ tslot,
                                                         double* __restrict__ parts, Sched* sched) {
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride)
    acc += (double)pcond[e] + (double)pcond[tslot[e]];
  double bs = block_sum_d(acc);
  if (threadIdx.x == 0) parts[blockIdx.x] = bs;
  if (arrive_last(&sched->red_done)) {
    double T = sum_partials(parts, gridDim.x);
    if (threadIdx.x == 0) {
      sched->red[0] = T;
      if (!isfinite(T)) atomicOr(&sched->flags, kFlagNonfiniteP);
    }
  }
}

__global__ void __launch_bounds__(kAffCta) k_joint_scale(int64_t nnz, const float* __restrict__ pcond,
                                                         const int64_t* __restrict__ tslot, float* __restrict__ P,
                                                         Sched* sched) {
  const double T = sched->red[0];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
    const double v = ((double)pcond[e] + (double)pcond[tslot[e]]) / T;
    const float p = (float)v;
    P[e] = p;
    if (!isfinite(p)) atomicOr(&sched->flags, kFlagNonfiniteP);
  }
}

}  // namespace

tsgne_status build_affinities(int n, const int64_t* rp, const int32_t* col, const int64_t* tslot, int64_t nnz,
                              const float* X, int d, float perplexity, float tol, int max_iter, float* P, Sched* sched,
                              cudaStream_t s) {
  int dev = 0, sms = 1;
  TS_CUDA(cudaGetDevice(&dev));
  TS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DevBuf<double> dist;
  DevBuf<float> pcond;
  TS_TRY(dist.alloc((size_t)nnz));
  TS_TRY(pcond.alloc((size_t)nnz));
  const double Hstar = std::log((double)perplexity);
  int64_t rows_per_cta = kAffCta / 32;
  int64_t g = ((int64_t)n + rows_per_cta - 1) / rows_per_cta;
  int grid = (int)(g < sms * 64 ? (g < 1 ? 1 : g) : sms * 64);
  const bool vec4 = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15u) == 0);
  if (vec4)
    k_cond_affinity<true><<<grid, kAffCta, 0, s>>>(n, rp, col, X, d, perplexity, Hstar, tol, max_iter, dist.get(),
                                                   pcond.get());
  else
    k_cond_affinity<false><<<grid, kAffCta, 0, s>>>(n, rp, col, X, d, perplexity, Hstar, tol, max_iter, dist.get(),
                                                    pcond.get());
  TS_CUDA(cudaGetLastError());
  TS_TRY(joint_affinities(nnz, pcond.get(), tslot, P, sched, s));
  return TSGNE_OK;
}

tsgne_status joint_affinities(int64_t nnz, const float* pcond, const int64_t* tslot, float* P, Sched* sched,
                              cudaStream_t s) {
  int dev = 0, sms = 1;
  TS_CUDA(cudaGetDevice(&dev));
  TS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int egrid = sms * 4;
  DevBuf<double> parts;
  TS_TRY(parts.alloc(egrid));
  k_joint_total<<<egrid, kAffCta, 0, s>>>(nnz, pcond, tslot, parts.get(), sched);
  k_joint_scale<<<egrid, kAffCta, 0, s>>>(nnz, pcond, tslot, P, sched);
  TS_CUDA(cudaGetLastError());
  TS_CUDA(cudaStreamSynchronize(s));  // temporaries are freed on return
  return TSGNE_OK;
}

}  // namespace tsgne
