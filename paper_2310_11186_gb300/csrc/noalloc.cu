// tsgne_repulsion_noalloc: the all-pairs repulsion pass for callers that may
// not allocate device memory.
//
// Who needs it: code that runs under a fixed device-memory budget owned by
// someone else (a custom operator inside an inference server or a plugin
// host whose framework owns the allocator), and code that must not call
// cudaMalloc / cudaFree because those calls can synchronise the whole device
// and stall unrelated work.  Such callers pass their layout and output
// buffers; every temporary this pass needs lives in one file-scope device
// array, allocated once when the library's device code is loaded on a GPU and
// held until the process exits.
//
// Limits and sharing rules:
//   - at most TSGNE_NOALLOC_MAX_N points (65,536); larger inputs are rejected
//     with TSGNE_ERR_INVALID_ARG before any work is enqueued;
//   - the first call on each device looks up the array's device address
//     (cudaGetSymbolAddress, with that device current); make that first call
//     before any stream capture;
//   - Y, frep_out and z_out must be 8-byte aligned (Y and frep_out are read
//     and written as float pairs, z_out as a double); a misaligned pointer
//     is rejected with TSGNE_ERR_INVALID_ARG before any work is enqueued;
//   - the device address of the array is cached per device ordinal for the
//     life of the process; it does not survive cudaDeviceReset (or any other
//     teardown of the device's primary context), after which this entry
//     point must not be called again in that process;
//   - all calls share the one array and it keeps the last call's contents:
//     every call clears the counters it needs and overwrites every region it
//     reads, so consecutive calls on one stream are independent, but calls
//     that overlap on the GPU (two streams, or two threads) race on it.
#include <cstdint>
#include <mutex>
#include <string>

#include "tsgne_internal.cuh"

namespace tsgne {

namespace {

constexpr int kNoAllocMaxN = TSGNE_NOALLOC_MAX_N;
constexpr int kNoAllocMaxChunks = 16;
constexpr int kNoAllocMaxGrid = 4096;
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kYBytes = align_up((size_t)kNoAllocMaxN * sizeof(float2));
constexpr size_t kPartBytes = align_up((size_t)kNoAllocMaxChunks * kNoAllocMaxN * sizeof(float2));
constexpr size_t kZBytes = align_up((size_t)kNoAllocMaxGrid * sizeof(double));
constexpr size_t kSchedBytes = align_up(sizeof(Sched));
constexpr size_t kScratchBytes = kYBytes + kPartBytes + kZBytes + kSchedBytes;  // about 8.6 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Layout copied into the padded scratch copy; the tail gets the sentinel.
__global__ void k_pad_copy(const float2* __restrict__ Y, int n, int n_pad, float2* __restrict__ Ypad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x)
    Ypad[i] = i < n ? Y[i] : make_float2(kSentinel, kSentinel);
}

// F^r_i = sum of the chunk partials in chunk order.
__global__ void k_sum_chunks(const float2* __restrict__ part, int chunks, int n_pad, int n, float2* __restrict__ out,
                             const Sched* __restrict__ sched, double* __restrict__ z_out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float fx = 0.f, fy = 0.f;
    for (int c = 0; c < chunks; ++c) {
      const float2 f = part[(size_t)c * n_pad + i];
      fx += f.x;
      fy += f.y;
    }
    out[i] = make_float2(fx, fy);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *z_out = sched->Z;
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_base[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
tsgne_status scratch_base(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    last_msg() = "device ordinal out of range for the no-allocation scratch table";
    return TSGNE_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void* p = nullptr;
    TS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_base[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_base[dev];
  return TSGNE_OK;
}

tsgne_status repulsion_noalloc(int32_t n, const float* Y, float* frep_out, double* z_out, cudaStream_t s) {
  if (n < 2 || !Y || !frep_out || !z_out) {
    last_msg() = "need n >= 2 and non-NULL Y, frep_out and z_out";
    return TSGNE_ERR_INVALID_ARG;
  }
  if (n > kNoAllocMaxN) {
    last_msg() = "n = " + std::to_string(n) + " exceeds the no-allocation maximum of TSGNE_NOALLOC_MAX_N = " +
                 std::to_string(kNoAllocMaxN) + " points";
    return TSGNE_ERR_INVALID_ARG;
  }
  if (((uintptr_t)Y | (uintptr_t)frep_out | (uintptr_t)z_out) & 7u) {
    last_msg() = "Y, frep_out and z_out must be 8-byte aligned";
    return TSGNE_ERR_INVALID_ARG;
  }
  int dev = 0, sms = 1;
  TS_CUDA(cudaGetDevice(&dev));
  TS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  RepShape sh = repulsion_shape(n, sms);
  if (sh.chunks > kNoAllocMaxChunks) {
    sh.chunks = kNoAllocMaxChunks;
    const long units = (long)sh.n_iblk * sh.chunks;
    const long slots = 2L * sms;
    sh.grid = (int)(units < slots ? units : slots);
  }
  if (sh.grid > kNoAllocMaxGrid || sh.n_pad > kNoAllocMaxN) {
    last_msg() = "launch shape exceeds the no-allocation scratch";
    return TSGNE_ERR_INVALID_ARG;
  }
  unsigned char* base = nullptr;
  TS_TRY(scratch_base(dev, &base));
  float2* Ypad = reinterpret_cast<float2*>(base);
  float2* part = reinterpret_cast<float2*>(base + kYBytes);
  double* zpart = reinterpret_cast<double*>(base + kYBytes + kPartBytes);
  Sched* sched = reinterpret_cast<Sched*>(base + kYBytes + kPartBytes + kZBytes);
  TS_CUDA(cudaMemsetAsync(sched, 0, sizeof(Sched), s));
  k_pad_copy<<<(sh.n_pad + 255) / 256, 256, 0, s>>>(reinterpret_cast<const float2*>(Y), n, sh.n_pad, Ypad);
  TS_CUDA(cudaGetLastError());
  TS_TRY(launch_repulsion(sh, n, Ypad, part, zpart, sched, 0, 1.f, 0, 0.f, 0.f, s));
  k_sum_chunks<<<(n + 255) / 256, 256, 0, s>>>(part, sh.chunks, sh.n_pad, n, reinterpret_cast<float2*>(frep_out),
                                               sched, z_out);
  TS_CUDA(cudaGetLastError());
  return TSGNE_OK;
}

}  // namespace

}  // namespace tsgne

extern "C" tsgne_status tsgne_repulsion_noalloc(int32_t n, const float* Y, float* frep_out, double* z_out,
                                                void* cuda_stream) {
  tsgne::last_msg().clear();
  return tsgne::repulsion_noalloc(n, Y, frep_out, z_out, static_cast<cudaStream_t>(cuda_stream));
}
