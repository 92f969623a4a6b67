// bege_search_noalloc: the whole search (segment spectrum, correlation,
// sigma, tails) for callers that are not allowed to allocate device memory.
//
// Some programs hand every byte of device memory to one allocator of their
// own (a framework's caching pool, or an arena reserved once at start-up so
// that a latency-critical loop never pays for cudaMalloc/cudaFree, which
// synchronise the device and fragment the heap).  Such a caller can pass its
// own input and output buffers, but the library must not allocate the
// intermediates behind its back.  This entry point keeps them in one
// file-scope device array of fixed size instead:
//   - the product coefficients A, B and the segment spectrum D of the
//     segment (at most N = 2^16 samples),
//   - the FP32 twiddle tables for that N (computed on the device in FP64
//     by every call, ahead of the call's own kernels on its stream, so no
//     call depends on what an earlier call left in the array).
// The array lives on every GPU that loads the library until the process
// exits (about 1.05 MiB).  All calls on a device share it and it keeps the
// contents of the last call, so two calls whose work overlaps on the GPU
// (for example on two streams) corrupt each other; callers serialise them.
#include <mutex>
#include <string>

#include "bege_corr.cuh"
#include "bege_internal.h"

namespace bege {

namespace {

constexpr int64_t kMaxN = 1 << 16;
constexpr int64_t kMaxH = kMaxN / 2;

constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte offsets of the regions of the scratch array (sized for N = 2^16).
constexpr size_t kOffAB = 0;
constexpr size_t kOffD = kOffAB + al256(kMaxH * sizeof(float4));
constexpr size_t kOffTw2 = kOffD + al256((kMaxH + 1) * sizeof(float2));
constexpr size_t kOffTw3 = kOffTw2 + al256(256 * sizeof(float2));
constexpr size_t kOffWH = kOffTw3 + al256(4096 * sizeof(float2));
constexpr size_t kOffWR0S = kOffWH + al256(256 * 8 * sizeof(float2));
constexpr size_t kOffW16S = kOffWR0S + al256(16 * 8 * sizeof(float2));
constexpr size_t kOffWS = kOffW16S + al256(16 * 8 * sizeof(float2));
constexpr size_t kOffWN = kOffWS + al256(8 * sizeof(float2));
constexpr size_t kScratchBytes = kOffWN + al256(kMaxH * sizeof(float2));

static __device__ __align__(256) unsigned char g_search_scratch[kScratchBytes];

// exp(-2 pi i k / M) from the FP64 sincospi, rounded once to FP32.
__device__ __forceinline__ float2 unit_root(int64_t k, int64_t M) {
  double s, c;
  sincospi(-2.0 * (double)(k % M) / (double)M, &s, &c);
  return make_float2((float)c, (float)s);
}

// The twiddle tables of PlanDev for geometry g, written into the scratch
// regions (same definitions as the tables the context uploads).
__global__ void search_tables_kernel(Geometry g, float2* tw2, float2* tw3, float2* wH,
                                     float2* wR0S, float2* w16S, float2* wS, float2* wN) {
  const int64_t n_tw2 = 16 * g.R0, n_tw3 = g.F, n_wH = 256 * (int64_t)g.S,
                n_wR0S = (int64_t)g.R0 * g.S, n_w16S = 16 * (int64_t)g.S, n_wS = g.S,
                n_wN = g.H;
  const int64_t total = n_tw2 + n_tw3 + n_wH + n_wR0S + n_w16S + n_wS + n_wN;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = i;
    if (j < n_tw2) {
      tw2[j] = unit_root((j % g.R0) * (j / g.R0), 16 * (int64_t)g.R0);
      continue;
    }
    j -= n_tw2;
    if (j < n_tw3) {
      const int64_t ns = g.F / 16;
      tw3[j] = unit_root((j % ns) * (j / ns), g.F);
      continue;
    }
    j -= n_tw3;
    if (j < n_wH) {
      wH[j] = unit_root(j, g.H);
      continue;
    }
    j -= n_wH;
    if (j < n_wR0S) {
      wR0S[j] = unit_root(j, (int64_t)g.R0 * g.S);
      continue;
    }
    j -= n_wR0S;
    if (j < n_w16S) {
      w16S[j] = unit_root(j, 16 * (int64_t)g.S);
      continue;
    }
    j -= n_w16S;
    if (j < n_wS) {
      wS[j] = unit_root(j, g.S);
      continue;
    }
    j -= n_wS;
    wN[j] = unit_root(j, g.N);
  }
}

// Per-device set-up: the device address of the scratch array, looked up once
// per device with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

}  // namespace

}  // namespace bege

extern "C" int bege_search_noalloc(const float* strain_dev, int64_t n, const float* bank_dev,
                                   int64_t ld, int64_t k_begin, int64_t k_end, float kappa,
                                   float* sigma_dev, bege_tail* tails_dev,
                                   uint64_t tail_capacity, unsigned long long* tail_count_dev,
                                   void* stream) {
  using namespace bege;
  if (!strain_dev || !bank_dev || !sigma_dev || !tail_count_dev || (tail_capacity && !tails_dev))
    return set_last_error(BEGE_EINVAL, "bege_search_noalloc: NULL pointer");
  if (n < 1024 || n > kMaxN || (n & (n - 1)))
    return set_last_error(BEGE_EINVAL,
                          "bege_search_noalloc: n must be a power of two in [2^10, 2^16]; "
                          "the fixed scratch array holds segments of at most 2^16 samples");
  if (ld < 8 || ld % 8 != 0 || ld > n)
    return set_last_error(BEGE_EINVAL,
                          "bege_search_noalloc: ld must be a multiple of 8 in [8, n]");
  if (k_begin < 0 || k_end <= k_begin)
    return set_last_error(BEGE_EINVAL, "bege_search_noalloc: empty template range");
  if (!(kappa >= 0.f) || kappa > 3.0e38f)
    return set_last_error(BEGE_EINVAL, "bege_search_noalloc: kappa must be finite and >= 0");
  if (reinterpret_cast<uintptr_t>(strain_dev) % 8 || reinterpret_cast<uintptr_t>(bank_dev) % 32 ||
      reinterpret_cast<uintptr_t>(tail_count_dev) % 8 ||
      reinterpret_cast<uintptr_t>(sigma_dev) % 4 || reinterpret_cast<uintptr_t>(tails_dev) % 4)
    return set_last_error(BEGE_EINVAL, "bege_search_noalloc: misaligned buffer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_last_error(BEGE_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return set_last_error(BEGE_EINVAL, "bege_search_noalloc: device index too large");

  const Geometry g = make_geometry(n);
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_search_scratch);
      if (e != cudaSuccess)
        return set_last_error(BEGE_ECUDA, std::string("cudaGetSymbolAddress: ") +
                                              cudaGetErrorString(e));
      g_addr[dev] = static_cast<unsigned char*>(p);
    }
    base = g_addr[dev];
    PlanDev p{};
    p.g = g;
    p.tw2 = reinterpret_cast<const float2*>(base + kOffTw2);
    p.tw3 = reinterpret_cast<const float2*>(base + kOffTw3);
    p.wH = reinterpret_cast<const float2*>(base + kOffWH);
    p.wR0S = reinterpret_cast<const float2*>(base + kOffWR0S);
    p.w16S = reinterpret_cast<const float2*>(base + kOffW16S);
    p.wS = reinterpret_cast<const float2*>(base + kOffWS);
    p.wN = reinterpret_cast<const float2*>(base + kOffWN);
    // The tables are rebuilt on every call, in stream order before this
    // call's kernels: the host keeps no record of which n the array holds,
    // which could disagree with the device's order of work.
    search_tables_kernel<<<64, 256, 0, s>>>(
        g, const_cast<float2*>(p.tw2), const_cast<float2*>(p.tw3), const_cast<float2*>(p.wH),
        const_cast<float2*>(p.wR0S), const_cast<float2*>(p.w16S), const_cast<float2*>(p.wS),
        const_cast<float2*>(p.wN));
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_last_error(BEGE_ECUDA, cudaGetErrorString(e));
    float4* AB = reinterpret_cast<float4*>(base + kOffAB);
    float2* D = reinterpret_cast<float2*>(base + kOffD);
    e = launch_segment(p, strain_dev, D, AB, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(tail_count_dev, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
      CorrelateArgs a{};
      a.AB = AB;
      a.bank = bank_dev;
      a.Lp = ld;
      a.k0 = k_begin;
      a.k1 = k_end;
      a.kappa = kappa;
      a.sigma = sigma_dev;  // row k writes sigma_dev[k - k_begin]
      a.recs = tails_dev;
      a.cap = tail_capacity;
      a.counter = tail_count_dev;
      a.dump = nullptr;
      a.max_clusters = 0;
      e = launch_correlate(p, a, default_config(g), s);
    }
    if (e != cudaSuccess) return set_last_error(BEGE_ECUDA, cudaGetErrorString(e));
  }
  return BEGE_OK;
}
