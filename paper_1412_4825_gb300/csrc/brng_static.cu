// brng_static.cu -- Gamma draws that allocate no device memory.
//
// The normal entry points keep their scratch (per-stream positions, error
// counters) in memory that brng_create obtains with cudaMalloc.  Some callers
// cannot call cudaMalloc: code that runs inside another framework's memory
// pool (where that pool must own every device allocation), or a loop that
// must not stall on the device-wide synchronisation cudaMalloc and cudaFree
// imply.  brng_gamma_static serves them: its scratch is a fixed array in the
// library's own device memory (file scope below), so a call enqueues only a
// clear of that array and one kernel.
//
// Costs and limits: every GPU that loads this library holds the array
// (BRNG_STATIC_MAX_STREAMS * 24 bytes + 64 bytes, about 1.5 MB) until the
// process exits; all calls share it, so calls whose work overlaps on the GPU
// (different streams, or different host threads) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "brng.h"
#include "brng_gamma.cuh"
#include "brng_internal.h"

namespace {

constexpr uint32_t kMaxStreams = BRNG_STATIC_MAX_STREAMS;
constexpr size_t kCounterWords = 8;  // brng::DevCounters (40 B) rounded up to 64 B
constexpr int kMaxDevices = 64;

// [0, 3 * kMaxStreams): stream positions, laid out [U | N | E][stream] for the
// call's stream count; then the error counters.
static __device__ __align__(256) unsigned long long g_scratch[3 * kMaxStreams + kCounterWords];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per
// device (host code cannot use the symbol itself as a device pointer).  The
// cached address belongs to the device's context at the time of the lookup:
// after cudaDeviceReset it is stale, so this entry point does not support a
// device reset during the life of the process.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BRNG_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return BRNG_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return BRNG_ECUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return BRNG_OK;
}

}  // namespace

extern "C" int brng_gamma_static(uint64_t seed, uint32_t n_streams, size_t n, const float* alpha,
                                 float* out, uint32_t* words, brng_stream_t stream) {
  if (n_streams == 0 || n_streams > kMaxStreams) return BRNG_EINVAL;
  if (n == 0) return BRNG_OK;
  if (!alpha || !out) return BRNG_EINVAL;
  void* base = nullptr;
  const int st = scratch_address(&base);
  if (st != BRNG_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* pos = static_cast<unsigned long long*>(base);
  unsigned long long* cnt = pos + 3ull * kMaxStreams;
  // the array keeps the previous call's contents: every stream starts at its
  // first element and the counters at zero
  cudaError_t e = cudaMemsetAsync(pos, 0, sizeof(unsigned long long) * 3ull * n_streams, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * kCounterWords, s);
  if (e != cudaSuccess) return BRNG_ECUDA;

  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return BRNG_ECUDA;
  // the same ring-length rule as brng_gamma's launch (a bulk ring holds at
  // least kBulkMinRing elements); N and U rings, words beside the values
  const uint32_t B = brng::ring_len_min8(brng::kDefaultBufLen);
  const size_t per_warp = 128u + 2u * static_cast<size_t>(B) * 128u * (words ? 2u : 1u);
  uint32_t warps = brng::kDefaultWarpsPerBlock;
  while (warps > 1 && per_warp * warps > static_cast<size_t>(optin)) --warps;

  brng::BulkArgs a;
  a.rk = brng::make_round_keys(seed);
  a.n = n;
  a.S = n_streams;
  a.B = B;
  a.tag = nullptr;
  a.p0 = alpha;
  a.p1 = nullptr;
  a.out = out;
  a.words = words;
  a.pos = reinterpret_cast<uint64_t*>(pos);
  a.cnt = reinterpret_cast<brng::DevCounters*>(cnt);
  e = brng::launch_bulk(BRNG_TAG_GAMMA, a, brng::Geometry{warps, B}, s);
  if (e == cudaSuccess) return BRNG_OK;
  return e == cudaErrorInvalidValue ? BRNG_EINVAL : BRNG_ECUDA;
}
