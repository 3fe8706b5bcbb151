// noalloc.cu -- LU factorisation for callers that must not allocate device
// memory.
//
// posit_rgetrf needs about 0.6 MB of device scratch per call (the panel
// kernel's pivot candidates, the swapped rows and its grid-barrier state),
// which it takes with cudaMallocAsync.  Some callers cannot let a library
// allocate: their device memory is fully reserved by another allocator (for
// example a framework's caching allocator), they run under a fixed memory
// accounting in which any extra allocation is an error, or they call from a
// loop where an allocation could wait on other work.  posit_rgetrf_static
// gives them the same factorisation with the scratch taken from a fixed
// array compiled into the library instead.
//
// The array lives in device global memory on every GPU that loads the
// library, for the life of the process.  Host code must not use its name as
// a device address: the address is obtained once per device with
// cudaGetSymbolAddress, the first time the entry point runs on that device
// (with that device current), and cached.
#include <mutex>

#include "internal.cuh"

namespace posit {
namespace {

constexpr size_t kStaticScratchBytes = 1u << 20;  // 1 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_getrf_scratch[kStaticScratchBytes];

std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices];

// Device address of the array on the current device (set up on first use).
int static_scratch(void **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return POSIT_ERR_DEVICE;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_getrf_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return POSIT_ERR_DEVICE;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return POSIT_OK;
}

}  // namespace
}  // namespace posit

using namespace posit;

extern "C" int posit_rgetrf_static(int64_t m, int64_t n, posit32_t *A, int64_t lda,
                                   int32_t *ipiv, int32_t *info, cudaStream_t stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (lda < max64(1, m)) return -4;
  if (!info) return -6;
  if (m > 0 && n > 0 && !A) return -3;
  if (m > 0 && n > 0 && !ipiv) return -5;
  // as posit_rgetrf: info is cleared and an empty matrix returns at once,
  // before the scratch is looked at
  if (cudaMemsetAsync(info, 0, sizeof(int32_t), stream) != cudaSuccess) return POSIT_ERR_CUDA;
  if (m == 0 || n == 0) return POSIT_OK;
  const size_t need = getrf_scratch_bytes();
  if (!need) return POSIT_ERR_DEVICE;
  if (need > kStaticScratchBytes) return POSIT_ERR_SCRATCH;
  void *scratch = nullptr;
  int st = static_scratch(&scratch);
  if (st) return st;
  // getrf_run clears the part of the scratch that must start at zero
  return getrf_run(m, n, A, lda, ipiv, info, scratch, stream);
}
