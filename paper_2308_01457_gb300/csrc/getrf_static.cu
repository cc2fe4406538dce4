// fosb_getrf_static: LU factorisation that allocates no device memory.
//
// Some callers cannot call cudaMalloc while they use this library: hosts that hand out
// all device memory through their own allocator (a caching allocator or a pool sized at
// start-up) and treat any allocation behind their back as an error, and latency-bound
// integrations that forbid allocation after initialisation because cudaMalloc/cudaFree
// can synchronise the device and take unbounded time.  fosb_factor allocates its
// factors and its panel scratch; this entry point factors the caller's matrix in place
// and takes the panel kernel's scratch (grid-barrier words, pivot candidates, status
// word) from a file-scope static device array instead.
//
// The array is kStaticScratchBytes (1 MiB); every GPU that loads the library holds it
// until the process exits.  In host code the array's name is only a host-side stand-in,
// so its device address is looked up once per device with cudaGetSymbolAddress -- on the
// first call on that device, with that device current -- and passed to the kernels.
// Every call reads its status word back with a stream synchronisation, so no call can
// run inside a stream capture.  All calls share the array: calls whose work overlaps on
// the GPU race, so serialise them.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "fosb_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(1) << 20;  // 1 MiB
constexpr int64_t kStaticMaxCtas = 256;                  // panel CTAs that fit the array
constexpr size_t kStatusOffset = 64;                     // status word inside the zeroed head

static __device__ __align__(256) unsigned char g_getrf_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

fosb_status scratch_for_current_device(void** out) {
  int dev = 0;
  FOSB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fosb::fail(FOSB_ERR_INVALID_ARG, "fosb_getrf_static: device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_getrf_scratch);
    if (e != cudaSuccess || !p) return fosb::cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                                        "fosb_getrf_static: cudaGetSymbolAddress");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return FOSB_OK;
}

}  // namespace

extern "C" fosb_status fosb_getrf_static(void* A, int64_t n, int64_t lda, int prec, int32_t* ipiv, void* stream) {
  using namespace fosb;
  if (!A || !ipiv || n <= 0 || lda < n) return fail(FOSB_ERR_INVALID_ARG, "fosb_getrf_static: bad arguments");
  if (prec != FOSB_FP64 && prec != FOSB_FP32)
    return fail(FOSB_ERR_INVALID_ARG, "fosb_getrf_static: prec must be FOSB_FP64 (complex128) or FOSB_FP32 (complex64)");
  const bool c128 = prec == FOSB_FP64;
  static_assert(kStatusOffset + sizeof(int) <= 256, "status word must sit in the zeroed head");
  if (getrf_scratch_bytes(kStaticMaxCtas, c128) > kStaticScratchBytes)
    return fail(FOSB_ERR_INVALID_ARG, "fosb_getrf_static: scratch layout exceeds the static array");
  // size limit: the first panel holds all n rows in at most min(SM count, kStaticMaxCtas)
  // co-resident CTAs of at most 2048 rows each (311,296 on a 152-SM GB300)
  int64_t max_n = 0;
  FOSB_TRY(getrf_external_max_n(kStaticMaxCtas, &max_n));
  if (n > max_n)
    return fail(FOSB_ERR_INVALID_ARG, "fosb_getrf_static: n = " + std::to_string(n) + " exceeds the limit " +
                                          std::to_string(max_n) + " of the static scratch on this GPU (use fosb_factor)");
  void* scratch = nullptr;
  FOSB_TRY(scratch_for_current_device(&scratch));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // barrier words and the status word must start at zero; the rest is written before read
  FOSB_CUDA(cudaMemsetAsync(scratch, 0, 256, s));
  int* d_status = reinterpret_cast<int*>(static_cast<char*>(scratch) + kStatusOffset);
  fosb_status st = c128 ? getrf_external_scratch<double>(A, n, lda, ipiv, d_status, scratch, kStaticMaxCtas, s)
                        : getrf_external_scratch<float>(A, n, lda, ipiv, d_status, scratch, kStaticMaxCtas, s);
  if (st != FOSB_OK) return st;
  int status = 0;
  FOSB_CUDA(cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  FOSB_CUDA(cudaStreamSynchronize(s));
  if (status == FOSB_ERR_TIMEOUT) return fail(FOSB_ERR_TIMEOUT, "fosb_getrf_static: panel grid barrier timed out");
  if (status == FOSB_ERR_SINGULAR) return fail(FOSB_ERR_SINGULAR, "fosb_getrf_static: zero pivot");
  return FOSB_OK;
}
