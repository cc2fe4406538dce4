// Throughput microbenchmarks of the execution units the hot-path kernels are bound by
// (diagnostics for the roofline denominators; fosb_peak_microbench):
//   kind 0: FP32 FMA pipe  (8 independent FMA chains per thread, every SM full)
//   kind 1: FP64 FMA pipe  (same, double)
//   kind 2: tcgen05.mma kind::tf32, M = 128, N = 256, K = 8, back to back from shared memory
//   kind 3: tcgen05.mma kind::f16 (bf16), M = 128, N = 256, K = 16, the same way
// One CTA per SM for the MMA kinds; one thread issues all MMAs into one TMEM accumulator,
// then a commit and a bounded mbarrier wait.  Rates are 2 flops per multiply-add.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "fosb_internal.h"

namespace fosb {
namespace {

template <typename T>
__global__ void fma_peak_kernel(T* out, int iters, T b, T c) {
  T a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = T(threadIdx.x & 7) * T(0.001) + T(i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = a[i] * b + c;
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == T(-1)) out[blockIdx.x] = s;  // never true; keeps the chains live
}

constexpr int kPeakM = 128, kPeakN = 256;
constexpr int kPeakSmemA = kPeakM * 32, kPeakSmemB = kPeakN * 32;  // one 32-byte K slab per row
constexpr long long kPeakSpinLimit = 1ll << 24;

__device__ __forceinline__ uint32_t peak_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// canonical K-major no-swizzle layout: 8-row x 16-byte core matrices, LBO 128 B, SBO 256 B
__device__ __forceinline__ uint64_t peak_desc(uint32_t addr) {
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t(128 >> 4) << 16) | (uint64_t(256 >> 4) << 32) |
         (uint64_t(1) << 46);
}

template <bool BF16>
__global__ void __launch_bounds__(128, 1) mma_peak_kernel(int reps, int* status) {
  __shared__ __align__(1024) unsigned char sm[kPeakSmemA + kPeakSmemB];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  for (int i = threadIdx.x; i < (kPeakSmemA + kPeakSmemB) / 4; i += blockDim.x) reinterpret_cast<int*>(sm)[i] = 0;
  asm volatile("fence.proxy.async.shared::cta;");
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(peak_smem_u32(&tmem_base)),
                 "r"(kPeakN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(peak_smem_u32(&bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  if (threadIdx.x == 0) {
    // D f32 (bits 4-5 = 1); A, B tf32 (2) or bf16 (1) at bits 7-9 / 10-12; K-major; N >> 3, M >> 4
    const uint32_t fmt = BF16 ? 1u : 2u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(kPeakN >> 3) << 17) |
                           (uint32_t(kPeakM >> 4) << 24);
    const uint64_t ad = peak_desc(peak_smem_u32(sm)), bd = peak_desc(peak_smem_u32(sm + kPeakSmemA));
    for (int r = 0; r < reps; ++r) {
      const uint32_t acc = r > 0 ? 1u : 0u;
      if (BF16)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        peak_smem_u32(&bar)));
    bool done = false;
    for (long long spins = 0; spins < kPeakSpinLimit && !done; ++spins) {
      uint32_t d;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(d)
          : "r"(peak_smem_u32(&bar)), "r"(0u));
      done = d != 0;
      if (!done) __nanosleep(64);
    }
    if (!done) atomicExch(status, FOSB_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPeakN));
}

}  // namespace
}  // namespace fosb

extern "C" fosb_status fosb_peak_microbench(int kind, double* tflops) {
  using namespace fosb;
  if (!tflops || kind < 0 || kind > 3) return fail(FOSB_ERR_INVALID_ARG, "fosb_peak_microbench: bad kind or NULL output");
  int dev = 0, nsm = 0;
  FOSB_CUDA(cudaGetDevice(&dev));
  FOSB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  void* buf = nullptr;
  FOSB_CUDA(cudaMalloc(&buf, 64 * sizeof(double) + sizeof(int) * 2));
  int* d_status = reinterpret_cast<int*>(static_cast<char*>(buf) + 64 * sizeof(double));
  cudaEvent_t a = nullptr, b = nullptr;
  fosb_status st = FOSB_OK;
  double flops = 0.0, best_ms = 1e30;
  auto launch = [&]() {
    if (kind == 0) {
      const int iters = 1 << 16;
      fma_peak_kernel<float><<<nsm * 4, 256, 0>>>(static_cast<float*>(buf), iters, 0.999999f, 1e-6f);
      flops = 2.0 * 8.0 * iters * 256.0 * nsm * 4;
    } else if (kind == 1) {
      const int iters = 1 << 10;
      fma_peak_kernel<double><<<nsm * 4, 256, 0>>>(static_cast<double*>(buf), iters, 0.999999, 1e-6);
      flops = 2.0 * 8.0 * iters * 256.0 * nsm * 4;
    } else {
      const int reps = 16384;
      if (kind == 2)
        mma_peak_kernel<false><<<nsm, 128, 0>>>(reps, d_status);
      else
        mma_peak_kernel<true><<<nsm, 128, 0>>>(reps, d_status);
      flops = 2.0 * kPeakM * kPeakN * (kind == 2 ? 8 : 16) * double(reps) * nsm;
    }
    note_launches(1);
    return cudaGetLastError();
  };
  cudaError_t e = cudaMemset(d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = launch();  // warm-up
  for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
    cudaEventRecord(a);
    e = launch();
    cudaEventRecord(b);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess) best_ms = std::min(best_ms, double(ms));
  }
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) st = cuda_fail(e, "fosb_peak_microbench");
  else if (status == FOSB_ERR_TIMEOUT) st = fail(FOSB_ERR_TIMEOUT, "fosb_peak_microbench: MMA completion wait timed out");
  else *tflops = flops / (best_ms * 1e-3) / 1e12;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(buf);
  return st;
}
