// Vector kernels of the GMRES correction solve (GMRES-based iterative refinement of the
// refined solves): complex128 y = alpha x and y += alpha x for strided vectors.
#include <cuda_runtime.h>

#include "fosb_internal.h"

namespace fosb {
namespace {

__global__ void zscal_copy_kernel(int64_t n, double ar, double ai, const double2* x, int64_t incx, double2* y,
                                  int64_t incy) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = x[i * incx];
  y[i * incy] = make_double2(ar * v.x - ai * v.y, ar * v.y + ai * v.x);
}

__global__ void zaxpy_kernel(int64_t n, double ar, double ai, const double2* x, int64_t incx, double2* y,
                             int64_t incy) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = x[i * incx];
  double2 w = y[i * incy];
  w.x += ar * v.x - ai * v.y;
  w.y += ar * v.y + ai * v.x;
  y[i * incy] = w;
}

}  // namespace

cudaError_t zscal_copy(int64_t n, double ar, double ai, const void* x, int64_t incx, void* y, int64_t incy,
                       cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  zscal_copy_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(n, ar, ai, static_cast<const double2*>(x), incx,
                                                            static_cast<double2*>(y), incy);
  return launched();
}

cudaError_t zaxpy(int64_t n, double ar, double ai, const void* x, int64_t incx, void* y, int64_t incy, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  zaxpy_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(n, ar, ai, static_cast<const double2*>(x), incx,
                                                       static_cast<double2*>(y), incy);
  return launched();
}

}  // namespace fosb
