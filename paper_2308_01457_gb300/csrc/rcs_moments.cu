// RCS mean and variance per observation direction from the far-field moments
// (Section II-C, eq. RCS; the first-order moments of Sections III and IV-B).
//
// For direction d with mean far field f = F_d (3 complex components), covariance block
// C = Cov[F'_d] and pseudo-covariance block P = E[F'_d F'_d^T] (3 x 3 each):
//   sigma_d  = |f|^2 / (4 pi)       (far field of the expansion E_sc ~ e^{ik|x|}/(4 pi |x|) F),
//   RCS_dB   = 10 log10 sigma_d,
//   Var[RCS_dB] = (20 / ln 10)^2 Var[Re z] / |f|^4 with z = f^H F'_d (first-order delta method:
//                 d|F|^2 = 2 Re z), Var[Re z] = (E|z|^2 + Re E[z^2]) / 2,
//                 E|z|^2 = f^H C f,  E[z^2] = f^H P conj(f),
//   Var[F_c] = C_cc (the variance of each far-field component).
// One thread per direction; FP64 arithmetic whatever the storage type of the moments.
#include <cuda_runtime.h>

#include <cmath>

#include "fosb_internal.h"

namespace fosb {
namespace {

template <typename V>
__device__ __forceinline__ double2 ld2(const V* p, int64_t i) {
  const V v = p[i];
  return make_double2(double(v.x), double(v.y));
}

template <typename V>
__global__ void rcs_moments_kernel(int64_t n_dir, const V* F, int64_t incf, const V* cov, int64_t ldc, const V* pcov,
                                   int64_t ldp, int convention, double* rcs_db, double* var_db, double* var_f) {
  const int64_t d = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (d >= n_dir) return;
  double2 f[3];
  double mag2 = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    f[c] = ld2(F, (3 * d + c) * incf);
    mag2 += f[c].x * f[c].x + f[c].y * f[c].y;
  }
  const double four_pi = 4.0 * 3.141592653589793238;
  if (rcs_db) rcs_db[d] = 10.0 * log10(convention == 1 ? four_pi * mag2 : mag2 / four_pi);
  if (var_f) {
#pragma unroll
    for (int c = 0; c < 3; ++c) var_f[3 * d + c] = ld2(cov, (3 * d + c) * ldc + 3 * d + c).x;
  }
  if (!var_db) return;
  // E|z|^2 = sum_ij conj(f_i) C_ij f_j and E[z^2] = sum_ij conj(f_i) P_ij conj(f_j): real parts
  double ez2 = 0.0, ezz = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double2 cij = ld2(cov, (3 * d + i) * ldc + 3 * d + j);
      const double2 pij = ld2(pcov, (3 * d + i) * ldp + 3 * d + j);
      // conj(f_i) c f_j: real part of (fi.x - i fi.y)(c)(fj.x + i fj.y)
      const double2 cf = make_double2(cij.x * f[j].x - cij.y * f[j].y, cij.x * f[j].y + cij.y * f[j].x);
      ez2 += f[i].x * cf.x + f[i].y * cf.y;
      // conj(f_i) p conj(f_j)
      const double2 pf = make_double2(pij.x * f[j].x + pij.y * f[j].y, pij.y * f[j].x - pij.x * f[j].y);
      ezz += f[i].x * pf.x + f[i].y * pf.y;
    }
  }
  const double k_db = 20.0 / 2.302585092994045684;  // 20 / ln 10
  var_db[d] = k_db * k_db * 0.5 * (ez2 + ezz) / (mag2 * mag2);
}

}  // namespace
}  // namespace fosb

extern "C" fosb_status fosb_rcs_moments(int64_t n_dir, const void* F, int64_t incf, const void* cov, int64_t ldc,
                                        const void* pcov, int64_t ldp, int prec, int convention, double* rcs_db,
                                        double* var_db, double* var_f, void* stream) {
  using namespace fosb;
  if (n_dir <= 0 || !F || incf < 1) return fail(FOSB_ERR_INVALID_ARG, "fosb_rcs_moments: bad n_dir, F or incf");
  if (prec != FOSB_FP64 && prec != FOSB_MIXED && prec != FOSB_FP32)
    return fail(FOSB_ERR_INVALID_ARG, "fosb_rcs_moments: unknown precision");
  if (convention != 0 && convention != 1) return fail(FOSB_ERR_INVALID_ARG, "fosb_rcs_moments: convention must be 0 or 1");
  if (!rcs_db && !var_db && !var_f) return fail(FOSB_ERR_INVALID_ARG, "fosb_rcs_moments: no output requested");
  if ((var_db || var_f) && (!cov || ldc < 3 * n_dir))
    return fail(FOSB_ERR_INVALID_ARG, "fosb_rcs_moments: the variances need cov with ldc >= 3 n_dir");
  if (var_db && (!pcov || ldp < 3 * n_dir))
    return fail(FOSB_ERR_INVALID_ARG, "fosb_rcs_moments: the RCS variance needs pcov with ldp >= 3 n_dir");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned grid = unsigned((n_dir + 127) / 128);
  if (prec == FOSB_FP32)
    rcs_moments_kernel<float2><<<grid, 128, 0, s>>>(n_dir, static_cast<const float2*>(F), incf,
                                                    static_cast<const float2*>(cov), ldc,
                                                    static_cast<const float2*>(pcov), ldp, convention, rcs_db, var_db,
                                                    var_f);
  else
    rcs_moments_kernel<double2><<<grid, 128, 0, s>>>(n_dir, static_cast<const double2*>(F), incf,
                                                     static_cast<const double2*>(cov), ldc,
                                                     static_cast<const double2*>(pcov), ldp, convention, rcs_db,
                                                     var_db, var_f);
  FOSB_CUDA(launched());
  return FOSB_OK;
}
