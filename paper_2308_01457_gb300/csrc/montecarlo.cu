// Monte Carlo over random normal perturbations of a scatterer: the paper's reference
// estimator for the shape statistics (Section V-C: samples of perturbed surfaces, each
// solved, and sample moments of the far field), against which FOSB is compared.
//
//   fosb_field_samples: xi_s = L z_s with K + jitter I = L L^T, K_pq = kernel(|x_p - x_q|) on
//                       the mesh vertices (the random normal velocity expanded at the
//                       vertices, Section III); z are the caller's standard normal draws.
//   fosb_mesh_perturb:  the sample surface x_p + t xi_p n_p (same triangles).
//   fosb_mc_moments:    sample mean of F_s and, with D_s = (F_s - F_0) / t, the sample
//                       covariance (1/S) sum_s D_s D_s^H and pseudo-covariance (1/S) sum_s D_s D_s^T
//                       on the device.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "fosb_internal.h"

namespace fosb {
namespace {

__global__ void mc_mean_kernel(int64_t n3, int64_t S, const double2* __restrict__ Fs, int64_t ldf,
                               double2* __restrict__ mean) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  double re = 0.0, im = 0.0;
  for (int64_t s = 0; s < S; ++s) {
    const double2 f = Fs[i * ldf + s];
    re += f.x;
    im += f.y;
  }
  mean[i] = make_double2(re / double(S), im / double(S));
}

// one thread per (i, j): the covariance entry and, if pcov, the pseudo-covariance entry
__global__ void mc_cov_kernel(int64_t n3, int64_t S, const double2* __restrict__ Fs, int64_t ldf,
                              const double2* __restrict__ F0, double inv_t, double2* __restrict__ cov, int64_t ldc,
                              double2* __restrict__ pcov, int64_t ldp) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n3 * n3) return;
  const int64_t i = e / n3, j = e % n3;
  const double2 fi0 = F0[i], fj0 = F0[j];
  double cr = 0.0, ci = 0.0, pr = 0.0, pi = 0.0;
  for (int64_t s = 0; s < S; ++s) {
    const double2 a = Fs[i * ldf + s], b = Fs[j * ldf + s];
    const double ar = (a.x - fi0.x) * inv_t, ai = (a.y - fi0.y) * inv_t;
    const double br = (b.x - fj0.x) * inv_t, bi = (b.y - fj0.y) * inv_t;
    cr += ar * br + ai * bi;  // a conj(b)
    ci += ai * br - ar * bi;
    pr += ar * br - ai * bi;  // a b
    pi += ai * br + ar * bi;
  }
  const double w = 1.0 / double(S);
  cov[i * ldc + j] = make_double2(cr * w, ci * w);
  if (pcov) pcov[i * ldp + j] = make_double2(pr * w, pi * w);
}

}  // namespace
}  // namespace fosb

extern "C" {

fosb_status fosb_field_samples(fosb_mesh mesh, const fosb_cov_kernel* ker, int64_t nsamp, const double* z,
                               double* xi) {
  using namespace fosb;
  if (!mesh || !ker || nsamp <= 0 || !z || !xi) return fail(FOSB_ERR_INVALID_ARG, "fosb_field_samples: bad arguments");
  if ((ker->kind != FOSB_COV_GAUSS && ker->kind != FOSB_COV_MATERN32) || !(ker->sigma > 0) || !(ker->ell > 0))
    return fail(FOSB_ERR_INVALID_ARG, "fosb_field_samples: bad covariance kernel");
  const int64_t V = int64_t(mesh->verts.size() / 3);
  const double* x = mesh->verts.data();
  const double s2 = ker->sigma * ker->sigma;
  // K (lower triangle, row-major) with a relative jitter of 1e-12 on the diagonal
  std::vector<double> L(size_t(V) * size_t(V), 0.0);
  for (int64_t p = 0; p < V; ++p)
    for (int64_t q = 0; q <= p; ++q) {
      const double dx = x[3 * p] - x[3 * q], dy = x[3 * p + 1] - x[3 * q + 1], dz = x[3 * p + 2] - x[3 * q + 2];
      const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
      double rho;
      if (ker->kind == FOSB_COV_GAUSS) {
        rho = std::exp(-r * r / (2.0 * ker->ell * ker->ell));
      } else {
        const double a = std::sqrt(3.0) * r / ker->ell;
        rho = (1.0 + a) * std::exp(-a);
      }
      L[size_t(p) * V + q] = s2 * rho + (p == q ? 1e-12 * s2 : 0.0);
    }
  // Cholesky K = L L^T in place (row-oriented: row p from the finished rows above it)
  for (int64_t p = 0; p < V; ++p) {
    double* Lp = &L[size_t(p) * V];
    for (int64_t q = 0; q < p; ++q) {
      const double* Lq = &L[size_t(q) * V];
      double acc = Lp[q];
      for (int64_t r = 0; r < q; ++r) acc -= Lp[r] * Lq[r];
      Lp[q] = acc / Lq[q];
    }
    double d = Lp[p];
    for (int64_t r = 0; r < p; ++r) d -= Lp[r] * Lp[r];
    if (!(d > 0.0)) return fail(FOSB_ERR_SINGULAR, "fosb_field_samples: the covariance is not positive definite");
    Lp[p] = std::sqrt(d);
  }
  for (int64_t s = 0; s < nsamp; ++s)
    for (int64_t p = 0; p < V; ++p) {
      const double* Lp = &L[size_t(p) * V];
      double acc = 0.0;
      for (int64_t q = 0; q <= p; ++q) acc += Lp[q] * z[s * V + q];
      xi[s * V + p] = acc;
    }
  return FOSB_OK;
}

fosb_status fosb_mesh_perturb(fosb_mesh base, const double* xi, double t, fosb_mesh* out) {
  using namespace fosb;
  if (!base || !xi || !out || !std::isfinite(t)) return fail(FOSB_ERR_INVALID_ARG, "fosb_mesh_perturb: bad arguments");
  const int64_t V = int64_t(base->verts.size() / 3), T = int64_t(base->tris.size() / 3);
  std::vector<double> v(base->verts);
  for (int64_t p = 0; p < V; ++p)
    for (int c = 0; c < 3; ++c) v[3 * p + c] += t * xi[p] * base->vnormals[3 * p + c];
  return fosb_mesh_create(v.data(), V, base->tris.data(), T, base->vnormals.data(), out);
}

fosb_status fosb_mc_moments(int64_t n3, int64_t nsamp, const void* Fs, int64_t ldf, const void* F0, double t,
                            void* mean, void* cov, int64_t ldc, void* pcov, int64_t ldp, void* stream) {
  using namespace fosb;
  if (n3 <= 0 || nsamp <= 0 || !Fs || ldf < nsamp || !F0 || !(t != 0.0) || !std::isfinite(t))
    return fail(FOSB_ERR_INVALID_ARG, "fosb_mc_moments: bad arguments");
  if ((cov && ldc < n3) || (pcov && (!cov || ldp < n3)))
    return fail(FOSB_ERR_INVALID_ARG, "fosb_mc_moments: bad covariance output (pcov needs cov)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double2* f = static_cast<const double2*>(Fs);
  if (mean) {
    mc_mean_kernel<<<unsigned((n3 + 127) / 128), 128, 0, s>>>(n3, nsamp, f, ldf, static_cast<double2*>(mean));
    FOSB_CUDA(launched());
  }
  if (cov) {
    mc_cov_kernel<<<unsigned((n3 * n3 + 127) / 128), 128, 0, s>>>(n3, nsamp, f, ldf, static_cast<const double2*>(F0),
                                                                 1.0 / t, static_cast<double2*>(cov), ldc,
                                                                 static_cast<double2*>(pcov), ldp);
    FOSB_CUDA(launched());
  }
  return FOSB_OK;
}

}  // extern "C"
