// Low-rank right-hand side of the tensor equations (Section VI, further work (ii)): the
// pivoted Cholesky factorisation of the covariance kernel matrix (Harbrecht, Peters and
// Schneider 2012), and the shape-derivative right-hand side applied to its columns.
//
// K_pq = sigma^2 rho(|x_p - x_q|) over n points (the vertices of several meshes, stacked)
// is never formed: each step evaluates one column.  With the residual diagonal d (d_p =
// K_pp = sigma^2 at the start) and the columns R_0 .. R_{m-1} written so far (R row-major,
// row k = column k of the factor over the n points), step m is
//   1. one CTA: err = sum of max(d, 0) over the points not chosen yet (the trace of the
//      Schur complement K - R^T R); stop if err <= tol trace(K) or no positive d is left;
//      otherwise p = argmax of d over those points (ties to the lowest index), l = sqrt(d_p),
//      and p is marked chosen;
//   2. per point j (32 points per CTA, the dot product split over its 8 warps):
//      R_m[j] = (K_jp - sum_{k<m} R_k[j] R_k[p]) / l, with l at j = p and 0 at points chosen
//      earlier; d_j -= R_m[j]^2.
// The host launches the steps in groups of 32 and reads the stop flag after each group, so
// no kernel waits on another.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "fosb_internal.h"

namespace fosb {
namespace {

struct LrState {
  int done;    // the stopping rule fired (or the last column was written)
  int rank;    // columns written
  double err;  // trace of the remainder with `rank` columns
};

constexpr int kPivThreads = 1024;
constexpr int kColGroups = 8;                 // warps per CTA of the column kernel
constexpr int kColThreads = 32 * kColGroups;  // 32 points per CTA
constexpr int kStage = 1024;  // R_k[p] values staged per pass

__device__ __forceinline__ double lr_kernel(int kind, double s2, double ell, const double* __restrict__ x, int64_t i,
                                            int64_t j) {
  const double dx = x[3 * i] - x[3 * j], dy = x[3 * i + 1] - x[3 * j + 1], dz = x[3 * i + 2] - x[3 * j + 2];
  const double r2 = dx * dx + dy * dy + dz * dz;
  if (kind == FOSB_COV_GAUSS) return s2 * exp(-r2 / (2.0 * ell * ell));
  const double sr = 1.7320508075688772 * sqrt(r2) / ell;  // sqrt(3) r / l
  return s2 * (1.0 + sr) * exp(-sr);
}

__global__ void lr_init_kernel(int64_t n, int kind, double s2, double ell, const double* __restrict__ x, double* d,
                               unsigned char* chosen, LrState* st) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j == 0) *st = LrState{0, 0, 0.0};
  if (j >= n) return;
  d[j] = lr_kernel(kind, s2, ell, x, j, j);
  chosen[j] = 0;
}

// Step m, part 1 (one CTA).  final_only: measure err and stop (after the last column).
__global__ void __launch_bounds__(kPivThreads) lr_pivot_kernel(int64_t n, double* d, unsigned char* chosen,
                                                               double thresh, int m, int final_only, int* piv,
                                                               double* lp, LrState* st) {
  if (st->done) return;
  __shared__ double s_v[kPivThreads / 32], s_e[kPivThreads / 32];
  __shared__ long long s_i[kPivThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double best = -1.0, err = 0.0;
  long long bi = -1;
  for (int64_t j = t; j < n; j += kPivThreads) {
    if (chosen[j]) continue;
    const double v = d[j];
    err += v > 0.0 ? v : 0.0;
    if (bi < 0 || v > best) {  // j grows within a thread: ties keep the lower index
      best = v;
      bi = j;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, best, o);
    const long long oi = __shfl_down_sync(0xffffffffu, bi, o);
    err += __shfl_down_sync(0xffffffffu, err, o);
    if (oi >= 0 && (bi < 0 || ov > best || (ov == best && oi < bi))) {
      best = ov;
      bi = oi;
    }
  }
  if (lane == 0) {
    s_v[warp] = best;
    s_i[warp] = bi;
    s_e[warp] = err;
  }
  __syncthreads();
  if (t == 0) {
    best = s_v[0];
    bi = s_i[0];
    err = s_e[0];
    for (int w = 1; w < kPivThreads / 32; ++w) {
      err += s_e[w];
      if (s_i[w] >= 0 && (bi < 0 || s_v[w] > best || (s_v[w] == best && s_i[w] < bi))) {
        best = s_v[w];
        bi = s_i[w];
      }
    }
    st->err = err;
    if (final_only || err <= thresh || bi < 0 || !(best > 0.0)) {
      st->done = 1;
      st->rank = m;
    } else {
      piv[m] = int(bi);
      lp[m] = sqrt(best);
      chosen[bi] = 1;
      st->rank = m + 1;
    }
  }
}

// Step m, part 2: column m of the factor and the diagonal update.  A CTA takes 32 points
// (lanes) and splits the dot product with the earlier columns over 8 warps (k = ty mod 8);
// the 8 partial sums are added in a fixed order by warp 0, which finishes the column.
__global__ void __launch_bounds__(kColThreads) lr_column_kernel(int64_t n, int kind, double s2, double ell,
                                                                const double* __restrict__ x, double* d,
                                                                const unsigned char* chosen, const int* piv,
                                                                const double* lp, double* R, int64_t ldr, int m,
                                                                const LrState* st) {
  if (st->rank <= m) return;  // the stopping rule fired at this step or earlier
  __shared__ double s_rp[kStage];
  __shared__ double s_part[kColGroups][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int p = piv[m];
  const double l = lp[m];
  const int64_t j = int64_t(blockIdx.x) * 32 + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < m; k0 += kStage) {
    const int kn = min(kStage, m - k0);
    __syncthreads();
    for (int i = threadIdx.x; i < kn; i += blockDim.x) s_rp[i] = R[int64_t(k0 + i) * ldr + p];
    __syncthreads();
    if (j < n)
      for (int k = ty; k < kn; k += kColGroups) acc += R[int64_t(k0 + k) * ldr + j] * s_rp[k];
  }
  s_part[ty][tx] = acc;
  __syncthreads();
  if (ty != 0 || j >= n) return;
  acc = 0.0;
#pragma unroll
  for (int g = 0; g < kColGroups; ++g) acc += s_part[g][tx];
  double v;
  if (j == p) {
    v = l;
  } else if (chosen[j]) {
    v = 0.0;
  } else {
    v = (lr_kernel(kind, s2, ell, x, j, p) - acc) / l;
    d[j] -= v * v;
  }
  R[int64_t(m) * ldr + j] = v;
}

// W[row, j] = sum_s B[row, s] R_j[col(row, s)], j < r: the shape-derivative right-hand side
// (4 ELL slots per row) applied to the factor's columns restricted to this mesh's vertices.
template <typename OutT>
__global__ void br_product_kernel(DevMesh m, const double* __restrict__ Bell, const double* __restrict__ R, int64_t ldr,
                                  int64_t r, OutT* W, int64_t ldw) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t row = blockIdx.y;
  if (j >= r) return;
  double wr = 0.0, wi = 0.0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const double v = R[j * ldr + m.ell_cols[4 * row + s]];
    wr += Bell[2 * (4 * row + s)] * v;
    wi += Bell[2 * (4 * row + s) + 1] * v;
  }
  W[2 * (row * ldw + j)] = OutT(wr);
  W[2 * (row * ldw + j) + 1] = OutT(wi);
}

inline unsigned lr_blocks(int64_t n, int bs) { return unsigned((n + bs - 1) / bs); }

}  // namespace

fosb_status pivoted_cholesky_kernel(const double* d_x, int64_t n, const fosb_cov_kernel& ker, double tol,
                                    int64_t max_rank, double* R, int64_t ldr, int64_t* rank, double* trace_err,
                                    cudaStream_t s) {
  const double s2 = ker.sigma * ker.sigma;
  const double thresh = tol * double(n) * s2;  // trace(K) = n sigma^2 (rho(0) = 1)
  Scratch dd(s), ch(s), pv(s), lv(s), stv(s);
  FOSB_CUDA(dd.alloc(sizeof(double) * n));
  FOSB_CUDA(ch.alloc(size_t(n)));
  FOSB_CUDA(pv.alloc(sizeof(int) * max_rank));
  FOSB_CUDA(lv.alloc(sizeof(double) * max_rank));
  FOSB_CUDA(stv.alloc(sizeof(LrState)));
  LrState* st = static_cast<LrState*>(stv.p);
  lr_init_kernel<<<lr_blocks(n, 256), 256, 0, s>>>(n, ker.kind, s2, ker.ell, d_x, dd.as<double>(),
                                                   static_cast<unsigned char*>(ch.p), st);
  FOSB_CUDA(launched());
  LrState h{};
  const unsigned gcol = lr_blocks(n, 32);
  for (int64_t m0 = 0; m0 < max_rank; m0 += 32) {
    const int64_t m1 = std::min<int64_t>(max_rank, m0 + 32);
    for (int64_t m = m0; m < m1; ++m) {
      lr_pivot_kernel<<<1, kPivThreads, 0, s>>>(n, dd.as<double>(), static_cast<unsigned char*>(ch.p), thresh, int(m), 0,
                                                static_cast<int*>(pv.p), lv.as<double>(), st);
      lr_column_kernel<<<gcol, kColThreads, 0, s>>>(n, ker.kind, s2, ker.ell, d_x, dd.as<double>(),
                                                    static_cast<const unsigned char*>(ch.p), static_cast<const int*>(pv.p),
                                                    lv.as<double>(), R, ldr, int(m), st);
      FOSB_CUDA(launched(2));
    }
    FOSB_CUDA(cudaMemcpyAsync(&h, st, sizeof(LrState), cudaMemcpyDeviceToHost, s));
    FOSB_CUDA(cudaStreamSynchronize(s));
    if (h.done) break;
  }
  if (!h.done) {  // every requested column written: the remainder's trace
    lr_pivot_kernel<<<1, kPivThreads, 0, s>>>(n, dd.as<double>(), static_cast<unsigned char*>(ch.p), thresh,
                                              int(max_rank), 1, static_cast<int*>(pv.p), lv.as<double>(), st);
    FOSB_CUDA(launched());
    FOSB_CUDA(cudaMemcpyAsync(&h, st, sizeof(LrState), cudaMemcpyDeviceToHost, s));
    FOSB_CUDA(cudaStreamSynchronize(s));
  }
  *rank = h.rank;
  if (trace_err) *trace_err = h.err;
  return FOSB_OK;
}

cudaError_t launch_br_product(const DevMesh& m, const double* B_ell, const double* R, int64_t ldr, int64_t r, bool fp32,
                              void* W, int64_t ldw, cudaStream_t s) {
  if (m.ne > 65535) return cudaErrorInvalidValue;  // grid.y bound
  dim3 grid(lr_blocks(r, 128), unsigned(m.ne));
  if (fp32)
    br_product_kernel<float><<<grid, 128, 0, s>>>(m, B_ell, R, ldr, r, static_cast<float*>(W), ldw);
  else
    br_product_kernel<double><<<grid, 128, 0, s>>>(m, B_ell, R, ldr, r, static_cast<double*>(W), ldw);
  return launched();
}

}  // namespace fosb
