// extern "C" entry points: argument checks, scratch management and the host loops
// (iterative refinement) around the kernels.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "fosb_internal.h"

using namespace fosb;

namespace {

int g_rules_nss[64];  // per device: the n_ss whose rules are in constant memory (0 = none)

fosb_status ensure_rules(int nss) {
  int dev = 0;
  FOSB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(FOSB_ERR_INVALID_ARG, "device index out of range");
  if (g_rules_nss[dev] != nss) {
    Rules r = make_rules(nss);
    upload_rules(r);
    upload_rules_adjoint(r);
    upload_rules_ff(r);
    upload_rules_pmchwt(r);
    FOSB_CUDA(cudaDeviceSynchronize());
    g_rules_nss[dev] = nss;
  }
  return FOSB_OK;
}

bool is_c64(int prec) { return prec == FOSB_FP32; }

fosb_status check_prec(int prec) {
  if (prec != FOSB_FP64 && prec != FOSB_MIXED && prec != FOSB_FP32)
    return fail(FOSB_ERR_INVALID_ARG, "unknown precision");
  return FOSB_OK;
}

fosb_status col_norms(const void* A, int64_t rows, int64_t cols, int64_t lda, double* d_buf, std::vector<double>& out,
                      cudaStream_t s) {
  FOSB_CUDA(absmax_c128(A, rows, cols, lda, d_buf, s));
  out.resize(cols);
  FOSB_CUDA(cudaMemcpyAsync(out.data(), d_buf, sizeof(double) * cols, cudaMemcpyDeviceToHost, s));
  FOSB_CUDA(cudaStreamSynchronize(s));
  return FOSB_OK;
}

// GMRES-based iterative refinement of one column (contiguous device n-vectors bc, xc; see
// FOSB_REFINE_GMRES in fosb.h): outer steps r = b - Z x (FP64-class), berr test, then the
// correction d from GMRES on M^-1 Z d = M^-1 r (M the complex64 factors) with FP64 Arnoldi
// (two-pass classical Gram-Schmidt, complex Givens rotations on the host) and x += d.
fosb_status gmres_ir_column(fosb_lu lu, const void* bc, void* xc, double bnorm, double tol, int max_outer,
                            int* iters, double* berr_out, cudaStream_t s) {
  using cd = std::complex<double>;
  const int64_t n = lu->n;
  constexpr int kM = 50;             // Krylov dimension per correction solve
  constexpr double kInnerTol = 1e-6;  // relative residual of the preconditioned correction equation
  Scratch V(s), w(s), r(s), hb(s), t32(s), nb(s);
  FOSB_CUDA(V.alloc(16 * n * (kM + 1)));
  FOSB_CUDA(w.alloc(16 * n));
  FOSB_CUDA(r.alloc(16 * n));
  FOSB_CUDA(hb.alloc(16 * (kM + 2)));
  FOSB_CUDA(t32.alloc(8 * n));
  FOSB_CUDA(nb.alloc(sizeof(double) * 2));
  char* Vp = static_cast<char*>(V.p);
  const int64_t ldv = kM + 1;
  auto col = [&](int j) { return static_cast<void*>(Vp + 16 * int64_t(j)); };
  auto precond = [&](const void* src, void* dst) -> fosb_status {  // dst = M^-1 src
    FOSB_CUDA(convert_c128_to_c64(src, n, 1, 1, t32.p, 1, s));
    FOSB_CUDA(getrs<float>(lu->lu, n, n, lu->ipiv, t32.p, 1, 1, s, lu->d_status, lu->dinv));
    FOSB_CUDA(convert_c64_to_c128(t32.p, n, 1, 1, dst, 1, s));
    return FOSB_OK;
  };
  // h (k values, host) = V(:, 0:k)^H x
  auto vdot = [&](int k, const void* x, int64_t incx, std::vector<cd>& h) -> fosb_status {
    FOSB_CUDA(gemm<double>(OP_C, OP_N, k, 1, n, 1.0, 0.0, V.p, ldv, x, incx, 0.0, hb.p, 1, s));
    h.resize(k);
    FOSB_CUDA(cudaMemcpyAsync(h.data(), hb.p, 16 * k, cudaMemcpyDeviceToHost, s));
    FOSB_CUDA(cudaStreamSynchronize(s));
    return FOSB_OK;
  };
  // ||x||_2 of a device vector with stride incx
  auto nrm2 = [&](const void* x, int64_t incx, double* out) -> fosb_status {
    FOSB_CUDA(gemm<double>(OP_C, OP_N, 1, 1, n, 1.0, 0.0, x, incx, x, incx, 0.0, hb.p, 1, s));
    cd v;
    FOSB_CUDA(cudaMemcpyAsync(&v, hb.p, 16, cudaMemcpyDeviceToHost, s));
    FOSB_CUDA(cudaStreamSynchronize(s));
    *out = std::sqrt(std::max(v.real(), 0.0));
    return FOSB_OK;
  };
  std::vector<double> rn, xn;
  double berr = INFINITY;
  int total = 0;
  for (int outer = 0;; ++outer) {
    FOSB_CUDA(copy_matrix(bc, n, 1, 1, r.p, 1, 16, s));
    FOSB_CUDA(gemm_c128_ff(OP_N, OP_N, n, 1, n, -1.0, 0.0, lu->zref, lu->ldz, xc, 1, 1.0, r.p, 1, s, lu->zff));
    FOSB_TRY(col_norms(r.p, n, 1, 1, nb.as<double>(), rn, s));
    FOSB_TRY(col_norms(xc, n, 1, 1, nb.as<double>(), xn, s));
    const double den = lu->znorm_inf * xn[0] + bnorm;
    berr = den > 0 ? rn[0] / den : 0.0;
    if (berr <= tol || outer >= max_outer) break;
    // GMRES on M^-1 Z d = M^-1 r, d = 0 initially
    FOSB_TRY(precond(r.p, w.p));
    double beta = 0.0;
    FOSB_TRY(nrm2(w.p, 1, &beta));
    if (!(beta > 0.0)) break;
    FOSB_CUDA(zscal_copy(n, 1.0 / beta, 0.0, w.p, 1, col(0), ldv, s));
    std::vector<std::vector<cd>> H;  // column j: H[0..j+1][j], rotated in place
    std::vector<double> cs;
    std::vector<cd> sn, g(1, cd(beta, 0.0)), h, h2;
    int jm = 0;
    for (int j = 0; j < kM; ++j) {
      FOSB_CUDA(gemm_c128_ff(OP_N, OP_N, n, 1, n, 1.0, 0.0, lu->zref, lu->ldz, col(j), ldv, 0.0, r.p, 1, s, lu->zff));
      FOSB_TRY(precond(r.p, w.p));
      // two passes of classical Gram-Schmidt against v_0 .. v_j
      FOSB_TRY(vdot(j + 1, w.p, 1, h));
      FOSB_CUDA(cudaMemcpyAsync(hb.p, h.data(), 16 * (j + 1), cudaMemcpyHostToDevice, s));
      FOSB_CUDA(gemm<double>(OP_N, OP_N, n, 1, j + 1, -1.0, 0.0, V.p, ldv, hb.p, 1, 1.0, w.p, 1, s));
      FOSB_TRY(vdot(j + 1, w.p, 1, h2));
      FOSB_CUDA(cudaMemcpyAsync(hb.p, h2.data(), 16 * (j + 1), cudaMemcpyHostToDevice, s));
      FOSB_CUDA(gemm<double>(OP_N, OP_N, n, 1, j + 1, -1.0, 0.0, V.p, ldv, hb.p, 1, 1.0, w.p, 1, s));
      for (int i = 0; i <= j; ++i) h[i] += h2[i];
      double hn = 0.0;
      FOSB_TRY(nrm2(w.p, 1, &hn));
      std::vector<cd> hc(h);
      hc.push_back(cd(hn, 0.0));
      for (int i = 0; i < j; ++i) {  // earlier rotations
        const cd a = hc[i], b = hc[i + 1];
        hc[i] = cs[i] * a + sn[i] * b;
        hc[i + 1] = -std::conj(sn[i]) * a + cs[i] * b;
      }
      const cd a = hc[j], b = hc[j + 1];
      double c;
      cd sv;
      if (std::abs(a) == 0.0) {
        c = 0.0;
        sv = cd(1.0, 0.0);
      } else {
        const double nu = std::sqrt(std::norm(a) + std::norm(b));
        c = std::abs(a) / nu;
        sv = (a / std::abs(a)) * std::conj(b) / nu;
      }
      cs.push_back(c);
      sn.push_back(sv);
      hc[j] = c * a + sv * b;
      hc[j + 1] = 0.0;
      g.push_back(-std::conj(sv) * g[j]);
      g[j] = c * g[j];
      H.push_back(hc);
      jm = j + 1;
      ++total;
      if (std::abs(g[j + 1]) <= kInnerTol * beta || !(hn > 0.0)) break;
      FOSB_CUDA(zscal_copy(n, 1.0 / hn, 0.0, w.p, 1, col(j + 1), ldv, s));
    }
    // y = R^-1 g (R upper triangular jm x jm), d = V y, x += d
    std::vector<cd> y(jm);
    for (int i = jm - 1; i >= 0; --i) {
      cd acc = g[i];
      for (int k = i + 1; k < jm; ++k) acc -= H[k][i] * y[k];
      y[i] = H[i][i] == cd(0.0) ? cd(0.0) : acc / H[i][i];
    }
    FOSB_CUDA(cudaMemcpyAsync(hb.p, y.data(), 16 * jm, cudaMemcpyHostToDevice, s));
    FOSB_CUDA(gemm<double>(OP_N, OP_N, n, 1, jm, 1.0, 0.0, V.p, ldv, hb.p, 1, 1.0, xc, 1, s));
    FOSB_CUDA(cudaStreamSynchronize(s));  // y is released at the end of this step
  }
  *iters += total;
  *berr_out = berr;
  return FOSB_OK;
}

// X = Z^{-1} B through the handle (see fosb_solve).
fosb_status solve_internal(fosb_lu lu, const void* B, int64_t nrhs, int64_t ldb, void* X, int64_t ldx,
                           const fosb_refine_opts* ropt, fosb_solve_stats* stats, cudaStream_t s) {
  const int64_t n = lu->n;
  if (stats) {
    stats->iters = 0;
    stats->backward_error = 0.0;
  }
  if (nrhs == 0 || n == 0) return FOSB_OK;
  if (lu->prec == FOSB_FP64) {
    if (X != B) FOSB_CUDA(copy_matrix(B, n, nrhs, ldb, X, ldx, 16, s));
    FOSB_CUDA(getrs<double>(lu->lu, n, n, lu->ipiv, X, nrhs, ldx, s));
    return FOSB_OK;
  }
  if (lu->prec == FOSB_FP32) {
    if (X != B) FOSB_CUDA(copy_matrix(B, n, nrhs, ldb, X, ldx, 8, s));
    FOSB_CUDA(getrs<float>(lu->lu, n, n, lu->ipiv, X, nrhs, ldx, s, lu->d_status, lu->dinv));
    return FOSB_OK;
  }
  // MIXED: complex64 factors, FP64 residuals.
  const int max_iters = ropt ? ropt->max_iters : 10;
  // default: the FP64 residual floor grows like sqrt(n) eps; stop at 8 sqrt(n) eps (>= 64 eps)
  const double eps = std::ldexp(1.0, -52);
  const double tol = (ropt && ropt->tol > 0) ? ropt->tol : std::max(64.0, 8.0 * std::sqrt(double(n))) * eps;
  Scratch r(s), d(s), bkeep(s), nb(s);
  FOSB_CUDA(r.alloc(sizeof(double) * 2 * n * nrhs));
  FOSB_CUDA(d.alloc(sizeof(float) * 2 * n * nrhs));
  FOSB_CUDA(nb.alloc(sizeof(double) * nrhs));
  const void* Bsrc = B;
  int64_t ldbs = ldb;
  if (X == B) {  // keep the right-hand side: X is overwritten
    FOSB_CUDA(bkeep.alloc(sizeof(double) * 2 * n * nrhs));
    FOSB_CUDA(copy_matrix(B, n, nrhs, ldb, bkeep.p, nrhs, 16, s));
    Bsrc = bkeep.p;
    ldbs = nrhs;
  }
  std::vector<double> bn, xn, rn;
  FOSB_TRY(col_norms(Bsrc, n, nrhs, ldbs, nb.as<double>(), bn, s));
  // x0
  FOSB_CUDA(convert_c128_to_c64(Bsrc, n, nrhs, ldbs, d.p, nrhs, s));
  FOSB_CUDA(getrs<float>(lu->lu, n, n, lu->ipiv, d.p, nrhs, nrhs, s, lu->d_status, lu->dinv));
  FOSB_CUDA(convert_c64_to_c128(d.p, n, nrhs, nrhs, X, ldx, s));
  const int solver = ropt ? ropt->solver : FOSB_REFINE_AUTO;
  if (solver < FOSB_REFINE_AUTO || solver > FOSB_REFINE_GMRES)
    return fail(FOSB_ERR_INVALID_ARG, "fosb_solve: unknown refinement solver");
  double prev = INFINITY, prev2 = INFINITY, berr = INFINITY;
  int it = 0;
  for (; solver != FOSB_REFINE_GMRES;) {
    FOSB_CUDA(copy_matrix(Bsrc, n, nrhs, ldbs, r.p, nrhs, 16, s));
    if (lu->zdig && nrhs > 4)  // 5 or more right-hand sides: digit-split bf16 tensor cores
      FOSB_CUDA(oz_gemm(n, nrhs, n, -1.0, 0.0, lu->zdig, lu->zex, X, ldx, 1.0, r.p, nrhs, lu->d_status, s));
    else
      FOSB_CUDA(gemm_c128_ff(OP_N, OP_N, n, nrhs, n, -1.0, 0.0, lu->zref, lu->ldz, X, ldx, 1.0, r.p, nrhs, s,
                             lu->zff));
    FOSB_TRY(col_norms(r.p, n, nrhs, nrhs, nb.as<double>(), rn, s));
    FOSB_TRY(col_norms(X, n, nrhs, ldx, nb.as<double>(), xn, s));
    berr = 0.0;
    for (int64_t c = 0; c < nrhs; ++c) {
      double den = lu->znorm_inf * xn[c] + bn[c];
      berr = std::max(berr, den > 0 ? rn[c] / den : 0.0);
    }
    if (berr <= tol || it >= max_iters) break;
    if (berr >= prev && prev >= prev2) break;  // no decrease over two steps
    if (berr < 1e-13 && berr > 0.5 * prev) break;  // at the rounding floor: progress has stalled
    prev2 = prev;
    prev = berr;
    FOSB_CUDA(convert_c128_to_c64(r.p, n, nrhs, nrhs, d.p, nrhs, s));
    FOSB_CUDA(getrs<float>(lu->lu, n, n, lu->ipiv, d.p, nrhs, nrhs, s, lu->d_status, lu->dinv));
    FOSB_CUDA(axpy_c64_into_c128(d.p, n, nrhs, nrhs, X, ldx, s));
    ++it;
  }
  if (solver == FOSB_REFINE_GMRES || (solver == FOSB_REFINE_AUTO && !(berr <= tol) && !(berr <= 1e-13))) {
    // GMRES-IR column by column for the columns refinement left above the tolerance
    Scratch xc(s);
    FOSB_CUDA(xc.alloc(16 * n));
    berr = 0.0;
    for (int64_t c = 0; c < nrhs; ++c) {
      const char* bcol = static_cast<const char*>(Bsrc) + 16 * c;
      char* xcol = static_cast<char*>(X) + 16 * c;
      Scratch bcs(s);
      FOSB_CUDA(bcs.alloc(16 * n));
      FOSB_CUDA(copy_matrix(bcol, n, 1, ldbs, bcs.p, 1, 16, s));
      FOSB_CUDA(copy_matrix(xcol, n, 1, ldx, xc.p, 1, 16, s));
      double bc_err = 0.0;
      FOSB_TRY(gmres_ir_column(lu, bcs.p, xc.p, bn[c], tol, max_iters, &it, &bc_err, s));
      FOSB_CUDA(copy_matrix(xc.p, n, 1, 1, xcol, ldx, 16, s));
      berr = std::max(berr, bc_err);
    }
  }
  if (stats) {
    stats->iters = it;
    stats->backward_error = berr;
  }
  int status = 0;  // tensor-core triangular updates report a bounded-wait time-out here
  FOSB_CUDA(cudaMemcpyAsync(&status, lu->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  FOSB_CUDA(cudaStreamSynchronize(s));
  if (status == FOSB_ERR_TIMEOUT) return fail(FOSB_ERR_TIMEOUT, "fosb_solve: tensor-core wait timed out");
  if (!(berr <= tol) && !(berr <= 1e-13)) {
    return fail(FOSB_ERR_NOT_CONVERGED, "fosb_solve: refinement stalled at backward error " + std::to_string(berr));
  }
  return FOSB_OK;
}

}  // namespace

fosb_status fosb::ensure_rules_for(int nss) { return ensure_rules(nss); }

extern "C" {

fosb_status fosb_assemble_efie(fosb_mesh mesh, double k, const fosb_quad_opts* opts, int prec, void* Z, int64_t ldz,
                               const double* inc, int64_t n_inc, void* b, int64_t ldb, void* stream) {
  if (!mesh || !Z) return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie: NULL mesh or Z");
  FOSB_TRY(check_prec(prec));
  const int64_t N = mesh->d.ne;
  if (!(k > 0.0) || !std::isfinite(k)) return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie: k must be > 0");
  if (ldz < N) return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie: ldz < N");
  if (n_inc < 0 || (n_inc > 0 && (!inc || !b || ldb < n_inc)))
    return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie: bad incidence arguments");
  int nss = opts && opts->n_ss > 0 ? opts->n_ss : 5;
  int arith = opts ? opts->arith : FOSB_ASM_FP64;
  if (nss > 12) return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie: n_ss must be in 1..12");
  if (arith < 0 || arith > 2) return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie: unknown arith");
  if (is_c64(prec)) arith = FOSB_ASM_FP32;
  else if (arith == FOSB_ASM_FP32)
    return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie: FP32 regular pairs need prec = FOSB_FP32");
  if (arith == FOSB_ASM_FF && k * mesh->d.diameter >= ff_max_phase())
    return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie: k * mesh diameter = " + std::to_string(k * mesh->d.diameter) +
                                          " exceeds the float-float phase range " + std::to_string(ff_max_phase()) +
                                          "; use FOSB_ASM_FP64");
  for (int64_t s = 0; s < n_inc; ++s)
    for (int c = 0; c < 9; ++c)
      if (!std::isfinite(inc[9 * s + c])) return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie: non-finite incidence");
  FOSB_TRY(ensure_rules(nss));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t elem = is_c64(prec) ? 8 : 16;
  FOSB_CUDA(cudaMemset2DAsync(Z, ldz * elem, 0, N * elem, N, s));
  FOSB_CUDA(launch_assemble_regular(mesh->d, k, arith, Z, ldz, s));
  FOSB_CUDA(launch_assemble_singular(mesh->d, k, nss, is_c64(prec), Z, ldz, s));
  if (n_inc > 0) {
    // copied from a pageable buffer of our own: cudaMemcpyAsync returns once the bytes are
    // staged, so the call needs no synchronisation whatever memory the caller's `inc` is in
    const std::vector<double> hinc(inc, inc + 9 * n_inc);
    Scratch dinc(s);
    FOSB_CUDA(dinc.alloc(sizeof(double) * 9 * n_inc));
    FOSB_CUDA(cudaMemcpyAsync(dinc.p, hinc.data(), sizeof(double) * 9 * n_inc, cudaMemcpyHostToDevice, s));
    FOSB_CUDA(cudaMemset2DAsync(b, ldb * elem, 0, n_inc * elem, N, s));
    FOSB_CUDA(launch_rhs(mesh->d, k, dinc.as<double>(), n_inc, is_c64(prec), b, ldb, s));
  }
  return FOSB_OK;
}

fosb_status fosb_factor(const void* Z, int64_t n, int64_t ldz, int prec, fosb_lu* out, void* stream) {
  if (!Z || !out || n <= 0 || ldz < n) return fail(FOSB_ERR_INVALID_ARG, "fosb_factor: bad arguments");
  FOSB_TRY(check_prec(prec));
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  fosb_lu lu = new (std::nothrow) fosb_lu_s;
  if (!lu) return fail(FOSB_ERR_OOM, "fosb_factor: host allocation");
  cudaGetDevice(&lu->device);
  lu->prec = prec;
  lu->n = n;
  const size_t elem = prec == FOSB_FP64 ? 16 : 8;
  auto cleanup = [&](fosb_status st) {
    fosb_lu_destroy(lu);
    return st;
  };
  cudaError_t e = cudaMalloc(&lu->lu, elem * n * n);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "fosb_factor: factor storage"));
  if ((e = cudaMalloc(&lu->ipiv, sizeof(int32_t) * n)) != cudaSuccess ||
      (e = cudaMalloc(&lu->d_status, sizeof(int) * 2)) != cudaSuccess)
    return cleanup(cuda_fail(e, "fosb_factor: pivots"));
  if ((e = cudaMemsetAsync(lu->d_status, 0, sizeof(int) * 2, s)) != cudaSuccess)
    return cleanup(cuda_fail(e, "fosb_factor"));
  if (prec == FOSB_FP64)
    e = copy_matrix(Z, n, n, ldz, lu->lu, n, 16, s);
  else if (prec == FOSB_MIXED)
    e = convert_c128_to_c64(Z, n, n, ldz, lu->lu, n, s);
  else
    e = copy_matrix(Z, n, n, ldz, lu->lu, n, 8, s);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "fosb_factor: copy"));
  if (prec == FOSB_MIXED) {
    lu->zref = Z;
    lu->ldz = ldz;
    // the residual GEMMs read Z as (hi, lo) float pairs: split it once here (n x n float4)
    if ((e = cudaMalloc(&lu->zff, sizeof(float) * 4 * n * n)) != cudaSuccess ||
        (e = split_ff(Z, n, n, ldz, lu->zff, n, s)) != cudaSuccess)
      return cleanup(cuda_fail(e, "fosb_factor: split copy of Z"));
    // and as exact bf16 digits for residuals with many right-hand sides (about 28 n^2 bytes)
    if (n >= 256) {
      if ((e = cudaMalloc(&lu->zdig, oz_a_bytes(n, n))) != cudaSuccess ||
          (e = cudaMalloc(reinterpret_cast<void**>(&lu->zex), sizeof(int) * n)) != cudaSuccess ||
          (e = oz_prepare_a(Z, n, n, ldz, lu->zdig, lu->zex, s)) != cudaSuccess)
        return cleanup(cuda_fail(e, "fosb_factor: digit tiles of Z"));
    }
    Scratch nrm(s);
    if ((e = nrm.alloc(sizeof(double))) != cudaSuccess || (e = norm_inf_c128(Z, n, n, ldz, nrm.as<double>(), s)) ||
        (e = cudaMemcpyAsync(&lu->znorm_inf, nrm.p, sizeof(double), cudaMemcpyDeviceToHost, s)))
      return cleanup(cuda_fail(e, "fosb_factor: norm"));
  }
  fosb_status st = prec == FOSB_FP64 ? getrf<double>(lu->lu, n, n, lu->ipiv, lu->d_status, s)
                                     : getrf<float>(lu->lu, n, n, lu->ipiv, lu->d_status, s);
  if (st != FOSB_OK) return cleanup(st);
  int status = 0;
  std::vector<int32_t> ipiv(n);
  if ((e = cudaMemcpyAsync(&status, lu->d_status, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(ipiv.data(), lu->ipiv, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return cleanup(cuda_fail(e, "fosb_factor: status"));
  if (status == FOSB_ERR_TIMEOUT) return cleanup(fail(FOSB_ERR_TIMEOUT, "fosb_factor: panel grid barrier timed out"));
  if (status == FOSB_ERR_SINGULAR) return cleanup(fail(FOSB_ERR_SINGULAR, "fosb_factor: zero pivot"));
  // compose the row interchanges into one permutation: (P b)[i] = b[perm[i]]
  std::vector<int32_t> perm(n);
  for (int64_t i = 0; i < n; ++i) perm[i] = int32_t(i);
  for (int64_t i = 0; i < n; ++i) {
    int32_t p = ipiv[i];
    if (p < 0 || p >= n) return cleanup(fail(FOSB_ERR_CUDA, "fosb_factor: corrupt pivot"));
    std::swap(perm[i], perm[p]);
  }
  // stream-ordered (a plain cudaMemcpy would also wait for the legacy default stream's work);
  // perm is pageable, so the call returns once it is staged
  if ((e = cudaMemcpyAsync(lu->ipiv, perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s)))
    return cleanup(cuda_fail(e, "fosb_factor: permutation"));
  if (prec != FOSB_FP64) {  // inverted diagonal blocks for the streaming triangular sweeps
    if ((e = cudaMalloc(&lu->dinv, tri_block_inverses_bytes(n))) != cudaSuccess ||
        (e = tri_block_inverses_c64(lu->lu, n, n, lu->dinv, s)) != cudaSuccess)
      return cleanup(cuda_fail(e, "fosb_factor: diagonal-block inverses"));
  }
  *out = lu;
  return FOSB_OK;
}

fosb_status fosb_solve(fosb_lu lu, char op, const void* B, int64_t nrhs, int64_t ldb, void* X, int64_t ldx,
                       const fosb_refine_opts* ropt, fosb_solve_stats* stats, void* stream) {
  if (!lu || !B || !X || nrhs < 0 || ldb < nrhs || ldx < nrhs) return fail(FOSB_ERR_INVALID_ARG, "fosb_solve: bad arguments");
  if (op != 'N' && op != 'n') return fail(FOSB_ERR_INVALID_ARG, "fosb_solve: only op = 'N' is supported");
  if (X == B && ldx != ldb) return fail(FOSB_ERR_INVALID_ARG, "fosb_solve: aliased X and B need equal leading dimensions");
  return solve_internal(lu, B, nrhs, ldb, X, ldx, ropt, stats, static_cast<cudaStream_t>(stream));
}

fosb_status fosb_lu_info(fosb_lu lu, int64_t* n, int* prec, double* znorm_inf) {
  if (!lu) return fail(FOSB_ERR_INVALID_ARG, "fosb_lu_info: NULL handle");
  if (n) *n = lu->n;
  if (prec) *prec = lu->prec;
  if (znorm_inf) *znorm_inf = lu->znorm_inf;
  return FOSB_OK;
}

fosb_status fosb_lu_destroy(fosb_lu lu) {
  if (!lu) return FOSB_OK;
  if (lu->lu) cudaFree(lu->lu);
  if (lu->ipiv) cudaFree(lu->ipiv);
  if (lu->d_status) cudaFree(lu->d_status);
  if (lu->zff) cudaFree(lu->zff);
  if (lu->dinv) cudaFree(lu->dinv);
  if (lu->zdig) cudaFree(lu->zdig);
  if (lu->zex) cudaFree(lu->zex);
  delete lu;
  return FOSB_OK;
}

fosb_status fosb_covariance(fosb_mesh m1, fosb_lu lu1, const void* u1, fosb_mesh m2, fosb_lu lu2, const void* u2,
                            double k, const fosb_cov_kernel* kernel, int pseudo, void* Sigma, int64_t lds,
                            const fosb_refine_opts* ropt, void* stream) {
  if (!m1 || !m2 || !lu1 || !lu2 || !u1 || !u2 || !kernel || !Sigma)
    return fail(FOSB_ERR_INVALID_ARG, "fosb_covariance: NULL argument");
  if (lu1->prec != lu2->prec) return fail(FOSB_ERR_INVALID_ARG, "fosb_covariance: factor precisions differ");
  if (lu1->n != m1->d.ne || lu2->n != m2->d.ne) return fail(FOSB_ERR_INVALID_ARG, "fosb_covariance: factor size != mesh edges");
  if (lds < m2->d.ne) return fail(FOSB_ERR_INVALID_ARG, "fosb_covariance: lds < N2");
  if (!(k > 0) || !(kernel->ell > 0) || !(kernel->sigma >= 0) || (kernel->kind != FOSB_COV_GAUSS && kernel->kind != FOSB_COV_MATERN32))
    return fail(FOSB_ERR_INVALID_ARG, "fosb_covariance: bad k or kernel");
  FOSB_TRY(ensure_rules(5));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int prec = lu1->prec;
  const bool c64 = is_c64(prec);
  const size_t elem = c64 ? 8 : 16;
  const DevMesh& d1 = m1->d;
  const DevMesh& d2 = m2->d;
  Scratch b1(s), b2(s), y1(s), y2(s);
  FOSB_CUDA(b1.alloc(sizeof(double) * 8 * d1.ne));
  FOSB_CUDA(b2.alloc(sizeof(double) * 8 * d2.ne));
  FOSB_CUDA(launch_sd_rhs(d1, k, u1, c64, b1.as<double>(), s));
  FOSB_CUDA(launch_sd_rhs(d2, k, u2, c64, b2.as<double>(), s));
  // rank r = min(V1, V2): Sigma = (Z1^{-1} L1)(Z2^{-1} L2)^H with L1 = B1 K12, L2 = B2 when V2 <= V1
  const bool k_on_1 = d2.nv <= d1.nv;
  const int64_t r = k_on_1 ? d2.nv : d1.nv;
  FOSB_CUDA(y1.alloc(elem * d1.ne * r));
  FOSB_CUDA(y2.alloc(elem * d2.ne * r));
  if (k_on_1) {
    FOSB_CUDA(launch_bk_product(d1, b1.as<double>(), d2, *kernel, c64, y1.p, r, s));
    FOSB_CUDA(launch_ell_to_dense(d2, b2.as<double>(), false, c64, y2.p, r, s));
  } else {
    FOSB_CUDA(launch_ell_to_dense(d1, b1.as<double>(), false, c64, y1.p, r, s));
    FOSB_CUDA(launch_bk_product(d2, b2.as<double>(), d1, *kernel, c64, y2.p, r, s));
  }
  FOSB_TRY(solve_internal(lu1, y1.p, r, r, y1.p, r, ropt, nullptr, s));
  FOSB_TRY(solve_internal(lu2, y2.p, r, r, y2.p, r, ropt, nullptr, s));
  cudaError_t e;
  if (c64)
    e = gemm<float>(OP_N, pseudo ? OP_T : OP_C, d1.ne, d2.ne, r, 1.0, 0.0, y1.p, r, y2.p, r, 0.0, Sigma, lds, s);
  else if (prec == FOSB_MIXED)
    e = gemm_c128_ff(OP_N, pseudo ? OP_T : OP_C, d1.ne, d2.ne, r, 1.0, 0.0, y1.p, r, y2.p, r, 0.0, Sigma, lds, s);
  else
    e = gemm<double>(OP_N, pseudo ? OP_T : OP_C, d1.ne, d2.ne, r, 1.0, 0.0, y1.p, r, y2.p, r, 0.0, Sigma, lds, s);
  FOSB_CUDA(e);
  return FOSB_OK;
}

fosb_status fosb_kernel_lowrank(const fosb_mesh* meshes, int64_t nmesh, const fosb_cov_kernel* kernel, double tol,
                                int64_t max_rank, double* R, int64_t ldr, int64_t* rank, double* trace_err,
                                void* stream) {
  if (!meshes || nmesh < 1 || !kernel || !R || !rank) return fail(FOSB_ERR_INVALID_ARG, "fosb_kernel_lowrank: NULL argument");
  if ((kernel->kind != FOSB_COV_GAUSS && kernel->kind != FOSB_COV_MATERN32) || !(kernel->sigma > 0) ||
      !(kernel->ell > 0) || !std::isfinite(kernel->sigma) || !std::isfinite(kernel->ell))
    return fail(FOSB_ERR_INVALID_ARG, "fosb_kernel_lowrank: bad covariance kernel");
  if (!(tol >= 0) || !std::isfinite(tol) || max_rank < 1) return fail(FOSB_ERR_INVALID_ARG, "fosb_kernel_lowrank: tol < 0 or max_rank < 1");
  std::vector<double> x;
  for (int64_t i = 0; i < nmesh; ++i) {
    if (!meshes[i]) return fail(FOSB_ERR_INVALID_ARG, "fosb_kernel_lowrank: NULL mesh");
    x.insert(x.end(), meshes[i]->verts.begin(), meshes[i]->verts.end());
  }
  const int64_t n = int64_t(x.size() / 3);
  if (ldr < n) return fail(FOSB_ERR_INVALID_ARG, "fosb_kernel_lowrank: ldr < total vertices");
  max_rank = std::min(max_rank, n);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Scratch dx(s);
  FOSB_CUDA(dx.alloc(sizeof(double) * x.size()));
  FOSB_CUDA(cudaMemcpyAsync(dx.p, x.data(), sizeof(double) * x.size(), cudaMemcpyHostToDevice, s));
  FOSB_TRY(pivoted_cholesky_kernel(dx.as<double>(), n, *kernel, tol, max_rank, R, ldr, rank, trace_err, s));
  return FOSB_OK;
}

namespace {
cudaError_t gemm_prec(int prec, int opA, int opB, int64_t M, int64_t N, int64_t K, double ar, const void* A, int64_t lda,
                      const void* B, int64_t ldb, double beta, void* C, int64_t ldc, cudaStream_t s) {
  if (is_c64(prec)) return gemm<float>(opA, opB, M, N, K, ar, 0.0, A, lda, B, ldb, beta, C, ldc, s);
  if (prec == FOSB_MIXED) return gemm_c128_ff(opA, opB, M, N, K, ar, 0.0, A, lda, B, ldb, beta, C, ldc, s);
  return gemm<double>(opA, opB, M, N, K, ar, 0.0, A, lda, B, ldb, beta, C, ldc, s);
}
}  // namespace

fosb_status fosb_covariance_lowrank(fosb_mesh mesh, fosb_lu lu, const void* u, double k, const double* R, int64_t ldr,
                                    int64_t r, const double* dirs, int64_t n_dir, const fosb_refine_opts* ropt,
                                    void* Y, int64_t ldy, void* stream) {
  if (!mesh || !lu || !u || !R || !dirs || !Y) return fail(FOSB_ERR_INVALID_ARG, "fosb_covariance_lowrank: NULL argument");
  if (lu->n != mesh->d.ne) return fail(FOSB_ERR_INVALID_ARG, "fosb_covariance_lowrank: factor size != mesh edges");
  if (r < 1 || ldr < mesh->d.nv || n_dir < 1 || ldy < r || !(k > 0))
    return fail(FOSB_ERR_INVALID_ARG, "fosb_covariance_lowrank: bad size, leading dimension or k");
  FOSB_TRY(ensure_rules(5));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int prec = lu->prec;
  const bool c64 = is_c64(prec);
  const size_t elem = c64 ? 8 : 16;
  const DevMesh& d = mesh->d;
  const int64_t N = d.ne, nd3 = 3 * n_dir;
  Scratch bell(s), w(s), ddirs(s), a(s);
  FOSB_CUDA(bell.alloc(sizeof(double) * 8 * N));
  FOSB_CUDA(launch_sd_rhs(d, k, u, c64, bell.as<double>(), s));
  FOSB_CUDA(w.alloc(elem * N * r));
  FOSB_CUDA(launch_br_product(d, bell.as<double>(), R, ldr, r, c64, w.p, r, s));
  FOSB_TRY(solve_internal(lu, w.p, r, r, w.p, r, ropt, nullptr, s));
  FOSB_CUDA(ddirs.alloc(sizeof(double) * 3 * n_dir));
  FOSB_CUDA(cudaMemcpyAsync(ddirs.p, dirs, sizeof(double) * 3 * n_dir, cudaMemcpyHostToDevice, s));
  FOSB_CUDA(a.alloc(elem * nd3 * N));
  FOSB_CUDA(cudaMemsetAsync(a.p, 0, elem * nd3 * N, s));
  FOSB_CUDA(launch_farfield_matrix(d, k, ddirs.as<double>(), n_dir, c64, a.p, s));
  FOSB_CUDA(gemm_prec(prec, OP_N, OP_N, nd3, r, N, 1.0, a.p, N, w.p, r, 0.0, Y, ldy, s));
  FOSB_CUDA(cudaStreamSynchronize(s));
  return FOSB_OK;
}

fosb_status fosb_lowrank_combine(int64_t nd3, int64_t r, const void* Y1, int64_t ldy1, const void* Y2, int64_t ldy2,
                                 double weight, int hermitian_mirror, int pseudo, int prec, void* out, int64_t ldo,
                                 int accumulate, void* stream) {
  if (!Y1 || !Y2 || !out || nd3 < 1 || r < 1 || ldy1 < r || ldy2 < r || ldo < nd3)
    return fail(FOSB_ERR_INVALID_ARG, "fosb_lowrank_combine: bad argument");
  FOSB_TRY(check_prec(prec));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int op = pseudo ? OP_T : OP_C;
  if (!hermitian_mirror) {
    FOSB_CUDA(gemm_prec(prec, OP_N, op, nd3, nd3, r, weight, Y1, ldy1, Y2, ldy2, accumulate ? 1.0 : 0.0, out, ldo, s));
    return FOSB_OK;
  }
  Scratch mm(s);
  FOSB_CUDA(mm.alloc((is_c64(prec) ? 8 : 16) * nd3 * nd3));
  FOSB_CUDA(gemm_prec(prec, OP_N, op, nd3, nd3, r, 1.0, Y1, ldy1, Y2, ldy2, 0.0, mm.p, nd3, s));
  FOSB_CUDA(add_mirrored(mm.p, nd3, nd3, op, weight, accumulate != 0, is_c64(prec), out, ldo, s));
  return FOSB_OK;
}

fosb_status fosb_farfield_moments(fosb_mesh m1, fosb_mesh m2, double k, const double* dirs, int64_t n_dir,
                                  const void* X, int64_t ldx, int64_t ncols, double weight, int hermitian_mirror,
                                  int pseudo, int prec, void* out, int64_t ldo, int accumulate, void* stream) {
  if (!m1 || !dirs || !X || !out || n_dir <= 0) return fail(FOSB_ERR_INVALID_ARG, "fosb_farfield_moments: NULL argument");
  FOSB_TRY(check_prec(prec));
  if (!(k > 0)) return fail(FOSB_ERR_INVALID_ARG, "fosb_farfield_moments: k must be > 0");
  const int64_t nd3 = 3 * n_dir;
  if (m2 ? (ldx < m2->d.ne || ldo < nd3) : (ncols <= 0 || ldx < ncols || ldo < ncols))
    return fail(FOSB_ERR_INVALID_ARG, "fosb_farfield_moments: bad leading dimension");
  FOSB_TRY(ensure_rules(5));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool c64 = is_c64(prec);
  const size_t elem = c64 ? 8 : 16;
  Scratch ddirs(s), a1(s), a2(s), t(s), mm(s);
  FOSB_CUDA(ddirs.alloc(sizeof(double) * 3 * n_dir));
  FOSB_CUDA(cudaMemcpyAsync(ddirs.p, dirs, sizeof(double) * 3 * n_dir, cudaMemcpyHostToDevice, s));
  FOSB_CUDA(a1.alloc(elem * nd3 * m1->d.ne));
  FOSB_CUDA(cudaMemsetAsync(a1.p, 0, elem * nd3 * m1->d.ne, s));
  FOSB_CUDA(launch_farfield_matrix(m1->d, k, ddirs.as<double>(), n_dir, c64, a1.p, s));
  auto G = [&](int opA, int opB, int64_t M, int64_t N, int64_t K, double ar, const void* A, int64_t lda,
               const void* B, int64_t ldb, double beta, void* C, int64_t ldc) {
    if (c64) return gemm<float>(opA, opB, M, N, K, ar, 0.0, A, lda, B, ldb, beta, C, ldc, s);
    if (prec == FOSB_MIXED) return gemm_c128_ff(opA, opB, M, N, K, ar, 0.0, A, lda, B, ldb, beta, C, ldc, s);
    return gemm<double>(opA, opB, M, N, K, ar, 0.0, A, lda, B, ldb, beta, C, ldc, s);
  };
  if (!m2) {
    FOSB_CUDA(G(OP_N, OP_N, nd3, ncols, m1->d.ne, weight, a1.p, m1->d.ne, X, ldx, accumulate ? 1.0 : 0.0, out, ldo));
    FOSB_CUDA(cudaStreamSynchronize(s));
    return FOSB_OK;
  }
  const int64_t N1 = m1->d.ne, N2 = m2->d.ne;
  FOSB_CUDA(a2.alloc(elem * nd3 * N2));
  FOSB_CUDA(cudaMemsetAsync(a2.p, 0, elem * nd3 * N2, s));
  FOSB_CUDA(launch_farfield_matrix(m2->d, k, ddirs.as<double>(), n_dir, c64, a2.p, s));
  // T = X op(A2) (N1 x 3 n_dir), M = A1 T
  FOSB_CUDA(t.alloc(elem * N1 * nd3));
  FOSB_CUDA(G(OP_N, pseudo ? OP_T : OP_C, N1, nd3, N2, 1.0, X, ldx, a2.p, N2, 0.0, t.p, nd3));
  if (!hermitian_mirror) {
    FOSB_CUDA(G(OP_N, OP_N, nd3, nd3, N1, weight, a1.p, N1, t.p, nd3, accumulate ? 1.0 : 0.0, out, ldo));
  } else {
    // out = beta out + w (M + op(M)), op = H (covariance) or T (pseudo-covariance)
    FOSB_CUDA(mm.alloc(elem * nd3 * nd3));
    FOSB_CUDA(G(OP_N, OP_N, nd3, nd3, N1, 1.0, a1.p, N1, t.p, nd3, 0.0, mm.p, nd3));
    FOSB_CUDA(add_mirrored(mm.p, nd3, nd3, pseudo ? OP_T : OP_C, weight, accumulate != 0, c64, out, ldo, s));
  }
  FOSB_CUDA(cudaStreamSynchronize(s));
  return FOSB_OK;
}

fosb_status fosb_debug_set_wait_limit(int64_t polls) {
  FOSB_CUDA(set_wait_limit_panels(polls));
  FOSB_CUDA(set_wait_limit_sweeps(polls));
  return FOSB_OK;
}

fosb_status fosb_rcs_monostatic(fosb_mesh mesh, fosb_lu lu, double k, const fosb_quad_opts* opts, const double* inc,
                                int64_t n_inc, const void* U, int64_t ldu, const double* weights, int db, double* sigma,
                                double* grad, void* stream) {
  if (!mesh || !inc || !U || n_inc <= 0 || ldu < n_inc) return fail(FOSB_ERR_INVALID_ARG, "fosb_rcs_monostatic: bad arguments");
  if (!(k > 0)) return fail(FOSB_ERR_INVALID_ARG, "fosb_rcs_monostatic: k must be > 0");
  if (grad && (!lu || !weights)) return fail(FOSB_ERR_INVALID_ARG, "fosb_rcs_monostatic: gradient needs lu and weights");
  if (db != 0 && db != 1) return fail(FOSB_ERR_INVALID_ARG, "fosb_rcs_monostatic: db must be 0 or 1");
  if (lu && (lu->prec == FOSB_FP32 || lu->n != mesh->d.ne))
    return fail(FOSB_ERR_INVALID_ARG, "fosb_rcs_monostatic: lu must be an FP64 or MIXED factorisation of this mesh");
  const int nss = opts && opts->n_ss > 0 ? opts->n_ss : 5;
  if (nss > 12) return fail(FOSB_ERR_INVALID_ARG, "fosb_rcs_monostatic: n_ss must be in 1..12");
  FOSB_TRY(ensure_rules(nss));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const DevMesh& d = mesh->d;
  const int64_t N = d.ne, n = n_inc, nd3 = 3 * n_inc;
  // observation directions of the monostatic set: xh_i = -d_i
  std::vector<double> xh(3 * n);
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < 3; ++c) xh[3 * i + c] = -inc[9 * i + c];
  Scratch dxh(s), A(s), FA(s);
  FOSB_CUDA(dxh.alloc(sizeof(double) * 3 * n));
  FOSB_CUDA(cudaMemcpyAsync(dxh.p, xh.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
  FOSB_CUDA(A.alloc(16 * nd3 * N));
  FOSB_CUDA(cudaMemsetAsync(A.p, 0, 16 * nd3 * N, s));
  FOSB_CUDA(launch_farfield_matrix(d, k, dxh.as<double>(), n, false, A.p, s));
  FOSB_CUDA(FA.alloc(16 * nd3 * n));
  FOSB_CUDA(gemm_c128_ff(OP_N, OP_N, nd3, n, N, 1.0, 0.0, A.p, N, U, ldu, 0.0, FA.p, n, s));
  std::vector<double> fa(2 * nd3 * n);
  FOSB_CUDA(cudaMemcpyAsync(fa.data(), FA.p, 16 * nd3 * n, cudaMemcpyDeviceToHost, s));
  FOSB_CUDA(cudaStreamSynchronize(s));
  // F_i = (A u_i) at xh_i: rows 3i..3i+2 of column i;  sigma_i = |F_i|^2 / (4 pi)
  std::vector<double> sig(n), Fr(3 * n), Fi(3 * n);
  for (int64_t i = 0; i < n; ++i) {
    double s2 = 0;
    for (int c = 0; c < 3; ++c) {
      Fr[3 * i + c] = fa[2 * ((3 * i + c) * n + i)];
      Fi[3 * i + c] = fa[2 * ((3 * i + c) * n + i) + 1];
      s2 += Fr[3 * i + c] * Fr[3 * i + c] + Fi[3 * i + c] * Fi[3 * i + c];
    }
    sig[i] = s2 / (4.0 * M_PI);
  }
  if (sigma) {
    for (int64_t i = 0; i < n; ++i) sigma[i] = db ? 10.0 * std::log10(sig[i]) : sig[i];
  }
  if (!grad) return FOSB_OK;
  // weights are dL/dsigma_i, or dL/dRCS_dB_i with db = 1: dRCS_dB/dsigma = 10 / (sigma ln 10)
  std::vector<double> w(n);
  for (int64_t i = 0; i < n; ++i) w[i] = db ? weights[i] * 10.0 / (sig[i] * std::log(10.0)) : weights[i];
  // Adjoint: dsigma_i = (2/(4 pi)) Re[conj(F_i).(dA_i u_i + A_i du_i)], du_i = Z^{-1}(db_i - dZ u_i);
  // with c_i = w_i (2/(4 pi)) conj(F_i) and lambda_i = Z^{-1} A_i^T c_i (Z^T = Z):
  //   sum_i w_i dsigma_i = Re[sum_i c_i.dA_i u_i + lambda_i^T db_i - lambda_i^T dZ u_i].
  std::vector<double> Cm(2 * nd3 * n, 0.0), pw(11 * 2 * n);
  for (int64_t i = 0; i < n; ++i) {
    double sc = w[i] * 2.0 / (4.0 * M_PI);
    double cr[3], ci[3];
    for (int c = 0; c < 3; ++c) {
      cr[c] = sc * Fr[3 * i + c];
      ci[c] = -sc * Fi[3 * i + c];
      Cm[2 * ((3 * i + c) * n + i)] = cr[c];
      Cm[2 * ((3 * i + c) * n + i) + 1] = ci[c];
    }
    // b-part: d_i, pi = p_i, alpha = -1 (weights lambda); A-part: -xh_i = d_i,
    // pi = (I - xh xh^T) c_i, alpha = -ik (weights U)
    double* pb = &pw[11 * i];
    double* pa = &pw[11 * (n + i)];
    const double* row = inc + 9 * i;
    for (int c = 0; c < 3; ++c) {
      pb[c] = row[c];
      pb[3 + c] = row[3 + c];
      pb[6 + c] = row[6 + c];
      pa[c] = row[c];
    }
    pb[9] = -1.0;
    pb[10] = 0.0;
    double xr = xh[3 * i] * cr[0] + xh[3 * i + 1] * cr[1] + xh[3 * i + 2] * cr[2];
    double xi = xh[3 * i] * ci[0] + xh[3 * i + 1] * ci[1] + xh[3 * i + 2] * ci[2];
    for (int c = 0; c < 3; ++c) {
      pa[3 + c] = cr[c] - xh[3 * i + c] * xr;
      pa[6 + c] = ci[c] - xh[3 * i + c] * xi;
    }
    pa[9] = 0.0;
    pa[10] = -k;
  }
  Scratch dC(s), lam(s), dpw(s);
  FOSB_CUDA(dC.alloc(16 * nd3 * n));
  FOSB_CUDA(cudaMemcpyAsync(dC.p, Cm.data(), 16 * nd3 * n, cudaMemcpyHostToDevice, s));
  FOSB_CUDA(lam.alloc(16 * N * n));
  FOSB_CUDA(gemm_c128_ff(OP_T, OP_N, N, n, nd3, 1.0, 0.0, A.p, N, dC.p, n, 0.0, lam.p, n, s));
  FOSB_TRY(solve_internal(lu, lam.p, n, n, lam.p, n, nullptr, nullptr, s));
  FOSB_CUDA(dpw.alloc(sizeof(double) * 11 * 2 * n));
  FOSB_CUDA(cudaMemcpyAsync(dpw.p, pw.data(), sizeof(double) * 11 * 2 * n, cudaMemcpyHostToDevice, s));
  FOSB_CUDA(cudaMemsetAsync(grad, 0, sizeof(double) * 3 * d.nv, s));
  const double* Uc = static_cast<const double*>(U);
  Scratch ucopy(s);
  if (ldu != n) {  // the pair kernel reads lambda and U with one leading dimension
    FOSB_CUDA(ucopy.alloc(16 * N * n));
    FOSB_CUDA(copy_matrix(U, N, n, ldu, ucopy.p, n, 16, s));
    Uc = ucopy.as<double>();
  }
  FOSB_CUDA(launch_adjoint_pairs(d, k, nss, lam.as<double>(), Uc, n, n, grad, s));
  FOSB_CUDA(launch_adjoint_planewave(d, k, n, dpw.as<double>(), lam.as<double>(), n, grad, s));
  FOSB_CUDA(launch_adjoint_planewave(d, k, n, dpw.as<double>() + 11 * n, static_cast<const double*>(U), ldu, grad, s));
  FOSB_CUDA(cudaStreamSynchronize(s));
  return FOSB_OK;
}

}  // extern "C"
