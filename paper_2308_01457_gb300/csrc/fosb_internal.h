// Internal declarations of the FOSB library (host + device).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fosb.h"

namespace fosb {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
fosb_status fail(fosb_status code, const std::string& msg);
fosb_status cuda_fail(cudaError_t e, const char* where);

#define FOSB_CUDA(call)                                       \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return fosb::cuda_fail(e_, #call); \
  } while (0)

// Count of kernels this library has launched (diagnostics: fosb_kernel_launches).
void note_launches(uint64_t n);
inline cudaError_t launched(uint64_t n = 1) {
  note_launches(n);
  return cudaGetLastError();
}

// Kernel-family timing (fosb_profile_enable): RAII scope recording CUDA events around a
// launch on its stream, with the launch's algorithmic work.
bool profiling();
class ProfScope {
 public:
  ProfScope(const char* family, cudaStream_t s, double work);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  const char* fam_;
  cudaStream_t s_;
  double work_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
  bool active_ = false;
};

// Stream-ordered scratch buffer released at scope exit.
struct Scratch {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  explicit Scratch(cudaStream_t st) : s(st) {}
  cudaError_t alloc(size_t bytes) { return cudaMallocAsync(&p, bytes > 16 ? bytes : size_t(16), s); }
  ~Scratch() {
    if (p) cudaFreeAsync(p, s);
  }
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

#define FOSB_TRY(call)                    \
  do {                                    \
    fosb_status s_ = (call);              \
    if (s_ != FOSB_OK) return s_;         \
  } while (0)

// ---------------------------------------------------------------- mesh
// Touching triangle pair in Sauter-Schwab orientation: x triangle t1 with its vertex
// order p[3], y triangle t2 with q[3]; kind 1 = vertex, 2 = edge, 3 = identical.
struct TouchPair {
  int32_t t1, t2, kind, pad;
  int32_t p[3], q[3];
};

// Per-triangle record (device, structure of arrays).  Local edge i is opposite local
// vertex i.
struct DevMesh {
  int64_t nv = 0, nt = 0, ne = 0, ntouch = 0;
  double* verts = nullptr;      // nv x 3
  double* vnormals = nullptr;   // nv x 3
  int32_t* tris = nullptr;      // nt x 3
  int32_t* tri_edge = nullptr;  // nt x 3
  double* tri_coef = nullptr;   // nt x 3: s l / (2A)
  double* tri_div = nullptr;    // nt x 3: s l / A
  double* tri_area = nullptr;   // nt
  double* tri_normal = nullptr; // nt x 3 unit normals
  double* tri_qp = nullptr;     // nt x 18: the 6 quadrature points (x, y, z)
  TouchPair* touch = nullptr;   // ntouch
  int32_t* ell_cols = nullptr;  // ne x 4: vertices a, b of edge m, opposite vertex in T+, in T-
  // Float-float copies (hi, lo) for the FP32-pipe assembly, field-major: tri_ff[f * nt + t].
  // Fields: 0..35 quadrature points minus vertex 0 ((q*3 + c)*2 + {hi,lo}); 36..41 vertex 0;
  // 42..47 vertex 1 - vertex 0; 48..53 vertex 2 - vertex 0; 54..59 s_i l_i.
  float* tri_ff = nullptr;
  double diameter = 0.0;        // bounding-box diagonal
};
constexpr int kTriFF = 60;

}  // namespace fosb

struct fosb_mesh_s {
  int device = 0;
  std::vector<double> verts, vnormals;
  std::vector<int32_t> tris;
  std::vector<int32_t> edges;      // ne x 2
  std::vector<int32_t> edge_tris;  // ne x 2 (T+, T-)
  std::vector<int32_t> tri_edge;   // nt x 3
  std::vector<double> tri_sign;    // nt x 3
  std::vector<fosb::TouchPair> touch;
  fosb::DevMesh d;
};

struct fosb_lu_s {
  int device = 0;
  int prec = 0;
  int64_t n = 0;
  void* lu = nullptr;          // n x n factors (complex128 for FP64, complex64 otherwise), row-major ld = n
  int32_t* ipiv = nullptr;     // n pivots (row swapped with i at step i), device
  const void* zref = nullptr;  // MIXED: non-owning complex128 Z for residuals
  int64_t ldz = 0;
  void* zff = nullptr;         // MIXED: (hi, lo) float split of Z (n x n float4) for the residual GEMMs
  void* dinv = nullptr;        // complex64 factors: inverses of the 64 x 64 diagonal blocks of L, then of U
  void* zdig = nullptr;        // MIXED: bf16 digit tiles of Z for the tensor-core residual GEMMs (oz_gemm)
  int* zex = nullptr;          // MIXED: their row exponents
  double znorm_inf = 0.0;      // ||Z||_inf (FP64)
  int* d_status = nullptr;     // device status word
};

namespace fosb {

// Quadrature rules in the device constant memory of every kernel family, for n_ss points
// per Sauter-Schwab coordinate (uploaded once per device and n_ss).
fosb_status ensure_rules_for(int nss);

// ---------------------------------------------------------------- quadrature rules
struct Rules {
  double bary[6][3];
  double w[6];
  int nss;
  double glx[16], glw[16];
};
Rules make_rules(int nss);

// ---------------------------------------------------------------- kernels (launchers)
// Assembly
cudaError_t launch_assemble_regular(const DevMesh& m, double k, int arith, void* Z, int64_t ldz, cudaStream_t s);
cudaError_t launch_assemble_singular(const DevMesh& m, double k, int nss, bool fp32_out, void* Z, int64_t ldz,
                                     cudaStream_t s);
cudaError_t launch_rhs(const DevMesh& m, double k, const double* d_inc, int64_t n_inc, bool fp32_out, void* b,
                       int64_t ldb, cudaStream_t s);
void upload_rules(const Rules& r);
void upload_rules_adjoint(const Rules& r);
void upload_rules_ff(const Rules& r);
void upload_rules_pmchwt(const Rules& r);
double ff_max_phase();  // k * mesh diameter must stay below this for the float-float kernel
// Adjoint shape gradients (see adjoint.cu): grad (V x 3) += -grad Re sum_i lam_i^T Z u_i, and
// += grad Re J_P for plane-wave moments with per-column parameters d_pw (ncols x 11:
// d(3), Re pi(3), Im pi(3), alpha (re, im)) and edge weights wgt (N x ncols, ldw).
cudaError_t launch_adjoint_pairs(const DevMesh& m, double k, int nss, const double* lam, const double* U, int64_t ld,
                                 int64_t nrhs, double* grad, cudaStream_t s);
cudaError_t launch_adjoint_planewave(const DevMesh& m, double k, int64_t ncols, const double* d_pw, const double* wgt,
                                     int64_t ldw, double* grad, cudaStream_t s);
cudaError_t launch_efie_regular_ff(const DevMesh& m, double k, double* Z, int64_t ldz, cudaStream_t s);
// PMCHWT regular pairs in float-float for one wavenumber: EFIO blocks into ZT, MFIO blocks into ZK.
cudaError_t launch_pmchwt_regular_ff(const DevMesh& m, double k, double* ZT, double* ZK, int64_t ldz, cudaStream_t s);

// Far field
cudaError_t launch_farfield_matrix(const DevMesh& m, double k, const double* d_dirs, int64_t n_dir, bool fp32,
                                   void* A, cudaStream_t s);

// Shape-derivative RHS in ELL form (N x 4 complex128 values on the columns ell_cols),
// its dense expansion (N x V), and W = B1 K12 (N1 x V2) with K evaluated on the fly.
cudaError_t launch_sd_rhs(const DevMesh& m, double k, const void* u, bool u_fp32, double* B_ell, cudaStream_t s);
// Low-rank kernel factor (lowrank.cu): pivoted Cholesky of the covariance kernel matrix over
// n device points d_x (n x 3), R rows = factor columns; and W (N x r) = B R^T for one mesh.
fosb_status pivoted_cholesky_kernel(const double* d_x, int64_t n, const fosb_cov_kernel& ker, double tol,
                                    int64_t max_rank, double* R, int64_t ldr, int64_t* rank, double* trace_err,
                                    cudaStream_t s);
cudaError_t launch_br_product(const DevMesh& m, const double* B_ell, const double* R, int64_t ldr, int64_t r, bool fp32,
                              void* W, int64_t ldw, cudaStream_t s);
cudaError_t launch_ell_to_dense(const DevMesh& m, const double* B_ell, bool conj_out, bool fp32, void* B, int64_t ldb,
                                cudaStream_t s);
cudaError_t launch_bk_product(const DevMesh& m1, const double* B1_ell, const DevMesh& m2,
                              const fosb_cov_kernel& ker, bool fp32, void* W, int64_t ldw, cudaStream_t s);

// Dense complex linear algebra (row-major).  T = double or float.
enum Op { OP_N = 0, OP_T = 1, OP_C = 2 };
template <typename T>
cudaError_t gemm(int opA, int opB, int64_t M, int64_t N, int64_t K, double alpha_re, double alpha_im, const void* A,
                 int64_t lda, const void* B, int64_t ldb, double beta, void* C, int64_t ldc, cudaStream_t s);
// C (M x N) -= A (M x K) B (K x N), complex64 row-major, tcgen05 tensor cores with 3xTF32;
// a bounded mbarrier wait that gives up sets *status = FOSB_ERR_TIMEOUT.  family names the
// timing record (fosb_profile_read): the LU's K = 64 updates ("lu_update64") and the solve
// sweeps ("trsm_update") are timed apart from the K = kLuBlock trailing updates ("lu_update")
cudaError_t cgemm_update_tc(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B, int64_t ldb,
                            void* C, int64_t ldc, int* status, cudaStream_t s, const char* family);
// Column block of the complex64 LU (four 64-column panels per block, one trailing update
// with K = kLuBlock per block).
constexpr int kLuBlock = 256;
// The same update for K <= kLuBlock with A and B split once into bulk-copy images
// (tc_update.cu): workspaces of update_split_a_bytes(M) and update_split_b_bytes(N) bytes.
size_t update_split_a_bytes(int64_t M);
size_t update_split_b_bytes(int64_t N);
cudaError_t cgemm_update_tc_split(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B,
                                  int64_t ldb, void* C, int64_t ldc, int* status, void* ws_a, void* ws_b,
                                  cudaStream_t s);
// complex128 GEMM computed in float-float on the FP32 pipe (FP64-class accuracy).  A_split,
// if given, is split_ff of A as stored (same shape, leading dimension lda).
cudaError_t gemm_c128_ff(int opA, int opB, int64_t M, int64_t N, int64_t K, double alpha_re, double alpha_im,
                         const void* A, int64_t lda, const void* B, int64_t ldb, double beta, void* C, int64_t ldc,
                         cudaStream_t s, const void* A_split = nullptr);
// FP64-class complex GEMM on the bf16 tensor cores by exact digit splitting (oz_gemm.cu):
// oz_prepare_a writes the digit tiles (oz_a_bytes(M, K) bytes) and row exponents (M ints)
// of the complex128 A (M x K, lda); oz_gemm then computes C <- beta C + alpha A B for a
// complex128 B (K x N, ldb); a bounded wait that gives up sets *status.
size_t oz_a_bytes(int64_t M, int64_t K);
cudaError_t oz_prepare_a(const void* A, int64_t M, int64_t K, int64_t lda, void* digits, int* ex, cudaStream_t s);
cudaError_t oz_gemm(int64_t M, int64_t N, int64_t K, double alpha_re, double alpha_im, const void* a_digits,
                    const int* a_ex, const void* B, int64_t ldb, double beta, void* C, int64_t ldc, int* status,
                    cudaStream_t s);
// dst (rows x cols float4, ldd) = (hi, lo) float split of the complex128 src
cudaError_t split_ff(const void* src, int64_t rows, int64_t cols, int64_t lds, void* dst, int64_t ldd,
                     cudaStream_t s);
template <typename T>
fosb_status getrf(void* A, int64_t n, int64_t lda, int32_t* ipiv, int* d_status, cudaStream_t s);
size_t getrf_scratch_bytes(int64_t max_ctas, bool c128);
// Tournament-pivoting factorisation of one complex64 panel (m x jb at Ap, jb <= 64, m >= jb)
// with scratch of tslu_scratch_bytes(n_max) bytes (n_max >= m); writes ipiv[0..jb) as
// absolute rows (row_base + panel row) and permutes the panel's own rows.
size_t tslu_scratch_bytes(int64_t n_max);
cudaError_t tslu_panel(void* Ap, int64_t m, int jb, int64_t lda, int32_t* ipiv, int64_t row_base, void* scratch,
                       int64_t n_max, int* d_status, cudaStream_t s);
// X (jb x ncols, leading dimension ldx) := L^{-1} X, L the unit lower jb x jb block at D
// (leading dimension ldd), complex64, jb <= 64: a thread per column (tslu.cu).
cudaError_t tri_lower_unit_cols(const void* D, int64_t ldd, int jb, void* X, int64_t ldx, int64_t ncols,
                                cudaStream_t s);
// The row interchanges of the last tslu_panel on the same scratch, applied to the columns
// of the n-column matrix A outside the panel's columns [j0, j0 + jb) (rows from j0 on).
cudaError_t tslu_swap(void* A, int64_t n, int64_t lda, int64_t j0, int jb, const void* scratch, cudaStream_t s);
template <typename T>
fosb_status getrf_external_scratch(void* A, int64_t n, int64_t lda, int32_t* ipiv, int* d_status, void* scratch,
                                   int64_t max_ctas, cudaStream_t s);
template <typename T>
cudaError_t getrs(const void* LU, int64_t n, int64_t ldlu, const int32_t* ipiv, void* X, int64_t nrhs, int64_t ldx,
                  cudaStream_t s, int* status = nullptr, const void* dinv = nullptr);
// One whole triangular sweep with complex64 factors (unit lower if upper == 0, else upper
// with its diagonal) for nrhs <= kTrsvStreamMaxRhs right-hand sides stored dense
// (n x nrhs), given the inverses of the diagonal blocks (tri_block_inverses_c64); scratch
// holds trsv_stream_scratch_ints(n, nrhs) ints; a bounded wait that gives up sets *status.
constexpr int64_t kTrsvStreamMaxRhs = 1024;
size_t trsv_stream_scratch_ints(int64_t n, int64_t nrhs);
size_t tri_block_inverses_bytes(int64_t n);
cudaError_t tri_block_inverses_c64(const void* LU, int64_t n, int64_t ld, void* Dinv, cudaStream_t s);
cudaError_t trsv_stream_c64(const void* LU, int64_t n, int64_t ld, const void* Dinv, void* X, int64_t nrhs, int upper,
                            int* scratch, int* status, cudaStream_t s);
cudaError_t convert_c128_to_c64(const void* src, int64_t rows, int64_t cols, int64_t lds, void* dst, int64_t ldd,
                                cudaStream_t s);
cudaError_t convert_c64_to_c128(const void* src, int64_t rows, int64_t cols, int64_t lds, void* dst, int64_t ldd,
                                cudaStream_t s);
cudaError_t copy_matrix(const void* src, int64_t rows, int64_t cols, int64_t lds, void* dst, int64_t ldd, size_t elem,
                        cudaStream_t s);
cudaError_t axpy_c64_into_c128(const void* d, int64_t rows, int64_t cols, int64_t ldd, void* x, int64_t ldx,
                               cudaStream_t s);
// out = (accumulate ? out : 0) + w (M + op(M)) for a square n x n matrix M (op = OP_T or OP_C)
cudaError_t add_mirrored(const void* M, int64_t n, int64_t ldm, int op, double w, bool accumulate, bool c64, void* out,
                         int64_t ldo, cudaStream_t s);
// complex128 vectors (strides in elements): y = alpha x, y += alpha x (krylov.cu)
cudaError_t zscal_copy(int64_t n, double ar, double ai, const void* x, int64_t incx, void* y, int64_t incy,
                       cudaStream_t s);
cudaError_t zaxpy(int64_t n, double ar, double ai, const void* x, int64_t incx, void* y, int64_t incy, cudaStream_t s);
// Poll limits of the bounded device waits on the current device (polls <= 0: default):
// panel grid barriers (linalg.cu) and streaming-sweep flags (trsv_stream.cu).
cudaError_t set_wait_limit_panels(long long polls);
cudaError_t set_wait_limit_sweeps(long long polls);
// Largest n that the external-scratch panel path can factor with at most max_ctas CTAs on
// the current device (co-resident panel CTAs x rows a CTA can hold).
fosb_status getrf_external_max_n(int64_t max_ctas, int64_t* max_n);
// row-wise inf-norm reductions: out[0] = max_i sum_j |Re|+|Im| (matrix), or max |.|
cudaError_t norm_inf_c128(const void* A, int64_t rows, int64_t cols, int64_t lda, double* d_out, cudaStream_t s);
cudaError_t absmax_c128(const void* A, int64_t rows, int64_t cols, int64_t lda, double* d_out, cudaStream_t s);

}  // namespace fosb
