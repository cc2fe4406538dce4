/*
 * fosb.h -- C ABI of the GB300 (sm_103a) FOSB / EFIE library.
 *
 * The library computes, on one GPU, the data-parallel hot path of the first-order
 * sparse boundary element method (FOSB) for a perfectly conducting scatterer
 * (Escapil-Inchauspe & Jerez-Hanckes, "Shape UQ for EM wave scattering via FOSB
 * approximation", arXiv:2308.01457):
 *
 *   - Galerkin assembly of the EFIE  <T_k j, phi>_x = <gamma_D E_inc, phi>_x
 *     with lowest-order RWG elements (Section II-B eq. boundary_operators, Section
 *     II-C eq. pec, Section IV-A), Z_L u_L = b_L (eq. linear_system);
 *   - LU factorisation and solves (FP64, or FP32 factors with FP64 iterative
 *     refinement) giving the nominal current u_L;
 *   - the first-order shape-derivative covariance: the tensor system
 *     (Z_l1 (x) conj Z_l2) Sigma_{l1,l2} = C_{l1,l2} (eq. linear_system2, eq.
 *     CTsubsystem) with C = E[g g^H] built from the PEC shape-derivative right-hand
 *     side g of Section III (eq. secondPEC);
 *   - far-field and RCS moments (Section II-C, the far-field expansion and eq. RCS),
 *     combined over the combination-technique index sets Lambda_+/- (Section IV-B);
 *   - for a dielectric scatterer, the PMCHWT system of Section II-C (eq. pmchwt) and its
 *     far field (fosb_assemble_pmchwt, fosb_farfield_pmchwt).
 *
 * Conventions (every call):
 *   - Complex arrays are interleaved (re, im): complex128 = 2 doubles, complex64 =
 *     2 floats.  Matrices are ROW-MAJOR with an explicit leading dimension (in
 *     elements).
 *   - Pointers documented "device" are caller-owned device memory (the library never
 *     frees them); "host" pointers are read during the call only.  Handles
 *     (fosb_mesh, fosb_lu) own library-allocated device memory released by their
 *     destroy call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Device work is enqueued on it; calls return after enqueueing unless stated.
 *   - Argument and mesh errors are detected on the host and returned before any
 *     work is enqueued.  CUDA launch errors return FOSB_ERR_CUDA.  A failed call
 *     leaves its outputs unspecified, except FOSB_ERR_NOT_CONVERGED, where the best
 *     iterate is written.  fosb_last_error() gives a thread-local message.
 *
 * RWG numbering (shared contract with any checker): edges are the unordered vertex
 * pairs (a < b) in lexicographic order; local edge i of a triangle is opposite its
 * local vertex i; the basis function of edge m is
 *     f_m(x) = +l_m/(2 A_+) (x - p_+) on T_+,   f_m(x) = -l_m/(2 A_-) (x - p_-) on T_-,
 * where T_+ is the triangle whose counter-clockwise order runs a -> b, and p_+/- are
 * the opposite vertices (Section IV: div-conforming lowest-order elements).
 */
#ifndef FOSB_H
#define FOSB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int fosb_status;
enum {
  FOSB_OK = 0,
  FOSB_ERR_INVALID_ARG = 1,   /* bad pointer, size, option or leading dimension */
  FOSB_ERR_MESH = 2,          /* non-manifold, degenerate or inconsistently oriented mesh */
  FOSB_ERR_SINGULAR = 3,      /* exactly zero pivot in the LU factorisation */
  FOSB_ERR_NOT_CONVERGED = 4, /* iterative refinement stalled; best iterate written */
  FOSB_ERR_OOM = 5,           /* device allocation failed */
  FOSB_ERR_CUDA = 6,          /* CUDA runtime / launch error */
  FOSB_ERR_TIMEOUT = 7        /* a bounded device-side wait gave up (status word set) */
};

/* Arithmetic of a call.
 *   FOSB_FP64  : all arithmetic in FP64; Z and solutions complex128.
 *   FOSB_MIXED : FP64-accurate Z (complex128), complex64 LU factors, FP64 residuals
 *                and iterative refinement to FP64 accuracy; outputs complex128.
 *   FOSB_FP32  : complex64 Z, LU and solutions, no refinement (about 1e-4 relative). */
typedef enum { FOSB_FP64 = 0, FOSB_MIXED = 1, FOSB_FP32 = 2 } fosb_precision;

/* Regular-pair assembly arithmetic (singular pairs are always FP64):
 *   FOSB_ASM_FP64  : FP64 everywhere;
 *   FOSB_ASM_FF    : float-float (unevaluated sums of two floats, ~48-bit significand)
 *                    on the FP32 pipe -- FP64-class accuracy at FP32 throughput;
 *   FOSB_ASM_FP32  : plain FP32 (the 1e-4 path). */
typedef enum { FOSB_ASM_FP64 = 0, FOSB_ASM_FF = 1, FOSB_ASM_FP32 = 2 } fosb_asm_arith;

typedef struct {
  int n_ss;        /* Gauss-Legendre points per coordinate of the Sauter-Schwab 4-cube (1..12), default 5 */
  int arith;       /* fosb_asm_arith for the regular pairs, default FOSB_ASM_FP64 */
} fosb_quad_opts;

typedef struct {
  int max_iters;     /* iterative-refinement steps (default 10) */
  double tol;        /* stop when ||b - Z x||_inf / (||Z||_inf ||x||_inf + ||b||_inf) <= tol per column;
                        tol <= 0 selects the default max(64, 8 sqrt(n)) * 2^-52.  Refinement also stops
                        when a step gains less than a factor 2 below 1e-13 (rounding floor reached) */
  int solver;        /* FOSB_REFINE_AUTO (0): refinement, then GMRES-IR for the columns it left above tol;
                        FOSB_REFINE_IR (1): refinement only; FOSB_REFINE_GMRES (2): GMRES-IR from the start */
} fosb_refine_opts;

/* GMRES-based iterative refinement (the Krylov part of the paper's solver stack, Section IV):
 * each step solves the correction equation Z d = r (r = b - Z x in FP64-class arithmetic) by
 * GMRES(50) on M^-1 Z d = M^-1 r, preconditioned by the complex64 factors M, with FP64-class
 * matrix-vector products and FP64 Arnoldi (two-pass classical Gram-Schmidt); it converges
 * where plain refinement stalls because kappa(Z) u_32 is not small (Carson and Higham,
 * SIAM J. Sci. Comput. 40, 2018). */
enum { FOSB_REFINE_AUTO = 0, FOSB_REFINE_IR = 1, FOSB_REFINE_GMRES = 2 };

typedef struct {
  int iters;             /* refinement steps taken plus GMRES iterations (0 for FOSB_FP64 / FOSB_FP32) */
  double backward_error; /* final normwise relative backward error (max over right-hand sides) */
} fosb_solve_stats;

typedef enum { FOSB_COV_GAUSS = 0, FOSB_COV_MATERN32 = 1 } fosb_cov_kind;
typedef struct {
  int kind;      /* fosb_cov_kind: sigma^2 exp(-r^2/(2 l^2)) or sigma^2 (1 + sqrt3 r/l) exp(-sqrt3 r/l) */
  double sigma;  /* pointwise standard deviation of the normal velocity v_n */
  double ell;    /* correlation length l (chordal distance r between mesh vertices) */
} fosb_cov_kernel;

typedef struct fosb_mesh_s* fosb_mesh;
typedef struct fosb_lu_s* fosb_lu;

/* Thread-local description of the last error (library-owned, valid until the next call). */
const char* fosb_last_error(void);

/* Library version string. */
const char* fosb_version(void);

/* Number of CUDA kernels this library has launched in this process (all devices);
 * diagnostics for launch accounting. */
uint64_t fosb_kernel_launches(void);

/* Kernel-family timing (diagnostics).  While enabled, the library brackets every launch of
 * the families below with CUDA events recorded on the launching stream and notes the
 * launch's algorithmic work.  fosb_profile_read waits for the recorded events and returns
 * (then clears) the family's total device time in ms, launch count and work:
 *   "lu_update"      tcgen05 complex64 trailing update, work = 8 M N K flops
 *   "lu_panel"       cooperative panel factorisation, work = 8 m jb^2 / 2 flops
 *   "asm_regular"    regular-pair assembly, work = point pairs (36 per triangle pair)
 *   "asm_singular"   Sauter-Schwab pairs, work = point pairs
 *   "gemm_ff"        float-float complex128 GEMM, work = 8 M N K flops
 * Any pointer may be NULL. */
fosb_status fosb_profile_enable(int on);
fosb_status fosb_profile_read(const char* family, double* total_ms, int64_t* launches, double* work);

/* ---- A1: mesh tables ------------------------------------------------------------
 * Builds the RWG tables of a closed, orientable, manifold triangulation (Section IV,
 * meshes Gamma_{h_l} of planar triangles) and uploads them to the current device.
 *   verts    : host, nv x 3 float64 vertex coordinates
 *   tris     : host, nt x 3 int32, counter-clockwise seen from outside
 *   vnormals : host, nv x 3 unit outward vertex normals n_p used for the normal
 *              perturbation v_n (Section III); NULL -> area-weighted normals
 *   out      : receives the handle (library-owned; free with fosb_mesh_destroy)
 * Errors: FOSB_ERR_INVALID_ARG (NULL/size), FOSB_ERR_MESH (index out of range,
 * degenerate triangle, edge not shared by exactly two oppositely oriented triangles,
 * non-finite coordinate), FOSB_ERR_OOM. */
fosb_status fosb_mesh_create(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                             const double* vnormals, fosb_mesh* out);

/* Sizes of a mesh: vertices, triangles, RWG edges (= unknowns N), touching triangle
 * pairs (unordered, including identical pairs).  Any output pointer may be NULL. */
fosb_status fosb_mesh_info(fosb_mesh mesh, int64_t* nv, int64_t* nt, int64_t* n_edges, int64_t* n_touching);

/* Host copy of the edge table: edges (N x 2 int32, a < b) and edge_tris (N x 2 int32,
 * T_+ then T_-).  Either pointer may be NULL. */
fosb_status fosb_mesh_edges(fosb_mesh mesh, int32_t* edges, int32_t* edge_tris);

fosb_status fosb_mesh_destroy(fosb_mesh mesh);

/* ---- A2-A4: EFIE assembly and plane-wave right-hand sides --------------------------
 * Z[m, n] = <T_k f_n, f_m>_x = -[ ik int int G f_m . f_n + 1/(ik) int int G div f_m div f_n ],
 * G = exp(ik|x-y|)/(4 pi |x-y|) (Section II-B), and
 * b[m, s] = <gamma_D E_inc_s, f_m>_x = -int E_inc_s . f_m, E_inc_s = p_s exp(ik d_s . x)
 * (Section V, eq. incidentNumexp).  Regular triangle pairs use the 6-point degree-4
 * triangle rule in x and y; pairs sharing a vertex, an edge, or identical use the
 * Sauter-Schwab regularised 4-cube rule with opts->n_ss Gauss points per coordinate.
 *   k       : wavenumber > 0
 *   opts    : quadrature options (NULL -> defaults)
 *   prec    : FOSB_FP64 / FOSB_MIXED write complex128 Z; FOSB_FP32 writes complex64 Z
 *   Z       : device, N x N, row-major, leading dimension ldz >= N; overwritten
 *   inc     : host, n_inc x 9 float64: d (3, unit), Re p (3), Im p (3); may be NULL if n_inc = 0
 *   b       : device, N x n_inc (leading dimension ldb >= n_inc), same complex type as Z; may be NULL
 * Enqueued on `stream` without synchronising it; `inc` may be reused once the call returns.
 * Errors: FOSB_ERR_INVALID_ARG. */
fosb_status fosb_assemble_efie(fosb_mesh mesh, double k, const fosb_quad_opts* opts, int prec, void* Z, int64_t ldz,
                               const double* inc, int64_t n_inc, void* b, int64_t ldb, void* stream);

/* ---- A5: LU factorisation -----------------------------------------------------------
 * P Z = L U.  complex128 factors (FOSB_FP64): partial pivoting (largest |Re| + |Im|, ties to
 * the lowest row).  complex64 factors (FOSB_MIXED, FOSB_FP32): 256-column blocks of 64-column
 * panels whose pivot rows a tournament chooses (leaves of 256 rows and a fan-in-4 tree, each
 * choosing by partial pivoting with the magnitudes compared on their top 15 mantissa bits).
 *   Z    : device, n x n row-major (complex128 for FP64/MIXED, complex64 for FP32);
 *          read, not modified.  For FOSB_MIXED the handle keeps a NON-owning reference
 *          to Z for the FP64 residuals: Z must stay alive and unchanged until
 *          fosb_lu_destroy.
 *   out  : receives a handle owning the factors and pivots (device memory).  A FOSB_MIXED
 *          handle also owns two residual copies of Z: a float-float split (16 n^2 bytes)
 *          and, for n >= 256, exact bf16 digit tiles (28 n^2 bytes) for the FP64-class
 *          tensor-core residuals of solves with 5 or more right-hand sides; and the
 *          inverses of its 64 x 64 diagonal blocks for the streaming triangular sweeps.
 * Synchronises `stream` at the end (the pivot search reports FOSB_ERR_SINGULAR).
 * Errors: FOSB_ERR_OOM when device memory runs out (nothing is leaked). */
fosb_status fosb_factor(const void* Z, int64_t n, int64_t ldz, int prec, fosb_lu* out, void* stream);

/* ---- A6: solves with iterative refinement -----------------------------------------
 * X = Z^{-1} B (op = 'N').  Z is complex symmetric for the EFIE, so Z^{-T} = Z^{-1}.
 *   B, X : device, n x nrhs row-major (ldb, ldx >= nrhs), complex128 for FP64/MIXED,
 *          complex64 for FP32.  X may alias B.
 *   ropt : refinement options (MIXED only; NULL -> defaults); stats may be NULL.
 * MIXED: x0 from the complex64 factors, then r = b - Z x in FP64, x += LU^{-1} r until
 * the backward error is below tol; synchronises `stream` once per step.  The residual
 * product is float-float for 1-4 right-hand sides and exact digit splitting on the bf16
 * tensor cores for more (n >= 256); both are accurate to a few units of 2^-52 of
 * |b| + |Z||x|.  Triangular sweeps of complex64 factors with up to 1024 right-hand sides
 * run as one persistent kernel per sweep.
 * Errors: FOSB_ERR_NOT_CONVERGED (best iterate written). */
fosb_status fosb_solve(fosb_lu lu, char op, const void* B, int64_t nrhs, int64_t ldb, void* X, int64_t ldx,
                       const fosb_refine_opts* ropt, fosb_solve_stats* stats, void* stream);

fosb_status fosb_lu_info(fosb_lu lu, int64_t* n, int* prec, double* znorm_inf);
fosb_status fosb_lu_destroy(fosb_lu lu);

/* ---- In-place LU that allocates no device memory -----------------------------------
 * The paper has no counterpart: this is a library-integration entry point.  For callers
 * that cannot call cudaMalloc/cudaFree while they use the library (hosts whose own
 * allocator owns all device memory, or that forbid allocation after start-up because it
 * can synchronise the device), it factors the caller's matrix in place, P A = L U with
 * classic partial pivoting (largest |Re| + |Im|, ties to the lowest row) by a cooperative
 * panel kernel in 64-column blocks, and allocates nothing: the panel kernel's scratch lives
 * in a 1 MiB static device array that every GPU loading the library holds until the
 * process exits.  For complex128 these are fosb_factor's pivots and kernels; for complex64
 * fosb_factor uses tournament pivoting in 256-column blocks, so the pivots and factors of
 * the two calls can differ while the solutions agree to rounding.
 *   A    : device, n x n row-major (lda >= n), complex128 (prec = FOSB_FP64) or complex64
 *          (prec = FOSB_FP32); overwritten by L (unit lower, below the diagonal) and U.
 *   ipiv : device, n int32: at step i row i was interchanged with row ipiv[i] (0-based).
 * Limits: n <= min(SM count, 256) x 2048 (the first panel's rows over the co-resident panel
 * CTAs, 2048 rows each): 311,296 on a 152-SM GB300; larger n -> FOSB_ERR_INVALID_ARG.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current.  Every call synchronises `stream` to read the status word, so
 * no call can be made inside a stream capture.  Calls share the array: calls that overlap
 * on the GPU race.  Errors: FOSB_ERR_SINGULAR, FOSB_ERR_TIMEOUT, FOSB_ERR_INVALID_ARG. */
fosb_status fosb_getrf_static(void* A, int64_t n, int64_t lda, int prec, int32_t* ipiv, void* stream);

/* ---- A7-A9: shape-derivative covariance of one combination-technique block --------
 * Sigma solves (Z_1 (x) conj Z_2) Sigma = C (eq. CTsubsystem), i.e. Z_1 Sigma Z_2^H = C,
 * with C = B_1 K_12 B_2^H = E[g_1 g_2^H]:
 *   B_l (N_l x V_l): g = B xi is the Galerkin right-hand side <g, f_m>_x of the PEC
 *   shape-derivative problem T_k dj' = grad_G[v_n E_n] x n - ik v_n gamma_T H
 *   (Section III) for v_n = sum_p xi_p psi_p (n_p . n_T), evaluated at the nominal
 *   current u_l of that level:  B_mp = -sum_n u_n int psi_p (n_p . n_T) [ik f_m . f_n
 *   + 1/(ik) div f_m div f_n];
 *   K_12[p, q] = kernel(|x_p^(1) - x_q^(2)|) between the vertices of the two meshes.
 * pseudo = 1 gives the pseudo-covariance Z_1 S Z_2^T = B_1 K_12 B_2^T instead.
 *   m1, m2   : meshes of levels l1 and l2 (may be the same handle)
 *   lu1, lu2 : factorisations of Z_l1, Z_l2 (same precision; MIXED refines both solves)
 *   u1, u2   : device, nominal currents (N_l, complex128 or complex64 per precision)
 *   Sigma    : device, N_1 x N_2 row-major (leading dimension lds), overwritten
 * The product is evaluated as Sigma = (Z_1^{-1} B_1 K_12)(Z_2^{-1} B_2)^H when V_2 <= V_1
 * (and symmetrically otherwise): the same Sigma with min(V_1, V_2) right-hand sides.
 * Synchronises `stream` (refinement).  Errors: FOSB_ERR_NOT_CONVERGED. */
fosb_status fosb_covariance(fosb_mesh m1, fosb_lu lu1, const void* u1, fosb_mesh m2, fosb_lu lu2, const void* u2,
                            double k, const fosb_cov_kernel* kernel, int pseudo, void* Sigma, int64_t lds,
                            const fosb_refine_opts* ropt, void* stream);

/* ---- A10-A11: far-field moments --------------------------------------------------
 * Far-field matrix A_l (3 n_dir x N_l): F(xh_d)_c = sum_n A[3d + c, n] u_n, from
 * E_sc = -E_k j and E_sc ~ exp(ik|x|)/(4 pi |x|) F (Section II-C):
 *     A[3d + c, n] = -ik [(I - xh xh^T) int f_n(y) exp(-ik xh . y) dy]_c  (6-point rule).
 * Mean mode (m2 == NULL): out (3 n_dir x ncols, leading dimension ldo) = weight * A_1 X,
 *   X device N_1 x ncols (ldx).
 * Covariance mode (m2 != NULL): out (3 n_dir x 3 n_dir, ldo) = weight * M,
 *   M = A_1 X A_2^H (pseudo = 0) or A_1 X A_2^T (pseudo = 1), X = Sigma (N_1 x N_2, ldx);
 *   hermitian_mirror = 1 adds M^H (resp. M^T): the Hermitian reduction of Section IV-B
 *   for an off-diagonal block (l1 != l2).
 * accumulate = 1 adds into out instead of overwriting (CT signed sum: weight = +1 on
 * Lambda_+, -1 on Lambda_-).  dirs: host n_dir x 3 unit vectors.  Complex128 (prec
 * FP64/MIXED) or complex64 (FP32) throughout. */
fosb_status fosb_farfield_moments(fosb_mesh m1, fosb_mesh m2, double k, const double* dirs, int64_t n_dir,
                                  const void* X, int64_t ldx, int64_t ncols, double weight, int hermitian_mirror,
                                  int pseudo, int prec, void* out, int64_t ldo, int accumulate, void* stream);

/* ---- Dielectric scatterer: the PMCHWT system (Section II-C eq. pmchwt) --------------
 * fosb_assemble_pmchwt: Galerkin matrix of A_0 + A^_1 (multitrace operators of eq.
 * BOmultitraceA, A_k = [[K_k, T_k], [-T_k, K_k]] and its eta-scaled form) for the exterior
 * Cauchy data (j, m) = (gamma_D^c E, gamma_N^c E) of the total field, tested with the
 * x-pairing against RWG functions:
 *     Z (2N x 2N) = [[K_0 + K_1, T_0 + eta T_1], [-T_0 - T_1/eta, K_0 + K_1]],
 *     T_k[m, n] = -[ik int int G f_m.f_n + 1/(ik) int int G div f_m div f_n]   (EFIO, as above),
 *     K_k[m, n] = -int int (x - y).(f_n(y) x f_m(x)) exp(ikr)(ikr - 1)/(4 pi r^3)  (MFIO
 *                 K_k = {gamma_D H_k}, Section II-B),
 * k = k0 outside, k1 = k0 sqrt(eps_r mu_r) inside, eta = sqrt(mu_r/eps_r) (eq.
 * relativeParameters).  The right-hand side is the tested incident Cauchy data,
 *     b[m, s] = -int E_inc_s . f_m,   b[N + m, s] = -int (d_s x p_s) exp(ik0 d_s.x) . f_m,
 * which with the incident field's Calderon identity is the printed system
 * (A_0 + A^_1) xi_sc = (I/2 - A^_1) xi_inc for xi_sc = (j, m) - xi_inc.
 * Regular pairs: the 6-point rule in x and y in FP64 or float-float (opts->arith; both
 * wavenumbers must keep k * mesh diameter below the float-float phase range, 48); touching
 * pairs: Sauter-Schwab in FP64 with opts->n_ss points per coordinate (identical pairs add
 * nothing to K_k on a flat triangle).
 *   eps_r, mu_r : relative permittivity and permeability (finite, > 0; lossless media)
 *   opts        : NULL (n_ss = 5, FP64) or n_ss with arith = FOSB_ASM_FP64 or FOSB_ASM_FF
 *   Z           : device, 2N x 2N complex128, leading dimension ldz >= 2N; overwritten
 *   inc         : host, n_inc x 9 as for fosb_assemble_efie (d, Re p, Im p)
 *   b           : device, 2N x n_inc complex128 (ldb >= n_inc) or NULL when n_inc = 0
 * Z is not complex symmetric; factor it with fosb_factor (FOSB_FP64 or FOSB_MIXED) and
 * solve with fosb_solve (op = 'N').  Enqueued on `stream` without synchronising it.
 * Errors: FOSB_ERR_INVALID_ARG. */
fosb_status fosb_assemble_pmchwt(fosb_mesh mesh, double k0, double eps_r, double mu_r, const fosb_quad_opts* opts,
                                 void* Z, int64_t ldz, const double* inc, int64_t n_inc, void* b, int64_t ldb,
                                 void* stream);

/* fosb_farfield_pmchwt: out (3 n_dir x ncols, ldo) = weight * A X (+ out if accumulate),
 * X (2N x ncols, ldx) exterior Cauchy data (j on rows 0..N-1, m on rows N..2N-1), with the
 * far field of E_sc = -E_k0 m - H_k0 j (Section II-C, E = E_inc + R(xi), R = (-H, -E)):
 *     F(xh) = -ik0 [xh x sum_n j_n v_n + (I - xh xh^T) sum_n m_n v_n],
 *     v_n = int f_n(y) exp(-ik0 xh.y) dy (6-point rule), row 3d + c = component c at xh_d.
 * dirs: host n_dir x 3 unit vectors.  complex128 throughout; synchronises `stream`.
 * Errors: FOSB_ERR_INVALID_ARG. */
fosb_status fosb_farfield_pmchwt(fosb_mesh mesh, double k0, const double* dirs, int64_t n_dir, const void* X,
                                 int64_t ldx, int64_t ncols, double weight, void* out, int64_t ldo, int accumulate,
                                 void* stream);

/* ---- Low-rank right-hand side of the tensor equations (Section VI, further work (ii)) ----
 * fosb_kernel_lowrank: pivoted Cholesky factorisation K ~ R^T R (Harbrecht, Peters and
 * Schneider 2012) of the covariance kernel matrix K_pq = sigma^2 rho(|x_p - x_q|) over the
 * vertices of nmesh meshes stacked in order (mesh i's vertices follow those of meshes
 * 0..i-1), so that for two of them K_12 ~ R_1^T R_2 with R_i the columns of mesh i.  Step m
 * takes as pivot the point with the largest diagonal entry of the remainder K - R^T R among
 * those not chosen yet (ties to the lowest index) and appends that remainder's column
 * divided by the square root of the pivot; the steps stop once the remainder's trace is
 * at most tol * trace(K) (trace(K) = V sigma^2), when no positive diagonal entry is left,
 * or after max_rank columns.  Kernel values are computed on the fly in FP64.
 *   meshes    : nmesh handles (host array)
 *   R         : device, max_rank x ldr float64 row-major (ldr >= total vertices V); row m is
 *               column m of the factor; rows >= *rank are left untouched
 *   rank      : host out, the number of columns written
 *   trace_err : host out (may be NULL), the trace of K - R^T R with *rank columns
 * Synchronises `stream` (the host checks the stopping rule every 32 columns).
 * Errors: FOSB_ERR_INVALID_ARG (bad kernel, tol < 0, max_rank < 1, ldr < V).
 *
 * fosb_covariance_lowrank: for one level, Y = A Z^{-1} B R_l^T (3 n_dir x r): the factor of
 * the far-field covariance under K ~ R^T R, since then
 *   A_1 Sigma_12 A_2^H ~ (A_1 Z_1^{-1} B_1 R_1^T)(A_2 Z_2^{-1} B_2 R_2^T)^H = Y_1 Y_2^H
 * (B, A and the refined solve as in fosb_covariance and fosb_farfield_moments).
 *   u   : device nominal current of this level; R : device r x V_l float64 (ldr >= V_l),
 *         the mesh's columns of the factor (a pointer into fosb_kernel_lowrank's R)
 *   Y   : device 3 n_dir x r row-major (ldy >= r), complex128 (FP64/MIXED factors) or
 *         complex64 (FP32), overwritten.  Synchronises `stream` (refinement).
 * fosb_lowrank_combine: out = (accumulate ? out : 0) + weight (M [+ op(M)]) with
 *   M = Y1 op(Y2), op = ^H (pseudo = 0) or ^T (pseudo = 1, the pseudo-covariance), the mirror
 *   added when hermitian_mirror = 1 (a block with l1 != l2 of the CT sum, Section IV-B).
 *   Y1, Y2 : device nd3 x r (ldy1, ldy2 >= r); out : device nd3 x nd3 (ldo >= nd3).
 *   Enqueued on `stream`. */
fosb_status fosb_kernel_lowrank(const fosb_mesh* meshes, int64_t nmesh, const fosb_cov_kernel* kernel, double tol,
                                int64_t max_rank, double* R, int64_t ldr, int64_t* rank, double* trace_err,
                                void* stream);
fosb_status fosb_covariance_lowrank(fosb_mesh mesh, fosb_lu lu, const void* u, double k, const double* R, int64_t ldr,
                                    int64_t r, const double* dirs, int64_t n_dir, const fosb_refine_opts* ropt,
                                    void* Y, int64_t ldy, void* stream);
fosb_status fosb_lowrank_combine(int64_t nd3, int64_t r, const void* Y1, int64_t ldy1, const void* Y2, int64_t ldy2,
                                 double weight, int hermitian_mirror, int pseudo, int prec, void* out, int64_t ldo,
                                 int accumulate, void* stream);

/* ---- A11: RCS mean and variance per direction ---------------------------------------
 * From the moments of fosb_farfield_moments, for every observation direction d (mean far
 * field f = F_d, 3 x 3 blocks C = Cov[F'_d] and P = E[F'_d F'_d^T] of the covariance and
 * pseudo-covariance, Sections II-C, III and IV-B):
 *   rcs_db[d] = 10 log10 sigma_d with sigma_d = |f|^2 / (4 pi) (convention 0: F of the expansion
 *               E_sc ~ exp(ik|x|)/(4 pi |x|) F, eq. RCS read with it), or sigma_d = 4 pi |f|^2
 *               (convention 1: the formula as printed; 10 log10((4 pi)^2) = 21.98 dB higher);
 *   var_db[d] = (20/ln 10)^2 Var[Re z] / |f|^4, z = f^H F'_d, Var[Re z] = (f^H C f + Re f^H P conj f)/2
 *               (first-order delta method; the same for both conventions);
 *   var_f[3d + c] = C_cc: the variance of each far-field component.
 *   F     : device, 3 n_dir complex (complex128 for FOSB_FP64/MIXED, complex64 for FOSB_FP32);
 *           component c of direction d at F[(3d + c) * incf] (incf = ncols of a mean-mode output)
 *   cov, pcov : device (3 n_dir) x (3 n_dir) row-major (ldc, ldp >= 3 n_dir); cov is needed by
 *           var_db and var_f, pcov by var_db, otherwise either may be NULL
 *   rcs_db, var_db : device n_dir float64; var_f : device 3 n_dir float64; each may be NULL
 * Enqueued on `stream` (no synchronisation).  Errors: FOSB_ERR_INVALID_ARG. */
fosb_status fosb_rcs_moments(int64_t n_dir, const void* F, int64_t incf, const void* cov, int64_t ldc, const void* pcov,
                             int64_t ldp, int prec, int convention, double* rcs_db, double* var_db, double* var_f,
                             void* stream);

/* ---- A12: monostatic RCS and its adjoint shape gradient --------------------------
 * For n plane waves E_inc_i = p_i exp(ik d_i . x) with solved currents U (u_i = Z^{-1} b_i),
 * the monostatic far field F_i = F(xh_i), xh_i = -d_i (Section II-C expansion), and
 *     sigma_i = |F_i|^2 / (4 pi)            (eq. RCS read with that expansion: RCS_dB = 10 log10 sigma).
 * With grad != NULL the call also writes grad = sum_i weights_i d q_i / dX (V x 3, the exact
 * derivative of the discrete q_i = sigma_i, or RCS_dB_i when db = 1, with respect to every
 * vertex coordinate):
 *     d sigma_i = (2/(4 pi)) Re[conj(F_i) . (dA_i u_i + A_i Z^{-1}(db_i - dZ u_i))],
 *     d RCS_dB_i = 10 / (sigma_i ln 10) d sigma_i,
 * evaluated by the adjoint lambda_i = Z^{-1} A_i^T c_i (Z^T = Z) and reverse-mode kernels
 * over the same triangle pairs and quadrature points as the assembly.  The paper
 * differentiates the continuous problem (Section III); this is the discrete counterpart.
 *   lu      : factorisation of Z (FOSB_FP64 or FOSB_MIXED); needed only with grad
 *   inc     : host, n x 9 (d, Re p, Im p) as in fosb_assemble_efie
 *   U       : device, N x n complex128 (ldu >= n)
 *   weights : host, n (dL/dq_i); needed only with grad
 *   db      : 0: q = sigma (m^2); 1: q = RCS_dB
 *   sigma   : host, n outputs q_i (may be NULL);  grad : device, V x 3 float64 (overwritten) or NULL
 * Synchronises `stream`. */
fosb_status fosb_rcs_monostatic(fosb_mesh mesh, fosb_lu lu, double k, const fosb_quad_opts* opts, const double* inc,
                                int64_t n_inc, const void* U, int64_t ldu, const double* weights, int db, double* sigma,
                                double* grad, void* stream);

/* ---- Batched scatterers -------------------------------------------------------------
 * Many independent scatterers of uneven size, each its own EFIE system Z_i u_i = b_i
 * (Sections II-C and IV-A), processed together: the paper solves its independent
 * sub-systems concurrently (Section V-D); here the units are whole scatterers. */
typedef struct {
  int warps;        /* test triangles per regular-pair tile of the persistent launch (4 or 8) */
  int ctas_per_sm;  /* CTAs per SM its register allocation is bounded for (4 warps: 5 or 4; 8 warps: 2 or 1) */
  double tuned_ms;  /* the chosen shape's time when the autotuner measured it, else 0 */
} fosb_batch_tuning;

/* Assembles Z_i (N_i x N_i complex128, ldz[i]) and, where n_inc[i] > 0, b_i (N_i x n_inc[i],
 * ldb[i]) for every item, as fosb_assemble_efie with prec = FOSB_MIXED would: regular pairs
 * in float-float (opts->arith = FOSB_ASM_FF, the default here) or FP64 (FOSB_ASM_FP64),
 * Sauter-Schwab touching pairs in FP64.  With float-float, the regular pairs of all items
 * run in ONE persistent launch whose CTAs take (item, 32 x W triangle tile) work items
 * from a device ticket; touching pairs and right-hand sides are one launch each.
 * tune = 1: the first call for a batch signature (item count, sum of T, sum of T^2) times
 * each candidate tile shape on this batch and keeps the fastest for later calls in the
 * process (the batch is then assembled once more with it); chosen (may be NULL) reports
 * the shape used.
 *   meshes, k     : host arrays of nbatch handles and wavenumbers
 *   Z             : host array of nbatch device pointers (caller-owned), ldz host array
 *   inc, n_inc    : host arrays: inc[i] host n_inc[i] x 9 (d, Re p, Im p); n_inc may be NULL
 *   b, ldb        : host arrays of device pointers and leading dimensions (used where n_inc[i] > 0)
 * Enqueued on `stream` (the tuning run synchronises it).  Errors: FOSB_ERR_INVALID_ARG. */
fosb_status fosb_assemble_efie_batched(int64_t nbatch, const fosb_mesh* meshes, const double* k,
                                       const fosb_quad_opts* opts, void* const* Z, const int64_t* ldz,
                                       const double* const* inc, const int64_t* n_inc, void* const* b,
                                       const int64_t* ldb, int tune, fosb_batch_tuning* chosen, void* stream);

/* Factors and solves every item: X_i = Z_i^{-1} B_i as fosb_factor + fosb_solve with prec
 * FOSB_MIXED (complex64 factors, FP64 refinement) or FOSB_FP64.  `workers` host threads
 * (<= 0: 4), each with its own stream, take the items largest first; every item waits for
 * the work already enqueued on `stream`.  The factorisations are kept until all items are
 * done and then released (peak memory: every item's factors at once).  stats and
 * item_status (host arrays of nbatch, may be NULL) receive each item's refinement record and
 * status.  Returns when all items are done: the first failing item's status, else FOSB_OK.
 *   Z, B, X : host arrays of device pointers (complex128, row-major), with n, ldz, nrhs,
 *             ldb, ldx host arrays; X_i may alias B_i. */
fosb_status fosb_solve_batched(int64_t nbatch, const void* const* Z, const int64_t* n, const int64_t* ldz,
                               const void* const* B, const int64_t* nrhs, const int64_t* ldb, void* const* X,
                               const int64_t* ldx, int prec, const fosb_refine_opts* ropt, int workers,
                               fosb_solve_stats* stats, int* item_status, void* stream);

/* ---- Monte Carlo over random shapes -------------------------------------------------
 * The paper's reference estimator of the shape statistics (Section V-C): sample surfaces
 * x_p + t xi_p n_p with xi ~ N(0, K), each solved, and sample moments of the far field.
 * The samples come from the caller's standard normal draws; the surfaces are solved with
 * the batched calls above; the moments are formed on the device. */

/* xi_s = L z_s for nsamp draws: K + 1e-12 sigma^2 I = L L^T with K_pq = kernel(|x_p - x_q|)
 * on the mesh vertices (the random normal velocity expanded at the vertices, Section III).
 *   z  : host, nsamp x nv standard normal draws;  xi : host, nsamp x nv outputs.
 * The Cholesky factorisation (nv^3/3 flops) runs on the host in the library.
 * Errors: FOSB_ERR_INVALID_ARG, FOSB_ERR_SINGULAR (K not positive definite). */
fosb_status fosb_field_samples(fosb_mesh mesh, const fosb_cov_kernel* kernel, int64_t nsamp, const double* z,
                               double* xi);

/* The sample surface x_p + t xi_p n_p of base (same triangles, the base's vertex normals n_p)
 * as a new mesh handle, as fosb_mesh_create would build it.  xi: host, nv values. */
fosb_status fosb_mesh_perturb(fosb_mesh base, const double* xi, double t, fosb_mesh* out);

/* Sample moments of nsamp far fields.  Fs: device n3 x nsamp complex128 (ldf >= nsamp; column s
 * the far field F_s of sample s, as a mean-mode fosb_farfield_moments output); F0: device n3,
 * the nominal far field.  Writes (device, complex128, each may be NULL; pcov needs cov):
 *   mean = (1/S) sum_s F_s (n3);
 *   cov  = (1/S) sum_s D_s D_s^H, pcov = (1/S) sum_s D_s D_s^T (n3 x n3, ldc / ldp), D_s = (F_s - F0)/t,
 * the Monte Carlo counterparts of the first-order Cov[F'] and E[F' F'^T] for perturbation
 * amplitude t.  Enqueued on `stream`.  Errors: FOSB_ERR_INVALID_ARG. */
fosb_status fosb_mc_moments(int64_t n3, int64_t nsamp, const void* Fs, int64_t ldf, const void* F0, double t,
                            void* mean, void* cov, int64_t ldc, void* pcov, int64_t ldp, void* stream);

/* ---- FP64-class complex matrix product ------------------------------------------------
 * C = A B for complex128 row-major A (M x K, lda), B (K x N, ldb), C (M x N, ldc) (device),
 * computed without the FP64 pipe (1.25 TFLOP/s on this part) by either of the two products
 * behind the refinement residuals:
 *   method 0: exact digit splitting on the bf16 tensor cores: each row of A and column of B is
 *             scaled by a power of two and cut into seven balanced base-256 digits; the digit
 *             products up to order 6 are summed exactly (integer order sums per 64-wide k chunk):
 *             within a few units of 2^-52 of (|A||B|)_ij, independent of K;
 *   method 1: float-float (pairs of floats, about 48 significant bits) on the FP32 pipe:
 *             within K 2^-48 of (|A||B|)_ij.
 * Allocates its digit scratch stream-ordered; synchronises `stream`.
 * Errors: FOSB_ERR_INVALID_ARG, FOSB_ERR_TIMEOUT. */
fosb_status fosb_zgemm_fp64class(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B,
                                 int64_t ldb, void* C, int64_t ldc, int method, void* stream);

/* ---- Diagnostics: bounded device waits ---------------------------------------------
 * Every spin-wait of the library's kernels gives up after a number of polls, sets the
 * status word of the call to FOSB_ERR_TIMEOUT and returns, so the call reports
 * FOSB_ERR_TIMEOUT and the context stays usable.  This sets that number for the LU panel
 * grid barriers and the streaming triangular-sweep flags on the current device (polls <= 0
 * restores the default 2^26, about 2 s); failure-detection tests use a tiny limit to make
 * the waits run out.  The tensor-core kernels keep their own limits.  A factorisation whose
 * wait ran out leaves its outputs unspecified; destroy and recreate its handle. */
fosb_status fosb_debug_set_wait_limit(int64_t polls);

/* Throughput microbenchmarks of the execution units the kernels are bound by (diagnostics
 * for roofline denominators).  kind 0: FP32 FMA pipe; 1: FP64 FMA pipe; 2: tcgen05.mma
 * kind::tf32 (M = 128, N = 256, K = 8) back to back from shared memory, one CTA per SM; 3: the
 * same with kind::f16 bf16 (K = 16).  Writes the best of five CUDA-event-timed launches on
 * the legacy default stream in TFLOP/s (2 flops per multiply-add).  Allocates and frees a few
 * bytes; synchronises the device.  Errors: FOSB_ERR_INVALID_ARG, FOSB_ERR_TIMEOUT. */
fosb_status fosb_peak_microbench(int kind, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* FOSB_H */
