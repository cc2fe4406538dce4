// Adjoint (reverse-mode) shape gradient of the discrete EFIE quantities with respect to
// the mesh vertex coordinates X (V x 3), used for gradients of monostatic RCS.
//
// For fixed coefficient vectors the kernels accumulate the real gradient of
//   J_Z = sum_i lambda_i^T Z(X) u_i                                  (pair kernels)
//   J_P = sum_i sum_t sum_j w_{e_j,i} alpha_i (s_j l_j / 2) sum_q w_q pi_i.(x_q - P_j) exp(ik d_i.x_q)
//                                                                    (triangle kernel)
// J_P covers both the plane-wave right-hand side (w = lambda, alpha = -1, pi = p_i,
// d = d_i: the term lambda^T b) and the far-field matrix (w = u, alpha = -ik,
// pi = (I - xh xh^T) c_i, d = -xh_i: the term c^T A u).
//
// With RWG functions the area factors cancel: a triangle-pair block is
//   Blk_jk = s_j s'_k l_j l'_k sum_pq w_pq G(r) [-(ik/4)(x_p - P_j).(y_q - Q_k) - 1/(ik)]
// (w_pq = product of the 6-point weights, or 4 x the Sauter-Schwab reference weights), so
// J_Z per pair is sum_pq w_pq G(r) H(x, y) with the bilinear
//   H = -(ik/4)(S x.y - x.U - V.y + c) + (i/k) S,   S = sum W_jk, U = sum W_jk Q_k,
//   V = sum W_jk P_j, c = sum W_jk P_j.Q_k,  W_jk = s_j s'_k l_j l'_k sum_i lambda_{j,i} u_{k,i}.
// Its derivatives with respect to the quadrature points (G' = G (ik - 1/r)), the opposite
// vertices and the edge lengths are accumulated (real parts) and chained to the vertices.
#include <cuda_runtime.h>

#include "fosb_internal.h"

namespace fosb {

// this translation unit's copy of the quadrature rules (uploaded with the assembly's)
__constant__ double c_bary[6][3];
__constant__ double c_w[6];
__constant__ double c_glx[16];
__constant__ double c_glw[16];

void upload_rules_adjoint(const Rules& r) {
  cudaMemcpyToSymbol(c_bary, r.bary, sizeof(r.bary));
  cudaMemcpyToSymbol(c_w, r.w, sizeof(r.w));
  cudaMemcpyToSymbol(c_glx, r.glx, sizeof(r.glx));
  cudaMemcpyToSymbol(c_glw, r.glw, sizeof(r.glw));
}

namespace {

constexpr double kInv4Pi = 0.07957747154594767;

struct Cx {
  double r, i;
};
__device__ __forceinline__ Cx operator+(Cx a, Cx b) { return {a.r + b.r, a.i + b.i}; }
__device__ __forceinline__ Cx operator-(Cx a, Cx b) { return {a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ Cx operator*(Cx a, Cx b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ Cx operator*(Cx a, double s) { return {a.r * s, a.i * s}; }

// Per-pair state: the coefficient matrix W (already scaled by s s' l l'), origins and the
// local (origin-relative) opposite vertices of both triangles.
struct PairCoef {
  Cx W[3][3];
  Cx S, U[3], V[3], c;
};

__device__ void make_coef(const double P[3][3], const double Q[3][3], PairCoef& pc) {
  pc.S = {0, 0};
  pc.c = {0, 0};
  for (int d = 0; d < 3; ++d) pc.U[d] = pc.V[d] = Cx{0, 0};
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) {
      Cx w = pc.W[j][k];
      pc.S = pc.S + w;
      double pq = P[j][0] * Q[k][0] + P[j][1] * Q[k][1] + P[j][2] * Q[k][2];
      pc.c = pc.c + w * pq;
      for (int d = 0; d < 3; ++d) {
        pc.U[d] = pc.U[d] + w * Q[k][d];
        pc.V[d] = pc.V[d] + w * P[j][d];
      }
    }
}

// Accumulators of one pair: real gradients at the points and complex moments.
struct PairAcc {
  double gx[6][3], gy[6][3];   // regular: per test / trial point
  Cx I0, Mx[3], My[3], Mxy;
};

// One point pair: x, y local coordinates (x - o1, y - o2), dvec = x - y (absolute),
// weight w (includes the 1/(4 pi) of G).  Returns the real gradient contributions with
// respect to x and y and adds the moments.
__device__ __forceinline__ void point_pair(double k, const PairCoef& pc, const double x[3], const double y[3],
                                           const double dvec[3], double w, double gx[3], double gy[3],
                                           PairAcc& A) {
  double r2 = dvec[0] * dvec[0] + dvec[1] * dvec[1] + dvec[2] * dvec[2];
  double rinv = rsqrt(r2);
  double r = r2 * rinv;
  double sn, cs;
  sincos(k * r, &sn, &cs);
  Cx G = {cs * rinv * w, sn * rinv * w};
  Cx Gp_over_r = G * Cx{-rinv * rinv, k * rinv};  // G'(r)/r = G (ik - 1/r)/r
  double xy = x[0] * y[0] + x[1] * y[1] + x[2] * y[2];
  Cx xU = pc.U[0] * x[0] + pc.U[1] * x[1] + pc.U[2] * x[2];
  Cx Vy = pc.V[0] * y[0] + pc.V[1] * y[1] + pc.V[2] * y[2];
  Cx B = pc.S * xy - xU - Vy + pc.c;
  const Cx mik4 = {0.0, -0.25 * k};
  Cx H = mik4 * B + Cx{0.0, 1.0 / k} * pc.S;
  Cx GH = Gp_over_r * H;
  Cx Gm = G * mik4;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Cx dHx = pc.S * y[d] - pc.U[d];  // (S y - U)
    Cx dHy = pc.S * x[d] - pc.V[d];  // (S x - V)
    gx[d] += GH.r * dvec[d] + (Gm * dHx).r;
    gy[d] += -GH.r * dvec[d] + (Gm * dHy).r;
  }
  A.I0 = A.I0 + G;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    A.Mx[d] = A.Mx[d] + G * x[d];
    A.My[d] = A.My[d] + G * y[d];
  }
  A.Mxy = A.Mxy + G * xy;
}

// Explicit (non point) terms of one pair: opposite vertices and edge lengths.
//   dJ/dP_j = (ik/4) sum_k W_jk (My - Q_k I0),  dJ/dQ_k = (ik/4) sum_j W_jk (Mx - P_j I0),
//   dJ/dl_j = sum_k W_jk K_jk / l_j,  K_jk = -(ik/4)(Mxy - Q_k.Mx - P_j.My + P_j.Q_k I0) + (i/k) I0.
__device__ void explicit_terms(double k, const PairCoef& pc, const PairAcc& A, const double P[3][3],
                               const double Q[3][3], const double l1[3], const double l2[3], double gP[3][3],
                               double gQ[3][3], double gl1[3], double gl2[3]) {
  const Cx ik4 = {0.0, 0.25 * k};
  for (int j = 0; j < 3; ++j) {
    gl1[j] = gl2[j] = 0.0;
    for (int d = 0; d < 3; ++d) gP[j][d] = gQ[j][d] = 0.0;
  }
  for (int j = 0; j < 3; ++j)
    for (int kk = 0; kk < 3; ++kk) {
      Cx w = pc.W[j][kk];
      Cx wik = w * ik4;
      for (int d = 0; d < 3; ++d) {
        gP[j][d] += (wik * (A.My[d] - A.I0 * Q[kk][d])).r;
        gQ[kk][d] += (wik * (A.Mx[d] - A.I0 * P[j][d])).r;
      }
      Cx QMx = A.Mx[0] * Q[kk][0] + A.Mx[1] * Q[kk][1] + A.Mx[2] * Q[kk][2];
      Cx PMy = A.My[0] * P[j][0] + A.My[1] * P[j][1] + A.My[2] * P[j][2];
      double pq = P[j][0] * Q[kk][0] + P[j][1] * Q[kk][1] + P[j][2] * Q[kk][2];
      Cx K = Cx{0.0, -0.25 * k} * (A.Mxy - QMx - PMy + A.I0 * pq) + Cx{0.0, 1.0 / k} * A.I0;
      double v = (w * K).r;
      gl1[j] += v / l1[j];
      gl2[kk] += v / l2[kk];
    }
}

// W_jk = s_j s'_k l_j l'_k sum_i lambda[e1_j, i] u[e2_k, i] (+ the mirrored term for
// touching pairs whose transpose block is not evaluated separately).
__device__ void load_w(const double* lam, const double* U, int64_t ld, int64_t m, const int e1[3], const int e2[3],
                       const double sl1[3], const double sl2[3], bool mirror, PairCoef& pc) {
  for (int j = 0; j < 3; ++j)
    for (int kk = 0; kk < 3; ++kk) {
      Cx acc = {0, 0};
      for (int64_t i = 0; i < m; ++i) {
        Cx a = {lam[2 * (e1[j] * ld + i)], lam[2 * (e1[j] * ld + i) + 1]};
        Cx b = {U[2 * (e2[kk] * ld + i)], U[2 * (e2[kk] * ld + i) + 1]};
        acc = acc + a * b;
        if (mirror) {
          Cx a2 = {lam[2 * (e2[kk] * ld + i)], lam[2 * (e2[kk] * ld + i) + 1]};
          Cx b2 = {U[2 * (e1[j] * ld + i)], U[2 * (e1[j] * ld + i) + 1]};
          acc = acc + a2 * b2;
        }
      }
      pc.W[j][kk] = acc * (sl1[j] * sl2[kk]);
    }
}

__device__ __forceinline__ void tri_edge_data(const DevMesh& m, int64_t t, int v[3], int e[3], double sl[3],
                                              double l[3], double V[3][3]) {
  for (int a = 0; a < 3; ++a) {
    v[a] = m.tris[3 * t + a];
    e[a] = m.tri_edge[3 * t + a];
    for (int d = 0; d < 3; ++d) V[a][d] = m.verts[3 * v[a] + d];
  }
  for (int j = 0; j < 3; ++j) {
    const double* A = V[(j + 1) % 3];
    const double* B = V[(j + 2) % 3];
    double dx = B[0] - A[0], dy = B[1] - A[1], dz = B[2] - A[2];
    l[j] = sqrt(dx * dx + dy * dy + dz * dz);
    sl[j] = (m.tri_coef[3 * t + j] > 0 ? 1.0 : -1.0) * l[j];
  }
}

// gradient of l_j (edge opposite local vertex j) into the vertex gradient array g (3 x 3)
__device__ __forceinline__ void chain_lengths(const double V[3][3], const double l[3], const double gl[3],
                                              double g[3][3]) {
  for (int j = 0; j < 3; ++j) {
    int a = (j + 1) % 3, b = (j + 2) % 3;
    for (int d = 0; d < 3; ++d) {
      double e = (V[b][d] - V[a][d]) / l[j];
      g[b][d] += gl[j] * e;
      g[a][d] -= gl[j] * e;
    }
  }
}

__device__ __forceinline__ void add_grad(double* grad, int v, const double g[3], double sgn) {
  for (int d = 0; d < 3; ++d) atomicAdd(grad + 3 * v + d, sgn * g[d]);
}

// ------------------------------------------------------------------ regular pairs
__global__ void __launch_bounds__(128) adjoint_regular_kernel(DevMesh m, double k, const double* lam, const double* U,
                                                              int64_t ld, int64_t nrhs, double* grad) {
  const int64_t t1 = int64_t(blockIdx.y) * 4 + (threadIdx.x >> 5);
  const int64_t t2 = int64_t(blockIdx.x) * 32 + (threadIdx.x & 31);
  if (t1 >= m.nt || t2 >= m.nt) return;
  int v1[3], v2[3], e1[3], e2[3];
  double sl1[3], sl2[3], l1[3], l2[3], V1[3][3], V2[3][3];
  tri_edge_data(m, t1, v1, e1, sl1, l1, V1);
  tri_edge_data(m, t2, v2, e2, sl2, l2, V2);
  bool touch = false;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) touch |= v1[a] == v2[b];
  if (touch) return;
  double P[3][3], Q[3][3], D[3];
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) {
      P[a][d] = V1[a][d] - V1[0][d];
      Q[a][d] = V2[a][d] - V2[0][d];
    }
  for (int d = 0; d < 3; ++d) D[d] = V1[0][d] - V2[0][d];
  PairCoef pc;
  load_w(lam, U, ld, nrhs, e1, e2, sl1, sl2, false, pc);
  make_coef(P, Q, pc);
  PairAcc A;
  A.I0 = A.Mxy = Cx{0, 0};
  for (int d = 0; d < 3; ++d) A.Mx[d] = A.My[d] = Cx{0, 0};
  double xq[6][3], yq[6][3];
  for (int q = 0; q < 6; ++q)
    for (int d = 0; d < 3; ++d) {
      xq[q][d] = m.tri_qp[18 * t1 + 3 * q + d] - V1[0][d];
      yq[q][d] = m.tri_qp[18 * t2 + 3 * q + d] - V2[0][d];
      A.gx[q][d] = A.gy[q][d] = 0.0;
    }
  for (int p = 0; p < 6; ++p)
    for (int q = 0; q < 6; ++q) {
      double dv[3] = {D[0] + xq[p][0] - yq[q][0], D[1] + xq[p][1] - yq[q][1], D[2] + xq[p][2] - yq[q][2]};
      point_pair(k, pc, xq[p], yq[q], dv, c_w[p] * c_w[q] * kInv4Pi, A.gx[p], A.gy[q], A);
    }
  double gP[3][3], gQ[3][3], gl1[3], gl2[3];
  explicit_terms(k, pc, A, P, Q, l1, l2, gP, gQ, gl1, gl2);
  double g1[3][3], g2[3][3];
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) {
      double s1 = gP[a][d], s2 = gQ[a][d];
      for (int q = 0; q < 6; ++q) {
        s1 += c_bary[q][a] * A.gx[q][d];
        s2 += c_bary[q][a] * A.gy[q][d];
      }
      g1[a][d] = s1;
      g2[a][d] = s2;
    }
  chain_lengths(V1, l1, gl1, g1);
  chain_lengths(V2, l2, gl2, g2);
  // J_Z enters the objective with a minus sign
  for (int a = 0; a < 3; ++a) {
    add_grad(grad, v1[a], g1[a], -1.0);
    add_grad(grad, v2[a], g2[a], -1.0);
  }
}

// ------------------------------------------------------------------ touching pairs
// One CTA (128 threads) per touching pair (t1 <= t2), Sauter-Schwab points in the
// orientation of the assembly; gradients at the points are chained immediately to the
// permuted vertices through the barycentric weights of chi.
__device__ __forceinline__ void chi_bary(double u1, double u2, double a[3]) {
  a[0] = 1.0 - u1;
  a[1] = u1 - u2;
  a[2] = u2;
}

__global__ void __launch_bounds__(128) adjoint_singular_kernel(DevMesh m, double k, int nss, const double* lam,
                                                               const double* U, int64_t ld, int64_t nrhs,
                                                               double* grad) {
  const TouchPair tp = m.touch[blockIdx.x];
  const int t1 = tp.t1, t2 = tp.t2;
  int v1[3], v2[3], e1[3], e2[3];
  double sl1[3], sl2[3], l1[3], l2[3], V1[3][3], V2[3][3];
  tri_edge_data(m, t1, v1, e1, sl1, l1, V1);
  tri_edge_data(m, t2, v2, e2, sl2, l2, V2);
  double Pp[3][3], Qp[3][3];  // permuted vertices (Sauter-Schwab order), absolute
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) {
      Pp[a][d] = m.verts[3 * tp.p[a] + d];
      Qp[a][d] = m.verts[3 * tp.q[a] + d];
    }
  // local coordinates relative to the shared vertex Pp[0] == Qp[0]
  double P[3][3], Q[3][3];
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) {
      P[a][d] = V1[a][d] - Pp[0][d];
      Q[a][d] = V2[a][d] - Qp[0][d];
    }
  PairCoef pc;
  load_w(lam, U, ld, nrhs, e1, e2, sl1, sl2, t1 != t2, pc);
  make_coef(P, Q, pc);
  PairAcc A;
  A.I0 = A.Mxy = Cx{0, 0};
  for (int d = 0; d < 3; ++d) A.Mx[d] = A.My[d] = Cx{0, 0};
  double gp[3][3] = {}, gq[3][3] = {};  // gradients w.r.t. the permuted vertices
  const int n2 = nss * nss, n4 = n2 * n2;
  auto visit = [&](double u1, double u2, double w1, double w2, double wt) {
    double ax[3], ay[3], x[3], y[3], dv[3];
    chi_bary(u1, u2, ax);
    chi_bary(w1, w2, ay);
    for (int d = 0; d < 3; ++d) {
      x[d] = u1 * (Pp[1][d] - Pp[0][d]) + u2 * (Pp[2][d] - Pp[1][d]);
      y[d] = w1 * (Qp[1][d] - Qp[0][d]) + w2 * (Qp[2][d] - Qp[1][d]);
      dv[d] = x[d] - y[d];
    }
    double gx[3] = {0, 0, 0}, gy[3] = {0, 0, 0};
    point_pair(k, pc, x, y, dv, 4.0 * wt * kInv4Pi, gx, gy, A);
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < 3; ++d) {
        gp[a][d] += ax[a] * gx[d];
        gq[a][d] += ay[a] * gy[d];
      }
  };
  for (int idx = threadIdx.x; idx < n4; idx += blockDim.x) {
    int a = idx / (n2 * nss), b = (idx / n2) % nss, c = (idx / nss) % nss, d = idx % nss;
    double xi = c_glx[a], e1 = c_glx[b], e2 = c_glx[c], e3 = c_glx[d];
    double w4 = c_glw[a] * c_glw[b] * c_glw[c] * c_glw[d];
    if (tp.kind == 3) {
      double w = w4 * xi * xi * xi * e1 * e1 * e2;
      visit(xi, xi * (1 - e1 + e1 * e2), xi * (1 - e1 * e2 * e3), xi * (1 - e1), w);
      visit(xi * (1 - e1 * e2 * e3), xi * (1 - e1), xi, xi * (1 - e1 + e1 * e2), w);
      visit(xi, xi * e1 * (1 - e2 + e2 * e3), xi * (1 - e1 * e2), xi * e1 * (1 - e2), w);
      visit(xi * (1 - e1 * e2), xi * e1 * (1 - e2), xi, xi * e1 * (1 - e2 + e2 * e3), w);
      visit(xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), xi, xi * e1 * (1 - e2), w);
      visit(xi, xi * e1 * (1 - e2), xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), w);
    } else if (tp.kind == 2) {
      double w0 = w4 * xi * xi * xi * e1 * e1, w1 = w0 * e2;
      visit(xi, xi * e1 * e3, xi * (1 - e1 * e2), xi * e1 * (1 - e2), w0);
      visit(xi, xi * e1, xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3), w1);
      visit(xi * (1 - e1 * e2), xi * e1 * (1 - e2), xi, xi * e1 * e2 * e3, w1);
      visit(xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3), xi, xi * e1, w1);
      visit(xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), xi, xi * e1 * e2, w1);
    } else {
      double w = w4 * xi * xi * xi * e2;
      visit(xi, xi * e1, xi * e2, xi * e2 * e3, w);
      visit(xi * e2, xi * e2 * e3, xi, xi * e1, w);
    }
  }
  // block reduction: 18 + 18 point-chained reals and the 16 moment reals
  __shared__ double red[4][52];
  double vals[52];
  int o = 0;
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) {
      vals[o++] = gp[a][d];
      vals[o++] = gq[a][d];
    }
  vals[o++] = A.I0.r; vals[o++] = A.I0.i; vals[o++] = A.Mxy.r; vals[o++] = A.Mxy.i;
  for (int d = 0; d < 3; ++d) {
    vals[o++] = A.Mx[d].r; vals[o++] = A.Mx[d].i; vals[o++] = A.My[d].r; vals[o++] = A.My[d].i;
  }
  for (int i = 0; i < 52; ++i) {
    double v = vals[i];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    vals[i] = v;
  }
  if ((threadIdx.x & 31) == 0)
    for (int i = 0; i < 52; ++i) red[threadIdx.x >> 5][i] = vals[i];
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int i = 0; i < 52; ++i) vals[i] = red[0][i] + red[1][i] + red[2][i] + red[3][i];
  o = 0;
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) {
      gp[a][d] = vals[o++];
      gq[a][d] = vals[o++];
    }
  A.I0 = {vals[o], vals[o + 1]}; o += 2;
  A.Mxy = {vals[o], vals[o + 1]}; o += 2;
  for (int d = 0; d < 3; ++d) {
    A.Mx[d] = {vals[o], vals[o + 1]};
    A.My[d] = {vals[o + 2], vals[o + 3]};
    o += 4;
  }
  double gP[3][3], gQ[3][3], gl1[3], gl2[3];
  explicit_terms(k, pc, A, P, Q, l1, l2, gP, gQ, gl1, gl2);
  double g1[3][3], g2[3][3];
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) {
      g1[a][d] = gP[a][d];
      g2[a][d] = gQ[a][d];
    }
  chain_lengths(V1, l1, gl1, g1);
  chain_lengths(V2, l2, gl2, g2);
  for (int a = 0; a < 3; ++a) {
    add_grad(grad, v1[a], g1[a], -1.0);
    add_grad(grad, v2[a], g2[a], -1.0);
    add_grad(grad, tp.p[a], gp[a], -1.0);
    add_grad(grad, tp.q[a], gq[a], -1.0);
  }
}

// ------------------------------------------------------------------ plane-wave moments
// J_P term for one (triangle, column i): coefficient vector pi (complex 3), direction dd,
// alpha (complex), edge weights w (N x m, column i).  Thread per (triangle, column).
__global__ void adjoint_planewave_kernel(DevMesh m, double k, int64_t ncols, const double* pw /* ncols x 11 */,
                                         const double* wgt, int64_t ldw, double* grad) {
  int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= m.nt * ncols) return;
  const int64_t t = gid / ncols, i = gid % ncols;
  const double* c = pw + 11 * i;  // d(3), Re pi(3), Im pi(3), alpha (re, im)
  const Cx pi3[3] = {{c[3], c[6]}, {c[4], c[7]}, {c[5], c[8]}};
  const Cx alpha = {c[9], c[10]};
  int v[3], e[3];
  double sl[3], l[3], V[3][3];
  tri_edge_data(m, t, v, e, sl, l, V);
  Cx kap[3];
  for (int j = 0; j < 3; ++j) {
    Cx w = {wgt[2 * (e[j] * ldw + i)], wgt[2 * (e[j] * ldw + i) + 1]};
    kap[j] = w * alpha * (0.5 * sl[j]);
  }
  double g[3][3] = {}, gl[3] = {0, 0, 0};
  for (int q = 0; q < 6; ++q) {
    double x[3];
    for (int d = 0; d < 3; ++d) x[d] = m.tri_qp[18 * t + 3 * q + d];
    double sn, cs;
    sincos(k * (c[0] * x[0] + c[1] * x[1] + c[2] * x[2]), &sn, &cs);
    Cx E = {cs * c_w[q], sn * c_w[q]};
    for (int j = 0; j < 3; ++j) {
      Cx pxp = {0, 0};
      for (int d = 0; d < 3; ++d) pxp = pxp + pi3[d] * (x[d] - V[j][d]);
      Cx kE = kap[j] * E;
      Cx term = kE * pxp;
      gl[j] += term.r / l[j];
      Cx ikd_pxp = Cx{0.0, k} * pxp;
      for (int d = 0; d < 3; ++d) {
        double gxd = (kE * (pi3[d] + ikd_pxp * c[d])).r;
        for (int a = 0; a < 3; ++a) g[a][d] += c_bary[q][a] * gxd;
        g[j][d] -= (kE * pi3[d]).r;  // explicit opposite vertex P_j
      }
    }
  }
  chain_lengths(V, l, gl, g);
  for (int a = 0; a < 3; ++a) add_grad(grad, v[a], g[a], 1.0);
}

inline unsigned cdiv(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }

}  // namespace

cudaError_t launch_adjoint_pairs(const DevMesh& m, double k, int nss, const double* lam, const double* U, int64_t ld,
                                 int64_t nrhs, double* grad, cudaStream_t s) {
  dim3 grid(cdiv(m.nt, 32), cdiv(m.nt, 4));
  if (grid.y > 65535u) return cudaErrorInvalidValue;
  adjoint_regular_kernel<<<grid, 128, 0, s>>>(m, k, lam, U, ld, nrhs, grad);
  note_launches(1);
  if (m.ntouch > 0) {
    adjoint_singular_kernel<<<unsigned(m.ntouch), 128, 0, s>>>(m, k, nss, lam, U, ld, nrhs, grad);
    note_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_adjoint_planewave(const DevMesh& m, double k, int64_t ncols, const double* d_pw, const double* wgt,
                                     int64_t ldw, double* grad, cudaStream_t s) {
  if (ncols == 0) return cudaSuccess;
  adjoint_planewave_kernel<<<cdiv(m.nt * ncols, 128), 128, 0, s>>>(m, k, ncols, d_pw, wgt, ldw, grad);
  return launched();
}

}  // namespace fosb
