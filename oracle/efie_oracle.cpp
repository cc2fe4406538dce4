// FP64 CPU oracle for the EFIE Galerkin quadrature of the FOSB method.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the CUDA
// library is checked against; it shares no code with the library and the library
// never calls it.  Only tests/, the smoke check and the benchmark's CPU-baseline leg
// load it.
//
// What it computes (all with std::complex<double>, one quadrature point at a time):
//   * Z_mn = <T_k f_n, f_m>_x  (Section II-B, EFIO T_k, and the Galerkin system of
//     Section IV-A).  With the x-pairing <u,v>_x = int u.(n x v), the EFIO
//     T_k = gamma_D E_k and surface integration by parts this is
//       Z_mn = -[ ik int int G f_m(x).f_n(y) + 1/(ik) int int G div f_m div f_n ],
//     G(x,y) = exp(ik|x-y|)/(4 pi |x-y|)  (Section II-B, the potentials).
//   * b_m = <gamma_D E_inc, f_m>_x = - int E_inc . f_m, E_inc = p exp(ik d.x)
//     (Section V, the incident field; the PEC EFIE of Section II-C).
//   * the far-field matrix: E_sc = -E_k j gives, in the expansion of Section II-C,
//       F(xh) = -ik (I - xh xh^T) sum_n u_n int f_n(y) exp(-ik xh.y) dy.
//   * the shape-derivative right-hand side of Section III, PEC case, in weak form:
//       g_m = - sum_n u_n int v_n [ ik f_m.f_n + 1/(ik) div f_m div f_n ],
//     v_n = sum_p xi_p psi_p nu_{p,T} (P1 hat psi_p, nu_{p,T} = n_p . n_T).
//   * the dielectric (PMCHWT) system of Section II-C: the MFIO blocks
//     <K_k f_n, f_m>_x, K_k = {gamma_D H_k}, the 2N x 2N matrix of A_0 + A^_1 and the
//     far field of the exterior Cauchy data (j, m).
//
// RWG functions (lowest-order div-conforming, Section IV): on the triangle T with
// opposite vertex p, f = s l/(2 A_T) (x - p), div f = s l/A_T, s = +1 on the
// triangle where the edge (a<b) runs a->b counter-clockwise, s = -1 on the other.
//
// Quadrature: regular (vertex-disjoint) triangle pairs use the 6-point degree-4
// symmetric triangle rule in x and y (36 point pairs).  Pairs that share a vertex,
// an edge or are identical use the Sauter-Schwab regularising maps (Sauter & Schwab,
// Boundary Element Methods, Section 5.2.1) with n_ss-point Gauss-Legendre per
// coordinate of the unit 4-cube.  Touching blocks are evaluated for the ordered
// pair (t1 < t2) and transposed for (t2, t1).
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

using cplx = std::complex<double>;

namespace {

struct Vec3 {
  double x, y, z;
};
inline Vec3 sub(Vec3 a, Vec3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline Vec3 add(Vec3 a, Vec3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline Vec3 scale(Vec3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline double dot(Vec3 a, Vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline Vec3 cross(Vec3 a, Vec3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double norm(Vec3 a) { return std::sqrt(dot(a, a)); }

struct MeshView {
  const double* verts;
  const int32_t* tris;
  int64_t nt;
  const int32_t* tri_edge;   // T x 3, local edge i is opposite local vertex i
  const double* tri_sign;    // T x 3, +1 / -1
  const double* edge_len;    // N
  Vec3 v(int32_t i) const { return {verts[3 * i], verts[3 * i + 1], verts[3 * i + 2]}; }
  Vec3 tv(int64_t t, int a) const { return v(tris[3 * t + a]); }
  double area(int64_t t) const { return 0.5 * norm(cross(sub(tv(t, 1), tv(t, 0)), sub(tv(t, 2), tv(t, 0)))); }
  Vec3 unit_normal(int64_t t) const {
    Vec3 n = cross(sub(tv(t, 1), tv(t, 0)), sub(tv(t, 2), tv(t, 0)));
    return scale(n, 1.0 / norm(n));
  }
};

struct Rules {
  const double* qb;  // nq x 3 barycentric coordinates of the triangle rule
  const double* qw;  // nq weights, summing to 1
  int nq;
  const double* glx;  // n_ss Gauss-Legendre nodes on [0,1]
  const double* glw;  // n_ss weights on [0,1]
  int nss;
};

inline cplx helmholtz_g(double k, double r) {
  // G = exp(ik r) / (4 pi r)
  return std::exp(cplx(0.0, k * r)) / (4.0 * M_PI * r);
}

// One point pair contributes w * G(x,y) * [ -ik f_i(x).f_j(y) - 1/(ik) div_i div_j ]
// to every entry (i, j) of the 3 x 3 local block of the triangle pair (t1, t2).
struct LocalRWG {
  Vec3 opp[3];     // opposite vertices p_i
  double coef[3];  // s_i l_i / (2 A)
  double div[3];   // s_i l_i / A
};

LocalRWG local_rwg(const MeshView& m, int64_t t) {
  LocalRWG r;
  double A = m.area(t);
  for (int i = 0; i < 3; ++i) {
    double s = m.tri_sign[3 * t + i];
    double l = m.edge_len[m.tri_edge[3 * t + i]];
    r.opp[i] = m.tv(t, i);
    r.coef[i] = s * l / (2.0 * A);
    r.div[i] = s * l / A;
  }
  return r;
}

void add_point_pair(double k, const LocalRWG& f, const LocalRWG& g, Vec3 x, Vec3 y, double w, cplx blk[3][3]) {
  const cplx ik(0.0, k);
  double r = norm(sub(x, y));
  cplx G = helmholtz_g(k, r) * w;
  for (int i = 0; i < 3; ++i) {
    Vec3 fi = scale(sub(x, f.opp[i]), f.coef[i]);
    for (int j = 0; j < 3; ++j) {
      Vec3 gj = scale(sub(y, g.opp[j]), g.coef[j]);
      blk[i][j] += -ik * G * dot(fi, gj) - G * (f.div[i] * g.div[j]) / ik;
    }
  }
}

// Regular pair: 6-point rule in each triangle.
void regular_block(const MeshView& m, const Rules& q, double k, int64_t t1, int64_t t2, cplx blk[3][3]) {
  LocalRWG f = local_rwg(m, t1), g = local_rwg(m, t2);
  double A1 = m.area(t1), A2 = m.area(t2);
  Vec3 a0 = m.tv(t1, 0), a1 = m.tv(t1, 1), a2 = m.tv(t1, 2);
  Vec3 b0 = m.tv(t2, 0), b1 = m.tv(t2, 1), b2 = m.tv(t2, 2);
  for (int p = 0; p < q.nq; ++p) {
    Vec3 x = add(add(scale(a0, q.qb[3 * p]), scale(a1, q.qb[3 * p + 1])), scale(a2, q.qb[3 * p + 2]));
    for (int s = 0; s < q.nq; ++s) {
      Vec3 y = add(add(scale(b0, q.qb[3 * s]), scale(b1, q.qb[3 * s + 1])), scale(b2, q.qb[3 * s + 2]));
      add_point_pair(k, f, g, x, y, q.qw[p] * A1 * q.qw[s] * A2, blk);
    }
  }
}

// Parameterisation of Sauter-Schwab: chi(xh) = P0 + xh1 (P1 - P0) + xh2 (P2 - P1) on
// the reference triangle {0 <= xh2 <= xh1 <= 1}; |det D chi| = 2 A.
inline Vec3 chi(const Vec3 P[3], double u1, double u2) {
  return add(add(P[0], scale(sub(P[1], P[0]), u1)), scale(sub(P[2], P[1]), u2));
}

enum PairKind { REGULAR = 0, VERTEX = 1, EDGE = 2, IDENTICAL = 3 };

// Sauter-Schwab point generator: visits every (x, y, weight) of the regularised
// 4-cube rule for a touching pair whose vertex orderings are P (x triangle) and Q
// (y triangle); "jac" is the product of the two parameterisation Jacobians.
template <class Visit>
void ss_points(PairKind kind, const Vec3 P[3], const Vec3 Q[3], const Rules& q, double jac, Visit&& visit) {
  const int n = q.nss;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < n; ++c)
        for (int d = 0; d < n; ++d) {
          double xi = q.glx[a], e1 = q.glx[b], e2 = q.glx[c], e3 = q.glx[d];
          double w4 = q.glw[a] * q.glw[b] * q.glw[c] * q.glw[d] * jac;
          if (kind == IDENTICAL) {
            double w = w4 * xi * xi * xi * e1 * e1 * e2;
            double xs[6][4] = {
                {xi, xi * (1 - e1 + e1 * e2), xi * (1 - e1 * e2 * e3), xi * (1 - e1)},
                {xi * (1 - e1 * e2 * e3), xi * (1 - e1), xi, xi * (1 - e1 + e1 * e2)},
                {xi, xi * e1 * (1 - e2 + e2 * e3), xi * (1 - e1 * e2), xi * e1 * (1 - e2)},
                {xi * (1 - e1 * e2), xi * e1 * (1 - e2), xi, xi * e1 * (1 - e2 + e2 * e3)},
                {xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), xi, xi * e1 * (1 - e2)},
                {xi, xi * e1 * (1 - e2), xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)}};
            for (auto& s : xs) visit(chi(P, s[0], s[1]), chi(Q, s[2], s[3]), w);
          } else if (kind == EDGE) {
            double w0 = w4 * xi * xi * xi * e1 * e1;
            double w1 = w0 * e2;
            visit(chi(P, xi, xi * e1 * e3), chi(Q, xi * (1 - e1 * e2), xi * e1 * (1 - e2)), w0);
            visit(chi(P, xi, xi * e1), chi(Q, xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3)), w1);
            visit(chi(P, xi * (1 - e1 * e2), xi * e1 * (1 - e2)), chi(Q, xi, xi * e1 * e2 * e3), w1);
            visit(chi(P, xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3)), chi(Q, xi, xi * e1), w1);
            visit(chi(P, xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)), chi(Q, xi, xi * e1 * e2), w1);
          } else {  // VERTEX
            double w = w4 * xi * xi * xi * e2;
            visit(chi(P, xi, xi * e1), chi(Q, xi * e2, xi * e2 * e3), w);
            visit(chi(P, xi * e2, xi * e2 * e3), chi(Q, xi, xi * e1), w);
          }
        }
}

// Sauter-Schwab block for an ordered touching pair.
void singular_block(const MeshView& m, const Rules& q, double k, int64_t t1, int64_t t2, PairKind kind,
                    const Vec3 P[3], const Vec3 Q[3], cplx blk[3][3]) {
  LocalRWG f = local_rwg(m, t1), g = local_rwg(m, t2);
  double jac = (2.0 * m.area(t1)) * (2.0 * m.area(t2));
  ss_points(kind, P, Q, q, jac, [&](Vec3 x, Vec3 y, double w) { add_point_pair(k, f, g, x, y, w, blk); });
}

// Classify the ordered pair (t1, t2) and order the vertices for Sauter-Schwab:
//  identical: both in stored order;
//  edge: the shared edge as it runs (a -> b) in t1's cyclic order, then the third
//        vertex, for both triangles;
//  vertex: the shared vertex, then the next two vertices of each triangle's own
//        cyclic order.
PairKind classify(const MeshView& m, int64_t t1, int64_t t2, Vec3 P[3], Vec3 Q[3]) {
  const int32_t* A = m.tris + 3 * t1;
  const int32_t* B = m.tris + 3 * t2;
  if (t1 == t2) {
    for (int i = 0; i < 3; ++i) P[i] = Q[i] = m.v(A[i]);
    return IDENTICAL;
  }
  int inB[3];
  int nshared = 0;
  for (int i = 0; i < 3; ++i) {
    inB[i] = -1;
    for (int j = 0; j < 3; ++j)
      if (A[i] == B[j]) inB[i] = j;
    if (inB[i] >= 0) ++nshared;
  }
  if (nshared == 0) return REGULAR;
  if (nshared == 1) {
    int i = inB[0] >= 0 ? 0 : (inB[1] >= 0 ? 1 : 2);
    int j = inB[i];
    for (int s = 0; s < 3; ++s) {
      P[s] = m.v(A[(i + s) % 3]);
      Q[s] = m.v(B[(j + s) % 3]);
    }
    return VERTEX;
  }
  // edge: find i with A[i], A[i+1] both shared
  int i0 = -1;
  for (int i = 0; i < 3; ++i)
    if (inB[i] >= 0 && inB[(i + 1) % 3] >= 0) i0 = i;
  int a = A[i0], b = A[(i0 + 1) % 3], c1 = A[(i0 + 2) % 3];
  int c2 = -1;
  for (int j = 0; j < 3; ++j)
    if (B[j] != a && B[j] != b) c2 = B[j];
  P[0] = m.v(a); P[1] = m.v(b); P[2] = m.v(c1);
  Q[0] = m.v(a); Q[1] = m.v(b); Q[2] = m.v(c2);
  return EDGE;
}

// Full 3 x 3 block of the ordered triangle pair (t1, t2).
void pair_block(const MeshView& m, const Rules& q, double k, int64_t t1, int64_t t2, cplx blk[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) blk[i][j] = 0.0;
  Vec3 P[3], Q[3];
  PairKind kind = classify(m, t1, t2, P, Q);
  if (kind == REGULAR) {
    regular_block(m, q, k, t1, t2, blk);
    return;
  }
  if (t1 <= t2) {
    singular_block(m, q, k, t1, t2, kind, P, Q, blk);
    return;
  }
  cplx tb[3][3] = {};
  classify(m, t2, t1, P, Q);
  singular_block(m, q, k, t2, t1, kind, P, Q, tb);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) blk[i][j] = tb[j][i];
}

// ---- MFIO blocks for the dielectric (PMCHWT) system of Section II-C -----------------
// K_k = {gamma_D H_k}, H_k v = curl int G v (Section II-B).  Tested with the x-pairing:
//   <K_k f_n, f_m>_x = -int f_m(x) . (curl_x int G(x,y) f_n(y) dy) dx
//                    = -int int (x - y) . (f_n(y) x f_m(x)) G'(r)/r,
//   G'(r)/r = exp(ikr) (ikr - 1) / (4 pi r^3),  r = |x - y|,
// the principal value: on one flat triangle x - y lies in the plane and f_n x f_m is
// normal to it, so identical pairs contribute nothing and need no special rule.
void add_point_pair_mfio(double k, const LocalRWG& f, const LocalRWG& g, Vec3 x, Vec3 y, double w, cplx blk[3][3]) {
  Vec3 d = sub(x, y);
  double r = norm(d);
  cplx gk = std::exp(cplx(0.0, k * r)) * cplx(-1.0, k * r) / (4.0 * M_PI * r * r * r) * w;
  for (int i = 0; i < 3; ++i) {
    Vec3 fi = scale(sub(x, f.opp[i]), f.coef[i]);
    for (int j = 0; j < 3; ++j) {
      Vec3 gj = scale(sub(y, g.opp[j]), g.coef[j]);
      blk[i][j] += -gk * dot(d, cross(gj, fi));
    }
  }
}

// 3 x 3 MFIO block of the ordered triangle pair (t1 test, t2 trial), with the same rules
// as the EFIO blocks (6-point rule in x and y for vertex-disjoint pairs, Sauter-Schwab
// with t1 < t2 and the transpose for touching ones; the block is symmetric under
// exchanging the two triangles, as the EFIO's is).
void pair_block_mfio(const MeshView& m, const Rules& q, double k, int64_t t1, int64_t t2, cplx blk[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) blk[i][j] = 0.0;
  Vec3 P[3], Q[3];
  PairKind kind = classify(m, t1, t2, P, Q);
  if (kind == REGULAR) {
    LocalRWG f = local_rwg(m, t1), g = local_rwg(m, t2);
    double A1 = m.area(t1), A2 = m.area(t2);
    Vec3 a0 = m.tv(t1, 0), a1 = m.tv(t1, 1), a2 = m.tv(t1, 2);
    Vec3 b0 = m.tv(t2, 0), b1 = m.tv(t2, 1), b2 = m.tv(t2, 2);
    for (int p = 0; p < q.nq; ++p) {
      Vec3 x = add(add(scale(a0, q.qb[3 * p]), scale(a1, q.qb[3 * p + 1])), scale(a2, q.qb[3 * p + 2]));
      for (int s = 0; s < q.nq; ++s) {
        Vec3 y = add(add(scale(b0, q.qb[3 * s]), scale(b1, q.qb[3 * s + 1])), scale(b2, q.qb[3 * s + 2]));
        add_point_pair_mfio(k, f, g, x, y, q.qw[p] * A1 * q.qw[s] * A2, blk);
      }
    }
    return;
  }
  int64_t a = t1 < t2 ? t1 : t2, b = t1 < t2 ? t2 : t1;
  if (t1 > t2) classify(m, a, b, P, Q);
  LocalRWG f = local_rwg(m, a), g = local_rwg(m, b);
  double jac = (2.0 * m.area(a)) * (2.0 * m.area(b));
  cplx tb[3][3] = {};
  ss_points(kind, P, Q, q, jac, [&](Vec3 x, Vec3 y, double w) { add_point_pair_mfio(k, f, g, x, y, w, tb); });
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) blk[i][j] = t1 <= t2 ? tb[i][j] : tb[j][i];
}

}  // namespace

extern "C" {

// Dense Z (N x N, row-major, interleaved complex) for all triangle pairs.
int orc_assemble_z(const double* verts, const int32_t* tris, int64_t nt, const int32_t* tri_edge,
                   const double* tri_sign, const double* edge_len, int64_t n_edges, double k,
                   const double* qb, const double* qw, int nq, const double* glx, const double* glw, int nss,
                   double* Z, int nthreads) {
  MeshView m{verts, tris, nt, tri_edge, tri_sign, edge_len};
  Rules q{qb, qw, nq, glx, glw, nss};
  std::memset(Z, 0, sizeof(double) * 2 * n_edges * n_edges);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t t1 = 0; t1 < nt; ++t1) {
    for (int64_t t2 = 0; t2 < nt; ++t2) {
      cplx blk[3][3];
      pair_block(m, q, k, t1, t2, blk);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          int64_t idx = 2 * (int64_t(tri_edge[3 * t1 + i]) * n_edges + tri_edge[3 * t2 + j]);
#ifdef _OPENMP
#pragma omp atomic
#endif
          Z[idx] += blk[i][j].real();
#ifdef _OPENMP
#pragma omp atomic
#endif
          Z[idx + 1] += blk[i][j].imag();
        }
    }
  }
  return 0;
}

// Selected entries Z[rows[e], cols[e]]: sum of the four triangle-pair blocks.
int orc_z_entries(const double* verts, const int32_t* tris, int64_t nt, const int32_t* tri_edge,
                  const double* tri_sign, const double* edge_len, const int32_t* edge_tris /*N x 2: T+, T-*/,
                  double k, const double* qb, const double* qw, int nq, const double* glx, const double* glw,
                  int nss, const int64_t* rows, const int64_t* cols, int64_t count, double* out, int nthreads) {
  MeshView m{verts, tris, nt, tri_edge, tri_sign, edge_len};
  Rules q{qb, qw, nq, glx, glw, nss};
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t e = 0; e < count; ++e) {
    cplx acc = 0.0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        int64_t t1 = edge_tris[2 * rows[e] + a], t2 = edge_tris[2 * cols[e] + b];
        int i = -1, j = -1;
        for (int s = 0; s < 3; ++s) {
          if (tri_edge[3 * t1 + s] == rows[e]) i = s;
          if (tri_edge[3 * t2 + s] == cols[e]) j = s;
        }
        cplx blk[3][3];
        pair_block(m, q, k, t1, t2, blk);
        acc += blk[i][j];
      }
    out[2 * e] = acc.real();
    out[2 * e + 1] = acc.imag();
  }
  return 0;
}

// Plane-wave right-hand sides b[m, s] = - int E_inc_s . f_m (N x n_inc, interleaved).
// inc: n_inc x 9 = d (3), Re p (3), Im p (3).
int orc_rhs(const double* verts, const int32_t* tris, int64_t nt, const int32_t* tri_edge,
            const double* tri_sign, const double* edge_len, int64_t n_edges, double k, const double* qb,
            const double* qw, int nq, const double* inc, int64_t n_inc, double* b) {
  MeshView m{verts, tris, nt, tri_edge, tri_sign, edge_len};
  std::memset(b, 0, sizeof(double) * 2 * n_edges * n_inc);
  for (int64_t t = 0; t < nt; ++t) {
    LocalRWG f = local_rwg(m, t);
    double A = m.area(t);
    Vec3 a0 = m.tv(t, 0), a1 = m.tv(t, 1), a2 = m.tv(t, 2);
    for (int64_t s = 0; s < n_inc; ++s) {
      const double* c = inc + 9 * s;
      Vec3 d{c[0], c[1], c[2]};
      cplx p[3] = {cplx(c[3], c[6]), cplx(c[4], c[7]), cplx(c[5], c[8])};
      for (int qp = 0; qp < nq; ++qp) {
        Vec3 x = add(add(scale(a0, qb[3 * qp]), scale(a1, qb[3 * qp + 1])), scale(a2, qb[3 * qp + 2]));
        cplx ph = std::exp(cplx(0.0, k * dot(d, x)));
        for (int i = 0; i < 3; ++i) {
          Vec3 fi = scale(sub(x, f.opp[i]), f.coef[i]);
          cplx e_dot_f = (p[0] * fi.x + p[1] * fi.y + p[2] * fi.z) * ph;
          int64_t idx = 2 * (int64_t(tri_edge[3 * t + i]) * n_inc + s);
          cplx v = -e_dot_f * (qw[qp] * A);
          b[idx] += v.real();
          b[idx + 1] += v.imag();
        }
      }
    }
  }
  return 0;
}

// Far-field matrix A[(d*3 + c), n] = -ik [(I - xh xh^T) int f_n(y) exp(-ik xh.y) dy]_c.
int orc_farfield_matrix(const double* verts, const int32_t* tris, int64_t nt, const int32_t* tri_edge,
                        const double* tri_sign, const double* edge_len, int64_t n_edges, double k,
                        const double* qb, const double* qw, int nq, const double* xh, int64_t n_dir, double* Aout) {
  MeshView m{verts, tris, nt, tri_edge, tri_sign, edge_len};
  std::memset(Aout, 0, sizeof(double) * 2 * 3 * n_dir * n_edges);
  const cplx ik(0.0, k);
  for (int64_t t = 0; t < nt; ++t) {
    LocalRWG f = local_rwg(m, t);
    double A = m.area(t);
    Vec3 a0 = m.tv(t, 0), a1 = m.tv(t, 1), a2 = m.tv(t, 2);
    for (int64_t dd = 0; dd < n_dir; ++dd) {
      Vec3 u{xh[3 * dd], xh[3 * dd + 1], xh[3 * dd + 2]};
      for (int i = 0; i < 3; ++i) {
        cplx J[3] = {0.0, 0.0, 0.0};
        for (int qp = 0; qp < nq; ++qp) {
          Vec3 y = add(add(scale(a0, qb[3 * qp]), scale(a1, qb[3 * qp + 1])), scale(a2, qb[3 * qp + 2]));
          cplx ph = std::exp(cplx(0.0, -k * dot(u, y))) * (qw[qp] * A);
          Vec3 fi = scale(sub(y, f.opp[i]), f.coef[i]);
          J[0] += fi.x * ph;
          J[1] += fi.y * ph;
          J[2] += fi.z * ph;
        }
        cplx uJ = u.x * J[0] + u.y * J[1] + u.z * J[2];
        cplx T[3] = {J[0] - u.x * uJ, J[1] - u.y * uJ, J[2] - u.z * uJ};
        int64_t n = tri_edge[3 * t + i];
        for (int c = 0; c < 3; ++c) {
          cplx v = -ik * T[c];
          int64_t idx = 2 * ((3 * dd + c) * n_edges + n);
          Aout[idx] += v.real();
          Aout[idx + 1] += v.imag();
        }
      }
    }
  }
  return 0;
}

// Shape-derivative right-hand side as triplets: for every triangle t, local edge i
// and local vertex a, vals[t*9 + i*3 + a] is the contribution to B[tri_edge[t,i], tris[t,a]]:
//   B_mp = - sum_n u_n int_T psi_p nu_{p,T} [ ik f_m.f_n + 1/(ik) div f_m div f_n ].
// vnormals: V x 3 unit vertex normals n_p.
int orc_sd_rhs(const double* verts, const int32_t* tris, int64_t nt, const int32_t* tri_edge,
               const double* tri_sign, const double* edge_len, double k, const double* qb, const double* qw,
               int nq, const double* vnormals, const double* u /*N complex*/, double* vals /*T x 9 complex*/) {
  MeshView m{verts, tris, nt, tri_edge, tri_sign, edge_len};
  const cplx ik(0.0, k);
  for (int64_t t = 0; t < nt; ++t) {
    LocalRWG f = local_rwg(m, t);
    double A = m.area(t);
    Vec3 nT = m.unit_normal(t);
    Vec3 a0 = m.tv(t, 0), a1 = m.tv(t, 1), a2 = m.tv(t, 2);
    cplx un[3];
    for (int j = 0; j < 3; ++j) {
      int64_t n = tri_edge[3 * t + j];
      un[j] = cplx(u[2 * n], u[2 * n + 1]);
    }
    double nu[3];
    for (int a = 0; a < 3; ++a) {
      int32_t p = tris[3 * t + a];
      nu[a] = vnormals[3 * p] * nT.x + vnormals[3 * p + 1] * nT.y + vnormals[3 * p + 2] * nT.z;
    }
    cplx acc[3][3] = {};
    for (int qp = 0; qp < nq; ++qp) {
      double lam[3] = {qb[3 * qp], qb[3 * qp + 1], qb[3 * qp + 2]};
      Vec3 x = add(add(scale(a0, lam[0]), scale(a1, lam[1])), scale(a2, lam[2]));
      double w = qw[qp] * A;
      for (int i = 0; i < 3; ++i) {
        Vec3 fi = scale(sub(x, f.opp[i]), f.coef[i]);
        cplx s = 0.0;
        for (int j = 0; j < 3; ++j) {
          Vec3 fj = scale(sub(x, f.opp[j]), f.coef[j]);
          s += un[j] * (ik * dot(fi, fj) + f.div[i] * f.div[j] / ik);
        }
        for (int a = 0; a < 3; ++a) acc[i][a] += -s * (w * lam[a] * nu[a]);
      }
    }
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 3; ++a) {
        vals[2 * (9 * t + 3 * i + a)] = acc[i][a].real();
        vals[2 * (9 * t + 3 * i + a) + 1] = acc[i][a].imag();
      }
  }
  return 0;
}

// Galerkin matrix of the PMCHWT operator A_0 + A^_1 (Section II-C eq. pmchwt, with the
// multitrace operators of eq. BOmultitraceA) for the exterior Cauchy data (j, m):
//   Z (2N x 2N) = [[ K_0 + K_1,        T_0 + eta T_1 ],
//                  [ -T_0 - T_1 / eta,  K_0 + K_1     ]],
// T_k the EFIO blocks above, K_k the MFIO blocks, k = k0 outside and k1 inside.
int orc_assemble_pmchwt(const double* verts, const int32_t* tris, int64_t nt, const int32_t* tri_edge,
                        const double* tri_sign, const double* edge_len, int64_t n_edges, double k0, double k1,
                        double eta, const double* qb, const double* qw, int nq, const double* glx, const double* glw,
                        int nss, double* Z, int nthreads) {
  MeshView m{verts, tris, nt, tri_edge, tri_sign, edge_len};
  Rules q{qb, qw, nq, glx, glw, nss};
  const int64_t N = n_edges, ld = 2 * n_edges;
  std::memset(Z, 0, sizeof(double) * 2 * ld * ld);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t t1 = 0; t1 < nt; ++t1) {
    for (int64_t t2 = 0; t2 < nt; ++t2) {
      cplx T0[3][3], T1[3][3], K0[3][3], K1[3][3];
      pair_block(m, q, k0, t1, t2, T0);
      pair_block(m, q, k1, t1, t2, T1);
      pair_block_mfio(m, q, k0, t1, t2, K0);
      pair_block_mfio(m, q, k1, t1, t2, K1);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          const int64_t r = tri_edge[3 * t1 + i], c = tri_edge[3 * t2 + j];
          const cplx kk = K0[i][j] + K1[i][j];
          const cplx v[4] = {kk, T0[i][j] + eta * T1[i][j], -T0[i][j] - T1[i][j] / eta, kk};
          const int64_t idx[4] = {r * ld + c, r * ld + N + c, (N + r) * ld + c, (N + r) * ld + N + c};
          for (int e = 0; e < 4; ++e) {
#ifdef _OPENMP
#pragma omp atomic
#endif
            Z[2 * idx[e]] += v[e].real();
#ifdef _OPENMP
#pragma omp atomic
#endif
            Z[2 * idx[e] + 1] += v[e].imag();
          }
        }
    }
  }
  return 0;
}

// MFIO matrix alone, <K_k f_n, f_m>_x (N x N), for the oracle's own pins.
int orc_assemble_mfio(const double* verts, const int32_t* tris, int64_t nt, const int32_t* tri_edge,
                      const double* tri_sign, const double* edge_len, int64_t n_edges, double k, const double* qb,
                      const double* qw, int nq, const double* glx, const double* glw, int nss, double* K,
                      int nthreads) {
  MeshView m{verts, tris, nt, tri_edge, tri_sign, edge_len};
  Rules q{qb, qw, nq, glx, glw, nss};
  std::memset(K, 0, sizeof(double) * 2 * n_edges * n_edges);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t t1 = 0; t1 < nt; ++t1) {
    for (int64_t t2 = 0; t2 < nt; ++t2) {
      cplx blk[3][3];
      pair_block_mfio(m, q, k, t1, t2, blk);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          int64_t idx = 2 * (int64_t(tri_edge[3 * t1 + i]) * n_edges + tri_edge[3 * t2 + j]);
#ifdef _OPENMP
#pragma omp atomic
#endif
          K[idx] += blk[i][j].real();
#ifdef _OPENMP
#pragma omp atomic
#endif
          K[idx + 1] += blk[i][j].imag();
        }
    }
  }
  return 0;
}

// Selected entries Z[rows[e], cols[e]] of the 2N x 2N PMCHWT matrix (orc_assemble_pmchwt),
// each from the four triangle-pair blocks of its two edges, for large-N parity samples.
int orc_pmchwt_entries(const double* verts, const int32_t* tris, int64_t nt, const int32_t* tri_edge,
                       const double* tri_sign, const double* edge_len, const int32_t* edge_tris, int64_t n_edges,
                       double k0, double k1, double eta, const double* qb, const double* qw, int nq,
                       const double* glx, const double* glw, int nss, const int64_t* rows, const int64_t* cols,
                       int64_t count, double* out, int nthreads) {
  MeshView m{verts, tris, nt, tri_edge, tri_sign, edge_len};
  Rules q{qb, qw, nq, glx, glw, nss};
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t e = 0; e < count; ++e) {
    const int br = rows[e] >= n_edges, bc = cols[e] >= n_edges;
    const int64_t r = rows[e] - br * n_edges, c = cols[e] - bc * n_edges;
    cplx T0 = 0.0, T1 = 0.0, K0 = 0.0, K1 = 0.0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        int64_t t1 = edge_tris[2 * r + a], t2 = edge_tris[2 * c + b];
        int i = -1, j = -1;
        for (int s = 0; s < 3; ++s) {
          if (tri_edge[3 * t1 + s] == r) i = s;
          if (tri_edge[3 * t2 + s] == c) j = s;
        }
        cplx blk[3][3];
        if (br == bc) {
          pair_block_mfio(m, q, k0, t1, t2, blk);
          K0 += blk[i][j];
          pair_block_mfio(m, q, k1, t1, t2, blk);
          K1 += blk[i][j];
        } else {
          pair_block(m, q, k0, t1, t2, blk);
          T0 += blk[i][j];
          pair_block(m, q, k1, t1, t2, blk);
          T1 += blk[i][j];
        }
      }
    cplx v = br == bc ? K0 + K1 : (br == 0 ? T0 + eta * T1 : -T0 - T1 / eta);
    out[2 * e] = v.real();
    out[2 * e + 1] = v.imag();
  }
  return 0;
}

// One 3 x 3 MFIO block (t1 test, t2 trial) for the oracle's pins.
int orc_mfio_block(const double* verts, const int32_t* tris, int64_t nt, const int32_t* tri_edge,
                   const double* tri_sign, const double* edge_len, double k, const double* qb, const double* qw, int nq,
                   const double* glx, const double* glw, int nss, int64_t t1, int64_t t2, double* out) {
  MeshView m{verts, tris, nt, tri_edge, tri_sign, edge_len};
  Rules q{qb, qw, nq, glx, glw, nss};
  cplx blk[3][3];
  pair_block_mfio(m, q, k, t1, t2, blk);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      out[2 * (3 * i + j)] = blk[i][j].real();
      out[2 * (3 * i + j) + 1] = blk[i][j].imag();
    }
  return 0;
}

// Far-field matrix of the dielectric problem (3 n_dir x 2N) for the exterior Cauchy data
// (j, m): the scattered field outside is E_sc = -E_k m - H_k j (Section II-C, the
// representation E = E_inc + R(xi) with R = (-H, -E)), so with v_n = int f_n(y) exp(-ik xh.y) dy
//   F(xh) = -ik [ xh x sum_n j_n v_n + (I - xh xh^T) sum_n m_n v_n ].
int orc_farfield_matrix_pmchwt(const double* verts, const int32_t* tris, int64_t nt, const int32_t* tri_edge,
                               const double* tri_sign, const double* edge_len, int64_t n_edges, double k,
                               const double* qb, const double* qw, int nq, const double* xh, int64_t n_dir,
                               double* Aout) {
  MeshView m{verts, tris, nt, tri_edge, tri_sign, edge_len};
  const int64_t ld = 2 * n_edges;
  std::memset(Aout, 0, sizeof(double) * 2 * 3 * n_dir * ld);
  const cplx ik(0.0, k);
  for (int64_t t = 0; t < nt; ++t) {
    LocalRWG f = local_rwg(m, t);
    double A = m.area(t);
    Vec3 a0 = m.tv(t, 0), a1 = m.tv(t, 1), a2 = m.tv(t, 2);
    for (int64_t dd = 0; dd < n_dir; ++dd) {
      Vec3 u{xh[3 * dd], xh[3 * dd + 1], xh[3 * dd + 2]};
      for (int i = 0; i < 3; ++i) {
        cplx J[3] = {0.0, 0.0, 0.0};
        for (int qp = 0; qp < nq; ++qp) {
          Vec3 y = add(add(scale(a0, qb[3 * qp]), scale(a1, qb[3 * qp + 1])), scale(a2, qb[3 * qp + 2]));
          cplx ph = std::exp(cplx(0.0, -k * dot(u, y))) * (qw[qp] * A);
          Vec3 fi = scale(sub(y, f.opp[i]), f.coef[i]);
          J[0] += fi.x * ph;
          J[1] += fi.y * ph;
          J[2] += fi.z * ph;
        }
        cplx uJ = u.x * J[0] + u.y * J[1] + u.z * J[2];
        cplx Tm[3] = {J[0] - u.x * uJ, J[1] - u.y * uJ, J[2] - u.z * uJ};
        cplx Xj[3] = {u.y * J[2] - u.z * J[1], u.z * J[0] - u.x * J[2], u.x * J[1] - u.y * J[0]};
        int64_t n = tri_edge[3 * t + i];
        for (int c = 0; c < 3; ++c) {
          cplx vj = -ik * Xj[c], vm = -ik * Tm[c];
          int64_t row = (3 * dd + c) * ld;
          Aout[2 * (row + n)] += vj.real();
          Aout[2 * (row + n) + 1] += vj.imag();
          Aout[2 * (row + n_edges + n)] += vm.real();
          Aout[2 * (row + n_edges + n) + 1] += vm.imag();
        }
      }
    }
  }
  return 0;
}

// Sauter-Schwab integral of a scalar test kernel over a touching pair (the same point
// generator as the assembly), used by the oracle's pins:
//   kernel 0: 1,  1: 1/|x-y|,  2: x.y
double orc_ss_integral(const double* P9, const double* Q9, int kind, const double* glx, const double* glw,
                       int nss, int kernel) {
  Vec3 P[3] = {{P9[0], P9[1], P9[2]}, {P9[3], P9[4], P9[5]}, {P9[6], P9[7], P9[8]}};
  Vec3 Q[3] = {{Q9[0], Q9[1], Q9[2]}, {Q9[3], Q9[4], Q9[5]}, {Q9[6], Q9[7], Q9[8]}};
  double A1 = 0.5 * norm(cross(sub(P[1], P[0]), sub(P[2], P[0])));
  double A2 = 0.5 * norm(cross(sub(Q[1], Q[0]), sub(Q[2], Q[0])));
  Rules q{nullptr, nullptr, 0, glx, glw, nss};
  double sum = 0.0;
  ss_points(PairKind(kind), P, Q, q, 4.0 * A1 * A2, [&](Vec3 x, Vec3 y, double w) {
    double v = kernel == 0 ? 1.0 : (kernel == 1 ? 1.0 / norm(sub(x, y)) : dot(x, y));
    sum += w * v;
  });
  return sum;
}

}  // extern "C"
