// FP64 CPU oracle for shape derivatives of the DISCRETE EFIE quantities with respect
// to one vertex coordinate X_{p,c}: (dZ/dX_pc) u, db/dX_pc and (dA/dX_pc) u.
//
// TEST INFRASTRUCTURE ONLY (see efie_oracle.cpp).  Forward-mode differentiation with
// dual numbers (value, derivative) of exactly the quadrature sums the oracle uses for
// Z, b and the far-field matrix (6-point rule on regular pairs, Sauter-Schwab on
// touching pairs, same vertex orderings): quadrature points, areas, edge lengths and
// opposite vertices all move with the seeded vertex, the reference weights do not.
// Only triangles that contain vertex p contribute.
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

struct D {  // dual number v + d eps
  double v, d;
};
inline D operator+(D a, D b) { return {a.v + b.v, a.d + b.d}; }
inline D operator-(D a, D b) { return {a.v - b.v, a.d - b.d}; }
inline D operator-(D a) { return {-a.v, -a.d}; }
inline D operator*(D a, D b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline D operator*(D a, double s) { return {a.v * s, a.d * s}; }
inline D operator*(double s, D a) { return {a.v * s, a.d * s}; }
inline D operator/(D a, D b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
inline D dsqrt(D a) {
  double s = std::sqrt(a.v);
  return {s, a.d / (2.0 * s)};
}
inline D dsin(D a) { return {std::sin(a.v), std::cos(a.v) * a.d}; }
inline D dcos(D a) { return {std::cos(a.v), -std::sin(a.v) * a.d}; }

struct CD {  // complex number with dual parts
  D re, im;
};
inline CD operator+(CD a, CD b) { return {a.re + b.re, a.im + b.im}; }
inline CD operator-(CD a, CD b) { return {a.re - b.re, a.im - b.im}; }
inline CD operator*(CD a, CD b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline CD operator*(CD a, D s) { return {a.re * s, a.im * s}; }
inline CD cmul_const(CD a, std::complex<double> z) {
  return {a.re * z.real() - a.im * z.imag(), a.re * z.imag() + a.im * z.real()};
}
inline CD expi(D t) { return {dcos(t), dsin(t)}; }  // exp(i t)

struct V3 {
  D x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(V3 a, D s) { return {a.x * s, a.y * s, a.z * s}; }
inline V3 operator*(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline D dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline D nrm(V3 a) { return dsqrt(dot(a, a)); }

struct Mesh {
  const double* verts;
  const int32_t* tris;
  int64_t nt;
  const int32_t* tri_edge;
  const double* tri_sign;
  int32_t seed_vertex;
  int seed_coord;
  V3 v(int32_t i) const {
    V3 r{{verts[3 * i], 0.0}, {verts[3 * i + 1], 0.0}, {verts[3 * i + 2], 0.0}};
    if (i == seed_vertex) (seed_coord == 0 ? r.x : seed_coord == 1 ? r.y : r.z).d = 1.0;
    return r;
  }
  V3 tv(int64_t t, int a) const { return v(tris[3 * t + a]); }
  D area(int64_t t) const { return nrm(cross(tv(t, 1) - tv(t, 0), tv(t, 2) - tv(t, 0))) * 0.5; }
  bool has_seed(int64_t t) const {
    return tris[3 * t] == seed_vertex || tris[3 * t + 1] == seed_vertex || tris[3 * t + 2] == seed_vertex;
  }
};

struct Rules {
  const double* qb;
  const double* qw;
  int nq;
  const double* glx;
  const double* glw;
  int nss;
};

struct Local {
  V3 opp[3];
  D coef[3];  // s l / (2A)
  D div[3];   // s l / A
};

Local local(const Mesh& m, int64_t t) {
  Local r;
  D A = m.area(t);
  for (int i = 0; i < 3; ++i) {
    V3 a = m.tv(t, (i + 1) % 3), b = m.tv(t, (i + 2) % 3);
    D l = nrm(b - a);
    double s = m.tri_sign[3 * t + i];
    r.opp[i] = m.tv(t, i);
    r.coef[i] = l * s / (A * 2.0);
    r.div[i] = l * s / A;
  }
  return r;
}

void add_pp(double k, const Local& f, const Local& g, V3 x, V3 y, D w, CD blk[3][3]) {
  D r = nrm(x - y);
  D scale = w / (r * (4.0 * M_PI));
  CD G = expi(r * k) * scale;
  const std::complex<double> mik(0.0, -k), minv(0.0, 1.0 / k);  // -ik and -1/(ik) = i/k
  for (int i = 0; i < 3; ++i) {
    V3 fi = (x - f.opp[i]) * f.coef[i];
    for (int j = 0; j < 3; ++j) {
      V3 gj = (y - g.opp[j]) * g.coef[j];
      CD t1 = cmul_const(G * dot(fi, gj), mik);
      CD t2 = cmul_const(G * (f.div[i] * g.div[j]), minv);
      blk[i][j] = blk[i][j] + t1 + t2;
    }
  }
}

inline V3 chi(const V3 P[3], double u1, double u2) { return P[0] + (P[1] - P[0]) * u1 + (P[2] - P[1]) * u2; }

enum Kind { REG = 0, VTX = 1, EDG = 2, IDN = 3 };

template <class Visit>
void ss_points(Kind kind, const V3 P[3], const V3 Q[3], const Rules& q, D jac, Visit&& visit) {
  const int n = q.nss;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < n; ++c)
        for (int d = 0; d < n; ++d) {
          double xi = q.glx[a], e1 = q.glx[b], e2 = q.glx[c], e3 = q.glx[d];
          D w4 = jac * (q.glw[a] * q.glw[b] * q.glw[c] * q.glw[d]);
          if (kind == IDN) {
            D w = w4 * (xi * xi * xi * e1 * e1 * e2);
            double xs[6][4] = {
                {xi, xi * (1 - e1 + e1 * e2), xi * (1 - e1 * e2 * e3), xi * (1 - e1)},
                {xi * (1 - e1 * e2 * e3), xi * (1 - e1), xi, xi * (1 - e1 + e1 * e2)},
                {xi, xi * e1 * (1 - e2 + e2 * e3), xi * (1 - e1 * e2), xi * e1 * (1 - e2)},
                {xi * (1 - e1 * e2), xi * e1 * (1 - e2), xi, xi * e1 * (1 - e2 + e2 * e3)},
                {xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), xi, xi * e1 * (1 - e2)},
                {xi, xi * e1 * (1 - e2), xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)}};
            for (auto& s : xs) visit(chi(P, s[0], s[1]), chi(Q, s[2], s[3]), w);
          } else if (kind == EDG) {
            D w0 = w4 * (xi * xi * xi * e1 * e1);
            D w1 = w0 * e2;
            visit(chi(P, xi, xi * e1 * e3), chi(Q, xi * (1 - e1 * e2), xi * e1 * (1 - e2)), w0);
            visit(chi(P, xi, xi * e1), chi(Q, xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3)), w1);
            visit(chi(P, xi * (1 - e1 * e2), xi * e1 * (1 - e2)), chi(Q, xi, xi * e1 * e2 * e3), w1);
            visit(chi(P, xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3)), chi(Q, xi, xi * e1), w1);
            visit(chi(P, xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)), chi(Q, xi, xi * e1 * e2), w1);
          } else {
            D w = w4 * (xi * xi * xi * e2);
            visit(chi(P, xi, xi * e1), chi(Q, xi * e2, xi * e2 * e3), w);
            visit(chi(P, xi * e2, xi * e2 * e3), chi(Q, xi, xi * e1), w);
          }
        }
}

Kind classify(const Mesh& m, int64_t t1, int64_t t2, V3 P[3], V3 Q[3]) {
  const int32_t* A = m.tris + 3 * t1;
  const int32_t* B = m.tris + 3 * t2;
  if (t1 == t2) {
    for (int i = 0; i < 3; ++i) P[i] = Q[i] = m.v(A[i]);
    return IDN;
  }
  int inB[3], ns = 0;
  for (int i = 0; i < 3; ++i) {
    inB[i] = -1;
    for (int j = 0; j < 3; ++j)
      if (A[i] == B[j]) inB[i] = j;
    ns += inB[i] >= 0;
  }
  if (ns == 0) return REG;
  if (ns == 1) {
    int i = inB[0] >= 0 ? 0 : (inB[1] >= 0 ? 1 : 2), j = inB[i];
    for (int s = 0; s < 3; ++s) {
      P[s] = m.v(A[(i + s) % 3]);
      Q[s] = m.v(B[(j + s) % 3]);
    }
    return VTX;
  }
  int i0 = 0;
  for (int i = 0; i < 3; ++i)
    if (inB[i] >= 0 && inB[(i + 1) % 3] >= 0) i0 = i;
  int a = A[i0], b = A[(i0 + 1) % 3], c1 = A[(i0 + 2) % 3], c2 = -1;
  for (int j = 0; j < 3; ++j)
    if (B[j] != a && B[j] != b) c2 = B[j];
  P[0] = m.v(a); P[1] = m.v(b); P[2] = m.v(c1);
  Q[0] = m.v(a); Q[1] = m.v(b); Q[2] = m.v(c2);
  return EDG;
}

void pair_block(const Mesh& m, const Rules& q, double k, int64_t t1, int64_t t2, CD blk[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) blk[i][j] = CD{{0, 0}, {0, 0}};
  V3 P[3], Q[3];
  Kind kind = classify(m, t1, t2, P, Q);
  if (kind == REG) {
    Local f = local(m, t1), g = local(m, t2);
    D A1 = m.area(t1), A2 = m.area(t2);
    V3 a0 = m.tv(t1, 0), a1 = m.tv(t1, 1), a2 = m.tv(t1, 2);
    V3 b0 = m.tv(t2, 0), b1 = m.tv(t2, 1), b2 = m.tv(t2, 2);
    for (int p = 0; p < q.nq; ++p) {
      V3 x = a0 * q.qb[3 * p] + a1 * q.qb[3 * p + 1] + a2 * q.qb[3 * p + 2];
      for (int s = 0; s < q.nq; ++s) {
        V3 y = b0 * q.qb[3 * s] + b1 * q.qb[3 * s + 1] + b2 * q.qb[3 * s + 2];
        add_pp(k, f, g, x, y, A1 * A2 * (q.qw[p] * q.qw[s]), blk);
      }
    }
    return;
  }
  if (t1 <= t2) {
    Local f = local(m, t1), g = local(m, t2);
    D jac = m.area(t1) * m.area(t2) * 4.0;
    ss_points(kind, P, Q, q, jac, [&](V3 x, V3 y, D w) { add_pp(k, f, g, x, y, w, blk); });
    return;
  }
  CD tb[3][3];
  pair_block(m, q, k, t2, t1, tb);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) blk[i][j] = tb[j][i];
}

}  // namespace

extern "C" {

// out[m] = sum_n (dZ_mn / dX_{p,c}) u_n  (N complex, interleaved).
int orc_grad_dz_u(const double* verts, const int32_t* tris, int64_t nt, const int32_t* tri_edge,
                  const double* tri_sign, int64_t n_edges, double k, const double* qb, const double* qw, int nq,
                  const double* glx, const double* glw, int nss, int32_t p, int c, const double* u, double* out) {
  Mesh m{verts, tris, nt, tri_edge, tri_sign, p, c};
  Rules q{qb, qw, nq, glx, glw, nss};
  std::memset(out, 0, sizeof(double) * 2 * n_edges);
  std::vector<int64_t> seeded;
  for (int64_t t = 0; t < nt; ++t)
    if (m.has_seed(t)) seeded.push_back(t);
  auto accumulate = [&](int64_t t1, int64_t t2) {
    CD blk[3][3];
    pair_block(m, q, k, t1, t2, blk);
    for (int i = 0; i < 3; ++i) {
      int64_t row = tri_edge[3 * t1 + i];
      for (int j = 0; j < 3; ++j) {
        int64_t col = tri_edge[3 * t2 + j];
        double ur = u[2 * col], ui = u[2 * col + 1];
        out[2 * row] += blk[i][j].re.d * ur - blk[i][j].im.d * ui;
        out[2 * row + 1] += blk[i][j].re.d * ui + blk[i][j].im.d * ur;
      }
    }
  };
  for (int64_t t1 : seeded)
    for (int64_t t2 = 0; t2 < nt; ++t2) accumulate(t1, t2);
  for (int64_t t1 = 0; t1 < nt; ++t1)
    if (!m.has_seed(t1))
      for (int64_t t2 : seeded) accumulate(t1, t2);
  return 0;
}

// out (N x n_inc) = db / dX_{p,c}, b[m, s] = -int E_inc_s . f_m (inc rows: d, Re p, Im p).
int orc_grad_db(const double* verts, const int32_t* tris, int64_t nt, const int32_t* tri_edge,
                const double* tri_sign, int64_t n_edges, double k, const double* qb, const double* qw, int nq,
                int32_t p, int c, const double* inc, int64_t n_inc, double* out) {
  Mesh m{verts, tris, nt, tri_edge, tri_sign, p, c};
  std::memset(out, 0, sizeof(double) * 2 * n_edges * n_inc);
  for (int64_t t = 0; t < nt; ++t) {
    if (!m.has_seed(t)) continue;
    Local f = local(m, t);
    D A = m.area(t);
    V3 a0 = m.tv(t, 0), a1 = m.tv(t, 1), a2 = m.tv(t, 2);
    for (int64_t s = 0; s < n_inc; ++s) {
      const double* cc = inc + 9 * s;
      for (int qp = 0; qp < nq; ++qp) {
        V3 x = a0 * qb[3 * qp] + a1 * qb[3 * qp + 1] + a2 * qb[3 * qp + 2];
        D phase = (x.x * cc[0] + x.y * cc[1] + x.z * cc[2]) * k;
        CD ph = expi(phase);
        for (int i = 0; i < 3; ++i) {
          V3 fi = (x - f.opp[i]) * f.coef[i];
          CD pf = {fi.x * cc[3] + fi.y * cc[4] + fi.z * cc[5], fi.x * cc[6] + fi.y * cc[7] + fi.z * cc[8]};
          CD v = pf * ph * (A * (-qw[qp]));
          int64_t idx = 2 * (int64_t(tri_edge[3 * t + i]) * n_inc + s);
          out[idx] += v.re.d;
          out[idx + 1] += v.im.d;
        }
      }
    }
  }
  return 0;
}

// out (3 n_dir x ncols) = (dA / dX_{p,c}) U, U (N x ncols complex),
// A[3d + c', n] = -ik [(I - xh xh^T) int f_n exp(-ik xh . y) dy]_c'.
int orc_grad_da_u(const double* verts, const int32_t* tris, int64_t nt, const int32_t* tri_edge,
                  const double* tri_sign, int64_t n_edges, double k, const double* qb, const double* qw, int nq,
                  int32_t p, int c, const double* xh, int64_t n_dir, const double* U, int64_t ncols, double* out) {
  Mesh m{verts, tris, nt, tri_edge, tri_sign, p, c};
  std::memset(out, 0, sizeof(double) * 2 * 3 * n_dir * ncols);
  for (int64_t t = 0; t < nt; ++t) {
    if (!m.has_seed(t)) continue;
    Local f = local(m, t);
    D A = m.area(t);
    V3 a0 = m.tv(t, 0), a1 = m.tv(t, 1), a2 = m.tv(t, 2);
    for (int64_t dd = 0; dd < n_dir; ++dd) {
      double u3[3] = {xh[3 * dd], xh[3 * dd + 1], xh[3 * dd + 2]};
      for (int i = 0; i < 3; ++i) {
        CD J[3] = {};
        for (int a = 0; a < 3; ++a) J[a] = CD{{0, 0}, {0, 0}};
        for (int qp = 0; qp < nq; ++qp) {
          V3 y = a0 * qb[3 * qp] + a1 * qb[3 * qp + 1] + a2 * qb[3 * qp + 2];
          D phase = (y.x * u3[0] + y.y * u3[1] + y.z * u3[2]) * (-k);
          CD ph = expi(phase) * (A * qw[qp]);
          V3 fi = (y - f.opp[i]) * f.coef[i];
          J[0] = J[0] + ph * fi.x;
          J[1] = J[1] + ph * fi.y;
          J[2] = J[2] + ph * fi.z;
        }
        CD uJ = J[0] * D{u3[0], 0} + J[1] * D{u3[1], 0} + J[2] * D{u3[2], 0};
        int64_t n = tri_edge[3 * t + i];
        for (int cc = 0; cc < 3; ++cc) {
          CD T = J[cc] - uJ * D{u3[cc], 0};
          CD a = cmul_const(T, std::complex<double>(0.0, -k));
          for (int64_t col = 0; col < ncols; ++col) {
            double ur = U[2 * (n * ncols + col)], ui = U[2 * (n * ncols + col) + 1];
            int64_t idx = 2 * ((3 * dd + cc) * ncols + col);
            out[idx] += a.re.d * ur - a.im.d * ui;
            out[idx + 1] += a.re.d * ui + a.im.d * ur;
          }
        }
      }
    }
  }
  return 0;
}

// Value check: the dual-number pair blocks' value parts assembled into Z (must equal
// orc_assemble_z up to rounding).  Used by a pin of this file.
int orc_grad_value_z(const double* verts, const int32_t* tris, int64_t nt, const int32_t* tri_edge,
                     const double* tri_sign, int64_t n_edges, double k, const double* qb, const double* qw, int nq,
                     const double* glx, const double* glw, int nss, double* Z) {
  Mesh m{verts, tris, nt, tri_edge, tri_sign, -1, 0};
  Rules q{qb, qw, nq, glx, glw, nss};
  std::memset(Z, 0, sizeof(double) * 2 * n_edges * n_edges);
  for (int64_t t1 = 0; t1 < nt; ++t1)
    for (int64_t t2 = 0; t2 < nt; ++t2) {
      CD blk[3][3];
      pair_block(m, q, k, t1, t2, blk);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          int64_t idx = 2 * (int64_t(tri_edge[3 * t1 + i]) * n_edges + tri_edge[3 * t2 + j]);
          Z[idx] += blk[i][j].re.v;
          Z[idx + 1] += blk[i][j].im.v;
        }
    }
  return 0;
}

}  // extern "C"
