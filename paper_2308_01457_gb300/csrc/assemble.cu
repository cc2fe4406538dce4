// EFIE Galerkin assembly on sm_103a (Sections II-B, II-C and IV-A):
//   Z_mn = -[ ik int int G f_m(x).f_n(y) + 1/(ik) int int G div f_m div f_n ],
//   G(x, y) = exp(ik|x-y|)/(4 pi |x-y|),
// plus the plane-wave right-hand side, the far-field matrix, the PEC shape-derivative
// right-hand side (Section III) and the covariance-kernel product used by the
// second-moment system (Section IV).
//
// Work decomposition of the regular (vertex-disjoint) triangle pairs: one thread per
// ordered triangle pair (t1, t2); a warp holds one test triangle t1 (uniform loads) and
// 32 consecutive trial triangles t2 (coalesced loads).  Each thread accumulates the
// eight complex moments
//     I0 = sum w G,  X = sum w G (x - o1),  Y = sum w G (y - o2),  XY = sum w G (x - o1).(y - o2)
// over the 6 x 6 point pairs (o1, o2 = first vertices: no cancellation), forms the
// 3 x 3 RWG block from them and adds it into Z with FP64 (or FP32) atomics.  Touching
// pairs are skipped here and handled by the Sauter-Schwab kernel.
#include <cuda_runtime.h>

#include <vector>

#include <cstdio>

#include "fosb_internal.h"

namespace fosb {

__constant__ double c_bary[6][3];
__constant__ double c_w[6];
__constant__ double c_glx[16];
__constant__ double c_glw[16];

void upload_rules(const Rules& r) {
  cudaMemcpyToSymbol(c_bary, r.bary, sizeof(r.bary));
  cudaMemcpyToSymbol(c_w, r.w, sizeof(r.w));
  cudaMemcpyToSymbol(c_glx, r.glx, sizeof(r.glx));
  cudaMemcpyToSymbol(c_glw, r.glw, sizeof(r.glw));
}

namespace {

constexpr double kInv4Pi = 0.07957747154594767;  // 1/(4 pi)

template <typename R>
struct Moments {
  R i0r, i0i;
  R xr[3], xi[3];
  R yr[3], yi[3];
  R xyr, xyi;
};

__device__ __forceinline__ void atomic_add_c(double* p, double re, double im) {
  atomicAdd(p, re);
  atomicAdd(p + 1, im);
}
__device__ __forceinline__ void atomic_add_c(float* p, double re, double im) {
  atomicAdd(p, float(re));
  atomicAdd(p + 1, float(im));
}

// Forms the 3 x 3 block from the moments and adds it to Z (or its transpose).
//   A_ij = c_i c'_j [XY - q_j.X - p_i.Y + (p_i.q_j) I0],  Phi_ij = d_i d'_j I0,
//   Z_ij += -ik A_ij - 1/(ik) Phi_ij = -ik A_ij + (i/k) Phi_ij
// with p_i, q_j the opposite vertices relative to the origins o1, o2.
template <typename OutT>
__device__ void scatter_block(double k, const double* m /*16 moments*/, const double p[3][3], const double q[3][3],
                              const double c1[3], const double d1[3], const double c2[3], const double d2[3],
                              const int e1[3], const int e2[3], OutT* Z, int64_t ldz, bool also_transpose) {
  const double i0r = m[0], i0i = m[1];
  for (int i = 0; i < 3; ++i) {
    // p_i . X and p_i . Y
    double pXr = p[i][0] * m[2] + p[i][1] * m[4] + p[i][2] * m[6];
    double pXi = p[i][0] * m[3] + p[i][1] * m[5] + p[i][2] * m[7];
    for (int j = 0; j < 3; ++j) {
      double qXr = q[j][0] * m[2] + q[j][1] * m[4] + q[j][2] * m[6];
      double qXi = q[j][0] * m[3] + q[j][1] * m[5] + q[j][2] * m[7];
      double pYr = p[i][0] * m[8] + p[i][1] * m[10] + p[i][2] * m[12];
      double pYi = p[i][0] * m[9] + p[i][1] * m[11] + p[i][2] * m[13];
      double pq = p[i][0] * q[j][0] + p[i][1] * q[j][1] + p[i][2] * q[j][2];
      double ar = m[14] - qXr - pYr + pq * i0r;
      double ai = m[15] - qXi - pYi + pq * i0i;
      double cc = c1[i] * c2[j], dd = d1[i] * d2[j];
      // -ik (ar + i ai) = k ai - i k ar ;  (i/k) dd (i0r + i i0i) = -(dd/k) i0i + i (dd/k) i0r
      double zr = k * cc * ai - (dd / k) * i0i;
      double zi = -k * cc * ar + (dd / k) * i0r;
      atomic_add_c(Z + 2 * (int64_t(e1[i]) * ldz + e2[j]), zr, zi);
      if (also_transpose) atomic_add_c(Z + 2 * (int64_t(e2[j]) * ldz + e1[i]), zr, zi);
    }
  }
}

__device__ __forceinline__ bool shares_vertex(const int a[3], const int b[3]) {
  bool s = false;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) s |= (a[i] == b[j]);
  return s;
}

// ------------------------------------------------------------------ regular pairs
// R = double (FP64) or float (FP32 path).  OutT = double (complex128 Z) or float.
template <typename R, typename OutT>
__global__ void __launch_bounds__(256) efie_regular_kernel(DevMesh m, double k, OutT* Z, int64_t ldz) {
  const int64_t t1 = int64_t(blockIdx.y) * 8 + (threadIdx.x >> 5);
  const int64_t t2 = int64_t(blockIdx.x) * 32 + (threadIdx.x & 31);
  if (t1 >= m.nt || t2 >= m.nt) return;
  int v1[3], v2[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    v1[a] = m.tris[3 * t1 + a];
    v2[a] = m.tris[3 * t2 + a];
  }
  if (shares_vertex(v1, v2)) return;
  double o1[3], o2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    o1[c] = m.verts[3 * v1[0] + c];
    o2[c] = m.verts[3 * v2[0] + c];
  }
  // quadrature points relative to the origins
  R xq[6][3], yq[6][3];
#pragma unroll
  for (int q = 0; q < 6; ++q)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      xq[q][c] = R(m.tri_qp[18 * t1 + 3 * q + c] - o1[c]);
      yq[q][c] = R(m.tri_qp[18 * t2 + 3 * q + c] - o2[c]);
    }
  R dox = R(o1[0] - o2[0]), doy = R(o1[1] - o2[1]), doz = R(o1[2] - o2[2]);
  const R kk = R(k);
  Moments<R> M{};
  M.i0r = M.i0i = M.xyr = M.xyi = R(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) M.xr[c] = M.xi[c] = M.yr[c] = M.yi[c] = R(0);
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    R s0r = 0, s0i = 0, syr[3] = {0, 0, 0}, syi[3] = {0, 0, 0};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      R dx = dox + xq[p][0] - yq[q][0];
      R dy = doy + xq[p][1] - yq[q][1];
      R dz = doz + xq[p][2] - yq[q][2];
      R r2 = dx * dx + dy * dy + dz * dz;
      R rinv, r;
      if constexpr (sizeof(R) == 8) {
        rinv = rsqrt(r2);
        r = r2 * rinv;
      } else {
        rinv = rsqrtf(r2);
        r = r2 * rinv;
      }
      R sn, cs;
      if constexpr (sizeof(R) == 8)
        sincos(kk * r, &sn, &cs);
      else
        sincosf(kk * r, &sn, &cs);
      R g = R(c_w[q]) * rinv;
      R gr = cs * g, gi = sn * g;
      s0r += gr;
      s0i += gi;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        syr[c] += gr * yq[q][c];
        syi[c] += gi * yq[q][c];
      }
    }
    R wp = R(c_w[p]);
    s0r *= wp;
    s0i *= wp;
    M.i0r += s0r;
    M.i0i += s0i;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      M.xr[c] += s0r * xq[p][c];
      M.xi[c] += s0i * xq[p][c];
      M.yr[c] += wp * syr[c];
      M.yi[c] += wp * syi[c];
      M.xyr += wp * xq[p][c] * syr[c];
      M.xyi += wp * xq[p][c] * syi[c];
    }
  }
  const double scale = m.tri_area[t1] * m.tri_area[t2] * kInv4Pi;
  double mom[16] = {double(M.i0r), double(M.i0i), double(M.xr[0]), double(M.xi[0]), double(M.xr[1]), double(M.xi[1]),
                    double(M.xr[2]), double(M.xi[2]), double(M.yr[0]), double(M.yi[0]), double(M.yr[1]), double(M.yi[1]),
                    double(M.yr[2]), double(M.yi[2]), double(M.xyr), double(M.xyi)};
#pragma unroll
  for (int i = 0; i < 16; ++i) mom[i] *= scale;
  double p[3][3], q[3][3], c1[3], d1[3], c2[3], d2[3];
  int e1[3], e2[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      p[i][c] = m.verts[3 * v1[i] + c] - o1[c];
      q[i][c] = m.verts[3 * v2[i] + c] - o2[c];
    }
    c1[i] = m.tri_coef[3 * t1 + i];
    d1[i] = m.tri_div[3 * t1 + i];
    c2[i] = m.tri_coef[3 * t2 + i];
    d2[i] = m.tri_div[3 * t2 + i];
    e1[i] = m.tri_edge[3 * t1 + i];
    e2[i] = m.tri_edge[3 * t2 + i];
  }
  scatter_block(k, mom, p, q, c1, d1, c2, d2, e1, e2, Z, ldz, false);
}

// ------------------------------------------------------------------ singular pairs
// One CTA of 128 threads per touching pair; the Sauter-Schwab 4-cube points are split
// over the threads, the moments reduced through shared memory.  FP64 throughout.
// chi(u) - P0 = u1 (P1 - P0) + u2 (P2 - P1), with the edge vectors E[0] = P1 - P0 and
// E[1] = P2 - P1 formed once per pair
__device__ __forceinline__ void chi_rel(const double E[2][3], double u1, double u2, double out[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) out[c] = fma(u1, E[0][c], u2 * E[1][c]);
}

// exp(i th) for 0 <= th <= 64 in FP64: Cody-Waite reduction th = n pi/2 + d (pi/2 split in
// three parts, the first with 33 significant bits so that n times it is exact), |d| <= pi/4,
// and the Taylor series of sin d / d to d^16 and of cos d to d^18 (truncation below 2e-20
// relative), then the quadrant n mod 4.  Larger phases, which no touching pair of a resolved
// mesh reaches, fall back to sincos.
__device__ __forceinline__ void ss_expi(double th, double& c, double& s) {
  if (!(th <= 64.0)) {
    sincos(th, &s, &c);
    return;
  }
  const double n = rint(th * 0.6366197723675814);
  const double d = fma(-n, 3.5215598651832e-27, fma(-n, 6.077100506506192e-11, fma(-n, 1.5707963267341256, th)));
  const double d2 = d * d;
  // sin d / d = sum_i (-d2)^i / (2i + 1)!,  cos d = sum_i (-d2)^i / (2i)!
  double ps = 1.0 / 355687428096000.0;          // 1/17!
  ps = fma(ps, -d2, 1.0 / 1307674368000.0);     // 1/15!
  ps = fma(ps, -d2, 1.0 / 6227020800.0);        // 1/13!
  ps = fma(ps, -d2, 1.0 / 39916800.0);          // 1/11!
  ps = fma(ps, -d2, 1.0 / 362880.0);            // 1/9!
  ps = fma(ps, -d2, 1.0 / 5040.0);              // 1/7!
  ps = fma(ps, -d2, 1.0 / 120.0);               // 1/5!
  ps = fma(ps, -d2, 1.0 / 6.0);                 // 1/3!
  ps = fma(ps, -d2, 1.0);
  double pc = 1.0 / 6402373705728000.0;         // 1/18!
  pc = fma(pc, -d2, 1.0 / 20922789888000.0);    // 1/16!
  pc = fma(pc, -d2, 1.0 / 87178291200.0);       // 1/14!
  pc = fma(pc, -d2, 1.0 / 479001600.0);         // 1/12!
  pc = fma(pc, -d2, 1.0 / 3628800.0);           // 1/10!
  pc = fma(pc, -d2, 1.0 / 40320.0);             // 1/8!
  pc = fma(pc, -d2, 1.0 / 720.0);               // 1/6!
  pc = fma(pc, -d2, 1.0 / 24.0);                // 1/4!
  pc = fma(pc, -d2, 0.5);                       // 1/2!
  pc = fma(pc, -d2, 1.0);
  const double sd = d * ps, cd = pc;
  // sin(d + q pi/2), cos(d + q pi/2) for q = n mod 4
  const int q = int(n) & 3;
  s = q == 0 ? sd : (q == 1 ? cd : (q == 2 ? -sd : -cd));
  c = q == 0 ? cd : (q == 1 ? -sd : (q == 2 ? -cd : sd));
}

__device__ __forceinline__ void ss_accumulate(double k, const double x[3], const double y[3], double w, double acc[16]) {
  const double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
  const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
  // 1/r from a float seed and two Newton steps in FP64, y <- y (3 - r2 y^2) / 2:
  // about 22, then 44, then full significant bits
  double yr = double(rsqrtf(float(r2)));
  yr = yr * fma(-0.5 * r2, yr * yr, 1.5);
  yr = yr * fma(-0.5 * r2, yr * yr, 1.5);
  double sn, cs;
  ss_expi(k * (r2 * yr), cs, sn);
  const double g = w * yr;
  const double gr = cs * g, gi = sn * g;
  acc[0] += gr;
  acc[1] += gi;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[2 + 2 * c] += gr * x[c];
    acc[3 + 2 * c] += gi * x[c];
    acc[8 + 2 * c] += gr * y[c];
    acc[9 + 2 * c] += gi * y[c];
  }
  double xy = x[0] * y[0] + x[1] * y[1] + x[2] * y[2];
  acc[14] += gr * xy;
  acc[15] += gi * xy;
}

// One touching pair (index pair of m.touch) by one warp: the lanes share the Sauter-Schwab
// 4-cube points, a butterfly reduction leaves the 16 moments in every lane, and lanes 0-8
// form one entry each of the 3 x 3 RWG block and add it (and its mirror) into Z.
template <typename OutT>
__device__ __forceinline__ void singular_pair(const DevMesh& m, double k, int nss, OutT* Z, int64_t ldz, int64_t pair) {
  const int lane = threadIdx.x & 31;
  const double kinv = 1.0 / k;
  const TouchPair tp = m.touch[pair];
  double P[3][3], Q[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      P[a][c] = m.verts[3 * tp.p[a] + c];
      Q[a][c] = m.verts[3 * tp.q[a] + c];
    }
  // P0 == Q0 for every touching kind, so x - y = (x - P0) - (y - Q0) exactly.
  double EP[2][3], EQ[2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    EP[0][c] = P[1][c] - P[0][c];
    EP[1][c] = P[2][c] - P[1][c];
    EQ[0][c] = Q[1][c] - Q[0][c];
    EQ[1][c] = Q[2][c] - Q[1][c];
  }
  const int n2 = nss * nss, n4 = n2 * n2;
  double acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.0;
  for (int idx = lane; idx < n4; idx += 32) {
    int a = idx / (n2 * nss), b = (idx / n2) % nss, c = (idx / nss) % nss, d = idx % nss;
    double xi = c_glx[a], e1 = c_glx[b], e2 = c_glx[c], e3 = c_glx[d];
    double w4 = c_glw[a] * c_glw[b] * c_glw[c] * c_glw[d];
    double x[3], y[3];
    if (tp.kind == 3) {
      double w = w4 * xi * xi * xi * e1 * e1 * e2;
      const double s[6][4] = {
          {xi, xi * (1 - e1 + e1 * e2), xi * (1 - e1 * e2 * e3), xi * (1 - e1)},
          {xi * (1 - e1 * e2 * e3), xi * (1 - e1), xi, xi * (1 - e1 + e1 * e2)},
          {xi, xi * e1 * (1 - e2 + e2 * e3), xi * (1 - e1 * e2), xi * e1 * (1 - e2)},
          {xi * (1 - e1 * e2), xi * e1 * (1 - e2), xi, xi * e1 * (1 - e2 + e2 * e3)},
          {xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), xi, xi * e1 * (1 - e2)},
          {xi, xi * e1 * (1 - e2), xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)}};
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        chi_rel(EP, s[j][0], s[j][1], x);
        chi_rel(EQ, s[j][2], s[j][3], y);
        ss_accumulate(k, x, y, w, acc);
      }
    } else if (tp.kind == 2) {
      double w0 = w4 * xi * xi * xi * e1 * e1, w1 = w0 * e2;
      const double s[5][5] = {
          {xi, xi * e1 * e3, xi * (1 - e1 * e2), xi * e1 * (1 - e2), w0},
          {xi, xi * e1, xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3), w1},
          {xi * (1 - e1 * e2), xi * e1 * (1 - e2), xi, xi * e1 * e2 * e3, w1},
          {xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3), xi, xi * e1, w1},
          {xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), xi, xi * e1 * e2, w1}};
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        chi_rel(EP, s[j][0], s[j][1], x);
        chi_rel(EQ, s[j][2], s[j][3], y);
        ss_accumulate(k, x, y, s[j][4], acc);
      }
    } else {
      double w = w4 * xi * xi * xi * e2;
      chi_rel(EP, xi, xi * e1, x);
      chi_rel(EQ, xi * e2, xi * e2 * e3, y);
      ss_accumulate(k, x, y, w, acc);
      chi_rel(EP, xi * e2, xi * e2 * e3, x);
      chi_rel(EQ, xi, xi * e1, y);
      ss_accumulate(k, x, y, w, acc);
    }
  }
  // butterfly reduction: every lane ends with the 16 sums
#pragma unroll
  for (int i = 0; i < 16; ++i) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], off);
  }
  if (lane >= 9) return;
  // lane = 3 i + j: entry (i, j) of the block,
  //   A_ij = c_i c'_j [XY - q_j.X - p_i.Y + (p_i.q_j) I0],  Phi_ij = d_i d'_j I0,
  //   Z_ij += -ik A_ij + (i/k) Phi_ij,
  // with p_i, q_j the opposite vertices relative to P0 = Q0
  const int i = lane / 3, j = lane % 3;
  const int t1 = tp.t1, t2 = tp.t2;
  const double jac = 4.0 * m.tri_area[t1] * m.tri_area[t2] * kInv4Pi;
  const int a = m.tris[3 * t1 + i], b = m.tris[3 * t2 + j];
  double pi_[3], qj[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    pi_[c] = m.verts[3 * a + c] - P[0][c];
    qj[c] = m.verts[3 * b + c] - Q[0][c];
  }
  double mo[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) mo[q] = acc[q] * jac;
  const double qXr = qj[0] * mo[2] + qj[1] * mo[4] + qj[2] * mo[6];
  const double qXi = qj[0] * mo[3] + qj[1] * mo[5] + qj[2] * mo[7];
  const double pYr = pi_[0] * mo[8] + pi_[1] * mo[10] + pi_[2] * mo[12];
  const double pYi = pi_[0] * mo[9] + pi_[1] * mo[11] + pi_[2] * mo[13];
  const double pq = pi_[0] * qj[0] + pi_[1] * qj[1] + pi_[2] * qj[2];
  const double ar = mo[14] - qXr - pYr + pq * mo[0];
  const double ai = mo[15] - qXi - pYi + pq * mo[1];
  const double cc = m.tri_coef[3 * t1 + i] * m.tri_coef[3 * t2 + j];
  const double dk = m.tri_div[3 * t1 + i] * m.tri_div[3 * t2 + j] * kinv;
  // -ik (ar + i ai) = k ai - i k ar;  (i/k) dd (I0r + i I0i) = -(dd/k) I0i + i (dd/k) I0r
  const double zr = k * cc * ai - dk * mo[1];
  const double zi = -k * cc * ar + dk * mo[0];
  const int e1 = m.tri_edge[3 * t1 + i], e2 = m.tri_edge[3 * t2 + j];
  atomic_add_c(Z + 2 * (int64_t(e1) * ldz + e2), zr, zi);
  if (t1 != t2) atomic_add_c(Z + 2 * (int64_t(e2) * ldz + e1), zr, zi);
}

// four touching pairs per 128-thread CTA, one per warp
template <typename OutT>
__global__ void __launch_bounds__(128) efie_singular_kernel(DevMesh m, double k, int nss, OutT* Z, int64_t ldz) {
  const int64_t pair = int64_t(blockIdx.x) * 4 + (threadIdx.x >> 5);
  if (pair < m.ntouch) singular_pair(m, k, nss, Z, ldz, pair);
}

// Batched forms over many meshes: a flat grid whose block (singular) or thread (RHS) index
// falls in the item with the largest start <= index.
struct BatchItem {
  DevMesh m;
  double k;
  double* Z;
  int64_t ldz;
  double* b;
  int64_t ldb;
  const double* inc;  // n_inc x 9
  int64_t n_inc;
  int64_t pair_start;  // first touching pair of this item in the batch
  int64_t rhs_start;   // first (triangle, incidence) of this item in the batch
};

__device__ __forceinline__ int batch_find(const BatchItem* items, int n, int64_t w, bool rhs) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((rhs ? items[mid].rhs_start : items[mid].pair_start) <= w) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(128) efie_singular_batched_kernel(const BatchItem* __restrict__ items, int nitems,
                                                                    int64_t pairs, int nss) {
  const int64_t w = int64_t(blockIdx.x) * 4 + (threadIdx.x >> 5);  // one pair per warp
  if (w >= pairs) return;
  const BatchItem& it = items[batch_find(items, nitems, w, false)];
  singular_pair(it.m, it.k, nss, it.Z, it.ldz, w - it.pair_start);
}

// ------------------------------------------------------------------ right-hand side
// b[m, s] = -int E_inc_s . f_m, one thread per (triangle, incidence).
template <typename OutT>
__device__ __forceinline__ void rhs_one(const DevMesh& m, double k, const double* inc, int64_t n_inc, OutT* b,
                                        int64_t ldb, int64_t t, int64_t s) {
  const double* c = inc + 9 * s;
  double acc_r[3] = {0, 0, 0}, acc_i[3] = {0, 0, 0};
  for (int qp = 0; qp < 6; ++qp) {
    const double* x = m.tri_qp + 18 * t + 3 * qp;
    double sn, cs;
    sincos(k * (c[0] * x[0] + c[1] * x[1] + c[2] * x[2]), &sn, &cs);
    for (int i = 0; i < 3; ++i) {
      int pv = m.tris[3 * t + i];
      double f[3];
      for (int d = 0; d < 3; ++d) f[d] = (x[d] - m.verts[3 * pv + d]) * m.tri_coef[3 * t + i];
      double pr = c[3] * f[0] + c[4] * f[1] + c[5] * f[2];
      double pi = c[6] * f[0] + c[7] * f[1] + c[8] * f[2];
      // (pr + i pi)(cs + i sn)
      acc_r[i] += c_w[qp] * (pr * cs - pi * sn);
      acc_i[i] += c_w[qp] * (pr * sn + pi * cs);
    }
  }
  double A = m.tri_area[t];
  for (int i = 0; i < 3; ++i)
    atomic_add_c(b + 2 * (int64_t(m.tri_edge[3 * t + i]) * ldb + s), -A * acc_r[i], -A * acc_i[i]);
}

template <typename OutT>
__global__ void rhs_kernel(DevMesh m, double k, const double* inc, int64_t n_inc, OutT* b, int64_t ldb) {
  int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= m.nt * n_inc) return;
  rhs_one(m, k, inc, n_inc, b, ldb, gid / n_inc, gid % n_inc);
}

__global__ void rhs_batched_kernel(const BatchItem* __restrict__ items, int nitems, int64_t total) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= total) return;
  const BatchItem& it = items[batch_find(items, nitems, gid, true)];
  const int64_t local = gid - it.rhs_start;
  rhs_one(it.m, it.k, it.inc, it.n_inc, it.b, it.ldb, local / it.n_inc, local % it.n_inc);
}

// ------------------------------------------------------------------ far-field matrix
// A[3d + c, n] = -ik [(I - xh xh^T) int f_n exp(-ik xh.y)]_c, thread per (triangle, direction).
template <typename OutT>
__global__ void farfield_kernel(DevMesh m, double k, const double* dirs, int64_t n_dir, OutT* A) {
  int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= m.nt * n_dir) return;
  int64_t t = gid / n_dir, d = gid % n_dir;
  const double u[3] = {dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2]};
  double Jr[3][3] = {}, Ji[3][3] = {};
  for (int qp = 0; qp < 6; ++qp) {
    const double* y = m.tri_qp + 18 * t + 3 * qp;
    double sn, cs;
    sincos(-k * (u[0] * y[0] + u[1] * y[1] + u[2] * y[2]), &sn, &cs);
    for (int i = 0; i < 3; ++i) {
      int pv = m.tris[3 * t + i];
      for (int c = 0; c < 3; ++c) {
        double f = (y[c] - m.verts[3 * pv + c]) * m.tri_coef[3 * t + i] * c_w[qp];
        Jr[i][c] += f * cs;
        Ji[i][c] += f * sn;
      }
    }
  }
  double A_t = m.tri_area[t];
  for (int i = 0; i < 3; ++i) {
    double uJr = u[0] * Jr[i][0] + u[1] * Jr[i][1] + u[2] * Jr[i][2];
    double uJi = u[0] * Ji[i][0] + u[1] * Ji[i][1] + u[2] * Ji[i][2];
    int64_t n = m.tri_edge[3 * t + i];
    for (int c = 0; c < 3; ++c) {
      double Tr = (Jr[i][c] - u[c] * uJr) * A_t, Ti = (Ji[i][c] - u[c] * uJi) * A_t;
      // -ik (Tr + i Ti) = k Ti - i k Tr
      atomic_add_c(A + 2 * ((3 * d + c) * m.ne + n), k * Ti, -k * Tr);
    }
  }
}

// ------------------------------------------------------------------ shape-derivative RHS
// B_mp = -sum_n u_n int_T psi_p nu_{p,T} [ik f_m.f_n + 1/(ik) div f_m div f_n], one
// thread per triangle; the nine (edge, vertex) contributions go to the ELL slots of row m:
// slot 0/1 = edge endpoints a/b, slot 2/3 = opposite vertex in T+/T-.
template <typename UT>
__global__ void sd_rhs_kernel(DevMesh m, double k, const UT* u, double* Bell) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= m.nt) return;
  int v[3], e[3];
  double un_r[3], un_i[3], nu[3];
  for (int a = 0; a < 3; ++a) {
    v[a] = m.tris[3 * t + a];
    e[a] = m.tri_edge[3 * t + a];
    un_r[a] = double(u[2 * e[a]]);
    un_i[a] = double(u[2 * e[a] + 1]);
    nu[a] = m.vnormals[3 * v[a]] * m.tri_normal[3 * t] + m.vnormals[3 * v[a] + 1] * m.tri_normal[3 * t + 1] +
            m.vnormals[3 * v[a] + 2] * m.tri_normal[3 * t + 2];
  }
  double acc_r[3][3] = {}, acc_i[3][3] = {};
  const double A = m.tri_area[t];
  for (int qp = 0; qp < 6; ++qp) {
    const double* x = m.tri_qp + 18 * t + 3 * qp;
    double f[3][3];
    for (int i = 0; i < 3; ++i)
      for (int c = 0; c < 3; ++c) f[i][c] = (x[c] - m.verts[3 * v[i] + c]) * m.tri_coef[3 * t + i];
    const double w = c_w[qp] * A;
    for (int i = 0; i < 3; ++i) {
      double sr = 0, si = 0;
      for (int j = 0; j < 3; ++j) {
        double ff = f[i][0] * f[j][0] + f[i][1] * f[j][1] + f[i][2] * f[j][2];
        double dd = m.tri_div[3 * t + i] * m.tri_div[3 * t + j];
        // ik ff + dd/(ik) = i (k ff - dd/k)
        double cim = k * ff - dd / k;
        sr += -un_i[j] * cim;
        si += un_r[j] * cim;
      }
      for (int a = 0; a < 3; ++a) {
        double wl = w * c_bary[qp][a] * nu[a];
        acc_r[i][a] -= sr * wl;
        acc_i[i][a] -= si * wl;
      }
    }
  }
  for (int i = 0; i < 3; ++i) {
    int64_t row = e[i];
    int a_id = m.ell_cols[4 * row];
    bool plus = m.tri_coef[3 * t + i] > 0;
    for (int a = 0; a < 3; ++a) {
      int slot = (a == i) ? (plus ? 2 : 3) : (v[a] == a_id ? 0 : 1);
      atomic_add_c(Bell + 2 * (4 * row + slot), acc_r[i][a], acc_i[i][a]);
    }
  }
}

template <typename OutT>
__global__ void ell_to_dense_kernel(DevMesh m, const double* Bell, bool conj_out, OutT* B, int64_t ldb) {
  int64_t row = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (row >= m.ne) return;
  for (int s = 0; s < 4; ++s) {
    int col = m.ell_cols[4 * row + s];
    B[2 * (row * ldb + col)] = OutT(Bell[2 * (4 * row + s)]);
    B[2 * (row * ldb + col) + 1] = OutT(conj_out ? -Bell[2 * (4 * row + s) + 1] : Bell[2 * (4 * row + s) + 1]);
  }
}

// W[m, q] = sum_s B1[m, s] K(|x_{col(m,s)} - y_q|), K = sigma^2 rho(r).
template <typename OutT>
__global__ void bk_product_kernel(DevMesh m1, const double* Bell, DevMesh m2, int kind, double sigma, double ell,
                                  OutT* W, int64_t ldw) {
  int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t row = blockIdx.y;
  if (q >= m2.nv) return;
  const double y[3] = {m2.verts[3 * q], m2.verts[3 * q + 1], m2.verts[3 * q + 2]};
  double wr = 0, wi = 0;
  for (int s = 0; s < 4; ++s) {
    int p = m1.ell_cols[4 * row + s];
    double dx = m1.verts[3 * p] - y[0], dy = m1.verts[3 * p + 1] - y[1], dz = m1.verts[3 * p + 2] - y[2];
    double r2 = dx * dx + dy * dy + dz * dz;
    double kv;
    if (kind == FOSB_COV_GAUSS) {
      kv = sigma * sigma * exp(-r2 / (2.0 * ell * ell));
    } else {
      double sr = 1.7320508075688772 * sqrt(r2) / ell;
      kv = sigma * sigma * (1.0 + sr) * exp(-sr);
    }
    wr += Bell[2 * (4 * row + s)] * kv;
    wi += Bell[2 * (4 * row + s) + 1] * kv;
  }
  W[2 * (row * ldw + q)] = OutT(wr);
  W[2 * (row * ldw + q) + 1] = OutT(wi);
}

inline unsigned blocks_for(int64_t n, int bs) { return unsigned((n + bs - 1) / bs); }

}  // namespace

cudaError_t launch_assemble_regular(const DevMesh& m, double k, int arith, void* Z, int64_t ldz, cudaStream_t s) {
  dim3 grid(blocks_for(m.nt, 32), blocks_for(m.nt, 8));
  ProfScope prof("asm_regular", s, 36.0 * (double(m.nt) * double(m.nt) - double(2 * m.ntouch - m.nt)));
  if (arith == FOSB_ASM_FP64) {
    efie_regular_kernel<double, double><<<grid, 256, 0, s>>>(m, k, static_cast<double*>(Z), ldz);
  } else if (arith == FOSB_ASM_FF) {
    return launch_efie_regular_ff(m, k, static_cast<double*>(Z), ldz, s);
  } else {
    efie_regular_kernel<float, float><<<grid, 256, 0, s>>>(m, k, static_cast<float*>(Z), ldz);
  }
  return launched();
}

cudaError_t launch_assemble_singular(const DevMesh& m, double k, int nss, bool fp32_out, void* Z, int64_t ldz,
                                     cudaStream_t s) {
  if (m.ntouch == 0) return cudaSuccess;
  ProfScope prof("asm_singular", s, double(m.ntouch));
  if (fp32_out)
    efie_singular_kernel<float><<<blocks_for(m.ntouch, 4), 128, 0, s>>>(m, k, nss, static_cast<float*>(Z), ldz);
  else
    efie_singular_kernel<double><<<blocks_for(m.ntouch, 4), 128, 0, s>>>(m, k, nss, static_cast<double*>(Z), ldz);
  return launched();
}

cudaError_t launch_rhs(const DevMesh& m, double k, const double* d_inc, int64_t n_inc, bool fp32_out, void* b,
                       int64_t ldb, cudaStream_t s) {
  if (n_inc == 0) return cudaSuccess;
  unsigned g = blocks_for(m.nt * n_inc, 128);
  if (fp32_out)
    rhs_kernel<float><<<g, 128, 0, s>>>(m, k, d_inc, n_inc, static_cast<float*>(b), ldb);
  else
    rhs_kernel<double><<<g, 128, 0, s>>>(m, k, d_inc, n_inc, static_cast<double*>(b), ldb);
  return launched();
}

cudaError_t launch_farfield_matrix(const DevMesh& m, double k, const double* d_dirs, int64_t n_dir, bool fp32,
                                   void* A, cudaStream_t s) {
  unsigned g = blocks_for(m.nt * n_dir, 128);
  if (fp32)
    farfield_kernel<float><<<g, 128, 0, s>>>(m, k, d_dirs, n_dir, static_cast<float*>(A));
  else
    farfield_kernel<double><<<g, 128, 0, s>>>(m, k, d_dirs, n_dir, static_cast<double*>(A));
  return launched();
}

cudaError_t launch_sd_rhs(const DevMesh& m, double k, const void* u, bool u_fp32, double* B_ell, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(B_ell, 0, sizeof(double) * 8 * m.ne, s);
  if (e != cudaSuccess) return e;
  if (u_fp32)
    sd_rhs_kernel<float><<<blocks_for(m.nt, 128), 128, 0, s>>>(m, k, static_cast<const float*>(u), B_ell);
  else
    sd_rhs_kernel<double><<<blocks_for(m.nt, 128), 128, 0, s>>>(m, k, static_cast<const double*>(u), B_ell);
  return launched();
}

cudaError_t launch_ell_to_dense(const DevMesh& m, const double* B_ell, bool conj_out, bool fp32, void* B, int64_t ldb,
                                cudaStream_t s) {
  size_t elem = fp32 ? 8 : 16;
  cudaError_t e = cudaMemset2DAsync(B, ldb * elem, 0, m.nv * elem, m.ne, s);
  if (e != cudaSuccess) return e;
  if (fp32)
    ell_to_dense_kernel<float><<<blocks_for(m.ne, 128), 128, 0, s>>>(m, B_ell, conj_out, static_cast<float*>(B), ldb);
  else
    ell_to_dense_kernel<double><<<blocks_for(m.ne, 128), 128, 0, s>>>(m, B_ell, conj_out, static_cast<double*>(B), ldb);
  return launched();
}

cudaError_t launch_bk_product(const DevMesh& m1, const double* B1_ell, const DevMesh& m2, const fosb_cov_kernel& ker,
                              bool fp32, void* W, int64_t ldw, cudaStream_t s) {
  if (m1.ne > 65535) return cudaErrorInvalidValue;  // grid.y bound
  dim3 grid(blocks_for(m2.nv, 128), unsigned(m1.ne));
  if (fp32)
    bk_product_kernel<float><<<grid, 128, 0, s>>>(m1, B1_ell, m2, ker.kind, ker.sigma, ker.ell, static_cast<float*>(W), ldw);
  else
    bk_product_kernel<double><<<grid, 128, 0, s>>>(m1, B1_ell, m2, ker.kind, ker.sigma, ker.ell, static_cast<double*>(W), ldw);
  return launched();
}

size_t batched_items_bytes(int nmesh) { return sizeof(BatchItem) * size_t(nmesh); }

// Singular pairs and plane-wave right-hand sides of a batch of meshes (complex128 Z and b,
// zeroed by the caller), one launch each; d_items: batched_items_bytes(nmesh) bytes of
// device scratch, inc[i]: device n_inc[i] x 9 (may be NULL when n_inc[i] = 0).
cudaError_t launch_singular_rhs_batched(const DevMesh* const* meshes, const double* ks, double* const* Z,
                                        const int64_t* ldz, double* const* b, const int64_t* ldb,
                                        const double* const* inc, const int64_t* n_inc, int nmesh, int nss,
                                        void* d_items, cudaStream_t s) {
  std::vector<BatchItem> items(nmesh);
  int64_t pairs = 0, rhs = 0;
  for (int i = 0; i < nmesh; ++i) {
    BatchItem& it = items[i];
    it.m = *meshes[i];
    it.k = ks[i];
    it.Z = Z[i];
    it.ldz = ldz[i];
    it.b = b[i];
    it.ldb = ldb[i];
    it.inc = inc[i];
    it.n_inc = n_inc[i];
    it.pair_start = pairs;
    it.rhs_start = rhs;
    pairs += it.m.ntouch;
    rhs += it.n_inc > 0 && it.b ? it.m.nt * it.n_inc : 0;
  }
  if (pairs > 0x7fffffff) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemcpyAsync(d_items, items.data(), sizeof(BatchItem) * nmesh, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const BatchItem* di = static_cast<const BatchItem*>(d_items);
  if (pairs > 0) {
    ProfScope prof("asm_singular", s, double(pairs));
    efie_singular_batched_kernel<<<blocks_for(pairs, 4), 128, 0, s>>>(di, nmesh, pairs, nss);
    e = launched();
    if (e != cudaSuccess) return e;
  }
  if (rhs > 0) {
    rhs_batched_kernel<<<blocks_for(rhs, 128), 128, 0, s>>>(di, nmesh, rhs);
    e = launched();
  }
  return e;
}

}  // namespace fosb
