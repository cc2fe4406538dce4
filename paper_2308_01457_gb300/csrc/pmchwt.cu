// Dielectric scatterer: Galerkin assembly of the PMCHWT system and its far field on sm_103a
// (Section II-C eq. pmchwt, with the multitrace operators of eq. BOmultitraceA).
//
// The unknowns are the exterior Cauchy data (j, m) = (gamma_D^c E, gamma_N^c E) of the total
// field in RWG coefficients.  The exterior field satisfies (I/2 + A_0)(j, m)_sc = 0, the
// interior one (I/2 - A_1) xi_1 = 0 with xi_1 = diag(1, eta) (j, m), and the incident field,
// regular inside, (I/2 - A_0) xi_inc = 0; subtracting gives
//     (A_0 + A^_1)(j, m) = xi_inc,   A^_1 = [[K_1, eta T_1], [-T_1/eta, K_1]],
// the printed system (A_0 + A^_1) xi_sc = (I/2 - A^_1) xi_inc written for xi_sc + xi_inc.
// Tested with the x-pairing against RWG functions:
//     Z (2N x 2N) = [[K_0 + K_1, T_0 + eta T_1], [-T_0 - T_1/eta, K_0 + K_1]],
//     T_k[m, n] = -[ik int int G f_m.f_n + 1/(ik) int int G div f_m div f_n]     (EFIO),
//     K_k[m, n] = -int int (x - y).(f_n(y) x f_m(x)) exp(ikr)(ikr - 1)/(4 pi r^3)  (MFIO),
// k = k0 outside and k1 = k0 sqrt(eps_r mu_r) inside, eta = sqrt(mu_r/eps_r).
//
// Work decomposition.  One launch per wavenumber computes, for every triangle pair, the
// EFIO and the MFIO 3 x 3 blocks from one set of point-pair evaluations (r, exp(ikr)) and
// adds them with FP64 atomics into two N x N blocks of Z: K into the (1,1) block for both
// wavenumbers, T_0 into the (1,2) block and T_1, as scratch, into the (2,2) block.  A final
// pass rewrites every entry: (1,2) = T_0 + eta T_1, (2,1) = -T_0 - T_1/eta, (2,2) = (1,1).
// So a triangle pair costs 18 complex atomics per wavenumber, the same as the PEC EFIE.
// The regular pairs run in FP64 here (FOSB_ASM_FP64) or in float-float on the FP32 pipe
// (FOSB_ASM_FF, pmchwt_regular_ff_kernel in ff_assemble.cu, from barycentric moment
// matrices); the touching pairs always run in FP64 here.
//
// Moments.  With x' = x - o1, y' = y - o2 (first vertices as origins) and D = o1 - o2,
//   EFIO:  I0 = sum w G, X = sum w G x', Y = sum w G y', XY = sum w G x'.y',   G = exp(ikr)/r;
//   MFIO:  J0 = sum w g, JX = sum w g x', JY = sum w g y', JYX = sum w g (y' x x'),
//          g = exp(ikr)(ikr - 1)/r^3.
// Since a - b = x - y - (p_i - q_j) for a = x - p_i, b = y - q_j, (x - y).(b x a) =
// (p_i - q_j).(b x a), so with p'_i, q'_j relative to o1, o2
//   K_ij = -c_i c'_j (p'_i - q'_j + D).[JYX - JY x p'_i - q'_j x JX + (q'_j x p'_i) J0].
// On one flat triangle x - y lies in the plane and b x a is normal to it: identical pairs
// add nothing to K (the principal value of the averaged trace).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "fosb_internal.h"

namespace fosb {
namespace {

__constant__ double c_pm_bary[6][3];
__constant__ double c_pm_w[6];
__constant__ double c_pm_glx[16];
__constant__ double c_pm_glw[16];

constexpr double kInv4PiPm = 0.07957747154594767;  // 1/(4 pi)

__device__ __forceinline__ void atomic_add_z(double* p, double re, double im) {
  atomicAdd(p, re);
  atomicAdd(p + 1, im);
}

// EFIO (16 doubles: I0, X, Y, XY as (re, im)) and MFIO (20 doubles: J0, JX, JY, JYX) moments
// of one triangle pair -> entry (i, j) of both blocks.  p, q: opposite vertices relative to
// o1, o2; D = o1 - o2.
__device__ __forceinline__ void pair_entry(double k, const double* e /*16*/, const double* h /*20*/, const double p[3],
                                           const double q[3], const double D[3], double cc, double dd, double& tr,
                                           double& ti, double& kr, double& ki) {
  // EFIO: -ik cc [XY - q.X - p.Y + (p.q) I0] + (i/k) dd I0
  const double qXr = q[0] * e[2] + q[1] * e[4] + q[2] * e[6];
  const double qXi = q[0] * e[3] + q[1] * e[5] + q[2] * e[7];
  const double pYr = p[0] * e[8] + p[1] * e[10] + p[2] * e[12];
  const double pYi = p[0] * e[9] + p[1] * e[11] + p[2] * e[13];
  const double pq = p[0] * q[0] + p[1] * q[1] + p[2] * q[2];
  const double ar = e[14] - qXr - pYr + pq * e[0];
  const double ai = e[15] - qXi - pYi + pq * e[1];
  tr = k * cc * ai - (dd / k) * e[1];
  ti = -k * cc * ar + (dd / k) * e[0];
  // MFIO: V = JYX - JY x p - q x JX + (q x p) J0 (complex 3-vector), K = -cc (p - q + D).V
  const double qp[3] = {q[1] * p[2] - q[2] * p[1], q[2] * p[0] - q[0] * p[2], q[0] * p[1] - q[1] * p[0]};
  const double d[3] = {p[0] - q[0] + D[0], p[1] - q[1] + D[1], p[2] - q[2] + D[2]};
  double vr = 0.0, vi = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
    // (JY x p)_c = JY_c1 p_c2 - JY_c2 p_c1 ;  (q x JX)_c = q_c1 JX_c2 - q_c2 JX_c1
    const double wr = h[14 + 2 * c] - (h[8 + 2 * c1] * p[c2] - h[8 + 2 * c2] * p[c1]) -
                      (q[c1] * h[2 + 2 * c2] - q[c2] * h[2 + 2 * c1]) + qp[c] * h[0];
    const double wi = h[15 + 2 * c] - (h[9 + 2 * c1] * p[c2] - h[9 + 2 * c2] * p[c1]) -
                      (q[c1] * h[3 + 2 * c2] - q[c2] * h[3 + 2 * c1]) + qp[c] * h[1];
    vr += d[c] * wr;
    vi += d[c] * wi;
  }
  kr = -cc * vr;
  ki = -cc * vi;
}

__device__ __forceinline__ bool pm_shares_vertex(const int a[3], const int b[3]) {
  bool s = false;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) s |= (a[i] == b[j]);
  return s;
}

// ------------------------------------------------------------------ regular pairs
// One thread per ordered vertex-disjoint triangle pair (t1 test, t2 trial); a warp holds one
// test triangle and 32 consecutive trial triangles.  FP64.
__global__ void __launch_bounds__(256) pmchwt_regular_kernel(DevMesh m, double k, double* ZT, double* ZK,
                                                             int64_t ldz) {
  const int64_t t1 = int64_t(blockIdx.y) * 8 + (threadIdx.x >> 5);
  const int64_t t2 = int64_t(blockIdx.x) * 32 + (threadIdx.x & 31);
  if (t1 >= m.nt || t2 >= m.nt) return;
  int v1[3], v2[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    v1[a] = m.tris[3 * t1 + a];
    v2[a] = m.tris[3 * t2 + a];
  }
  if (pm_shares_vertex(v1, v2)) return;
  double o1[3], o2[3], D[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    o1[c] = m.verts[3 * v1[0] + c];
    o2[c] = m.verts[3 * v2[0] + c];
    D[c] = o1[c] - o2[c];
  }
  double xq[6][3], yq[6][3];
#pragma unroll
  for (int q = 0; q < 6; ++q)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      xq[q][c] = m.tri_qp[18 * t1 + 3 * q + c] - o1[c];
      yq[q][c] = m.tri_qp[18 * t2 + 3 * q + c] - o2[c];
    }
  double e[16], h[20];
#pragma unroll
  for (int i = 0; i < 16; ++i) e[i] = 0.0;
#pragma unroll
  for (int i = 0; i < 20; ++i) h[i] = 0.0;
#pragma unroll 1
  for (int p = 0; p < 6; ++p) {
    double s0r = 0, s0i = 0, syr[3] = {0, 0, 0}, syi[3] = {0, 0, 0};
    double j0r = 0, j0i = 0, jyr[3] = {0, 0, 0}, jyi[3] = {0, 0, 0};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const double dx = D[0] + xq[p][0] - yq[q][0];
      const double dy = D[1] + xq[p][1] - yq[q][1];
      const double dz = D[2] + xq[p][2] - yq[q][2];
      const double r2 = dx * dx + dy * dy + dz * dz;
      const double rinv = rsqrt(r2);
      const double r = r2 * rinv;
      double sn, cs;
      sincos(k * r, &sn, &cs);
      const double g = c_pm_w[q] * rinv;
      const double gr = cs * g, gi = sn * g;  // w G
      // w g = w G (ikr - 1)/r^2
      const double kr = k * r, rinv2 = rinv * rinv;
      const double hr = (-gr - gi * kr) * rinv2, hi = (gr * kr - gi) * rinv2;
      s0r += gr;
      s0i += gi;
      j0r += hr;
      j0i += hi;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        syr[c] += gr * yq[q][c];
        syi[c] += gi * yq[q][c];
        jyr[c] += hr * yq[q][c];
        jyi[c] += hi * yq[q][c];
      }
    }
    const double wp = c_pm_w[p];
    const double* x = xq[p];
    e[0] += wp * s0r;
    e[1] += wp * s0i;
    h[0] += wp * j0r;
    h[1] += wp * j0i;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      e[2 + 2 * c] += wp * s0r * x[c];
      e[3 + 2 * c] += wp * s0i * x[c];
      e[8 + 2 * c] += wp * syr[c];
      e[9 + 2 * c] += wp * syi[c];
      e[14] += wp * x[c] * syr[c];
      e[15] += wp * x[c] * syi[c];
      h[2 + 2 * c] += wp * j0r * x[c];
      h[3 + 2 * c] += wp * j0i * x[c];
      h[8 + 2 * c] += wp * jyr[c];
      h[9 + 2 * c] += wp * jyi[c];
      const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;  // (jy x x)_c
      h[14 + 2 * c] += wp * (jyr[c1] * x[c2] - jyr[c2] * x[c1]);
      h[15 + 2 * c] += wp * (jyi[c1] * x[c2] - jyi[c2] * x[c1]);
    }
  }
  const double scale = m.tri_area[t1] * m.tri_area[t2] * kInv4PiPm;
#pragma unroll
  for (int i = 0; i < 16; ++i) e[i] *= scale;
#pragma unroll
  for (int i = 0; i < 20; ++i) h[i] *= scale;
#pragma unroll 1
  for (int i = 0; i < 3; ++i) {
    double p[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c] = m.verts[3 * v1[i] + c] - o1[c];
    const double c1 = m.tri_coef[3 * t1 + i], d1 = m.tri_div[3 * t1 + i];
    const int64_t row = m.tri_edge[3 * t1 + i];
#pragma unroll 1
    for (int j = 0; j < 3; ++j) {
      double q[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) q[c] = m.verts[3 * v2[j] + c] - o2[c];
      double tr, ti, kr, ki;
      pair_entry(k, e, h, p, q, D, c1 * m.tri_coef[3 * t2 + j], d1 * m.tri_div[3 * t2 + j], tr, ti, kr, ki);
      const int64_t off = 2 * (row * ldz + m.tri_edge[3 * t2 + j]);
      atomic_add_z(ZT + off, tr, ti);
      atomic_add_z(ZK + off, kr, ki);
    }
  }
}

// ------------------------------------------------------------------ singular pairs
// One touching pair per warp (four per CTA): the lanes share the Sauter-Schwab 4-cube
// points (Sauter & Schwab, Boundary Element Methods, Section 5.2: six maps for identical,
// five for edge-adjacent, two for vertex-adjacent pairs), a butterfly reduction leaves the
// 36 moments in every lane, and lanes 0-8 form one entry each of the two 3 x 3 blocks and
// add it and its mirror (both blocks are symmetric under exchanging the triangles).
__device__ __forceinline__ void pm_chi(const double E[2][3], double u1, double u2, double out[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) out[c] = fma(u1, E[0][c], u2 * E[1][c]);
}

__device__ __forceinline__ void pm_accumulate(double k, bool mfio, const double x[3], const double y[3], double w,
                                              double acc[36]) {
  const double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
  const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
  const double rinv = rsqrt(r2);
  const double r = r2 * rinv;
  double sn, cs;
  sincos(k * r, &sn, &cs);
  const double g = w * rinv;
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
  const double xy = x[0] * y[0] + x[1] * y[1] + x[2] * y[2];
  acc[14] += gr * xy;
  acc[15] += gi * xy;
  if (!mfio) return;
  const double kr = k * r, rinv2 = rinv * rinv;
  const double hr = (-gr - gi * kr) * rinv2, hi = (gr * kr - gi) * rinv2;
  double* h = acc + 16;
  h[0] += hr;
  h[1] += hi;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
    const double yx = y[c1] * x[c2] - y[c2] * x[c1];  // (y x x)_c
    h[2 + 2 * c] += hr * x[c];
    h[3 + 2 * c] += hi * x[c];
    h[8 + 2 * c] += hr * y[c];
    h[9 + 2 * c] += hi * y[c];
    h[14 + 2 * c] += hr * yx;
    h[15 + 2 * c] += hi * yx;
  }
}

__global__ void __launch_bounds__(128) pmchwt_singular_kernel(DevMesh m, double k, int nss, double* ZT, double* ZK,
                                                              int64_t ldz) {
  const int64_t pair = int64_t(blockIdx.x) * 4 + (threadIdx.x >> 5);
  if (pair >= m.ntouch) return;
  const int lane = threadIdx.x & 31;
  const TouchPair tp = m.touch[pair];
  const bool mfio = tp.kind != 3;
  double P[3][3], Q[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      P[a][c] = m.verts[3 * tp.p[a] + c];
      Q[a][c] = m.verts[3 * tp.q[a] + c];
    }
  // P0 == Q0 for every touching kind: coordinates relative to it, D = 0
  double EP[2][3], EQ[2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    EP[0][c] = P[1][c] - P[0][c];
    EP[1][c] = P[2][c] - P[1][c];
    EQ[0][c] = Q[1][c] - Q[0][c];
    EQ[1][c] = Q[2][c] - Q[1][c];
  }
  const int n2 = nss * nss, n4 = n2 * n2;
  double acc[36];
#pragma unroll
  for (int i = 0; i < 36; ++i) acc[i] = 0.0;
  for (int idx = lane; idx < n4; idx += 32) {
    const int a = idx / (n2 * nss), b = (idx / n2) % nss, c = (idx / nss) % nss, d = idx % nss;
    const double xi = c_pm_glx[a], e1 = c_pm_glx[b], e2 = c_pm_glx[c], e3 = c_pm_glx[d];
    const double w4 = c_pm_glw[a] * c_pm_glw[b] * c_pm_glw[c] * c_pm_glw[d];
    double x[3], y[3];
    if (tp.kind == 3) {
      const double w = w4 * xi * xi * xi * e1 * e1 * e2;
      const double s[6][4] = {
          {xi, xi * (1 - e1 + e1 * e2), xi * (1 - e1 * e2 * e3), xi * (1 - e1)},
          {xi * (1 - e1 * e2 * e3), xi * (1 - e1), xi, xi * (1 - e1 + e1 * e2)},
          {xi, xi * e1 * (1 - e2 + e2 * e3), xi * (1 - e1 * e2), xi * e1 * (1 - e2)},
          {xi * (1 - e1 * e2), xi * e1 * (1 - e2), xi, xi * e1 * (1 - e2 + e2 * e3)},
          {xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), xi, xi * e1 * (1 - e2)},
          {xi, xi * e1 * (1 - e2), xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)}};
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        pm_chi(EP, s[j][0], s[j][1], x);
        pm_chi(EQ, s[j][2], s[j][3], y);
        pm_accumulate(k, false, x, y, w, acc);
      }
    } else if (tp.kind == 2) {
      const double w0 = w4 * xi * xi * xi * e1 * e1, w1 = w0 * e2;
      const double s[5][5] = {
          {xi, xi * e1 * e3, xi * (1 - e1 * e2), xi * e1 * (1 - e2), w0},
          {xi, xi * e1, xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3), w1},
          {xi * (1 - e1 * e2), xi * e1 * (1 - e2), xi, xi * e1 * e2 * e3, w1},
          {xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3), xi, xi * e1, w1},
          {xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3), xi, xi * e1 * e2, w1}};
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        pm_chi(EP, s[j][0], s[j][1], x);
        pm_chi(EQ, s[j][2], s[j][3], y);
        pm_accumulate(k, true, x, y, s[j][4], acc);
      }
    } else {
      const double w = w4 * xi * xi * xi * e2;
      pm_chi(EP, xi, xi * e1, x);
      pm_chi(EQ, xi * e2, xi * e2 * e3, y);
      pm_accumulate(k, true, x, y, w, acc);
      pm_chi(EP, xi * e2, xi * e2 * e3, x);
      pm_chi(EQ, xi, xi * e1, y);
      pm_accumulate(k, true, x, y, w, acc);
    }
  }
#pragma unroll
  for (int i = 0; i < 36; ++i) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], off);
  }
  if (lane >= 9) return;
  const int i = lane / 3, j = lane % 3;
  const int t1 = tp.t1, t2 = tp.t2;
  const double jac = 4.0 * m.tri_area[t1] * m.tri_area[t2] * kInv4PiPm;
#pragma unroll
  for (int q = 0; q < 36; ++q) acc[q] *= jac;
  const int va = m.tris[3 * t1 + i], vb = m.tris[3 * t2 + j];
  double p[3], q[3];
  const double D[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    p[c] = m.verts[3 * va + c] - P[0][c];
    q[c] = m.verts[3 * vb + c] - Q[0][c];
  }
  double tr, ti, kr, ki;
  pair_entry(k, acc, acc + 16, p, q, D, m.tri_coef[3 * t1 + i] * m.tri_coef[3 * t2 + j],
             m.tri_div[3 * t1 + i] * m.tri_div[3 * t2 + j], tr, ti, kr, ki);
  if (!mfio) kr = ki = 0.0;
  const int64_t e1 = m.tri_edge[3 * t1 + i], e2 = m.tri_edge[3 * t2 + j];
  atomic_add_z(ZT + 2 * (e1 * ldz + e2), tr, ti);
  atomic_add_z(ZK + 2 * (e1 * ldz + e2), kr, ki);
  if (t1 != t2) {
    atomic_add_z(ZT + 2 * (e2 * ldz + e1), tr, ti);
    atomic_add_z(ZK + 2 * (e2 * ldz + e1), kr, ki);
  }
}

// ------------------------------------------------------------------ block combination
// (1,2) = T_0 + eta T_1, (2,1) = -T_0 - T_1/eta, (2,2) = (1,1); T_0 in (1,2), T_1 in (2,2).
__global__ void pmchwt_combine_kernel(int64_t N, double eta, double2* Z, int64_t ldz) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= N * N) return;
  const int64_t r = e / N, c = e % N;
  const double2 kk = Z[r * ldz + c];
  const double2 t0 = Z[r * ldz + N + c];
  const double2 t1 = Z[(N + r) * ldz + N + c];
  const double ie = 1.0 / eta;
  Z[r * ldz + N + c] = make_double2(t0.x + eta * t1.x, t0.y + eta * t1.y);
  Z[(N + r) * ldz + c] = make_double2(-t0.x - ie * t1.x, -t0.y - ie * t1.y);
  Z[(N + r) * ldz + N + c] = kk;
}

// ------------------------------------------------------------------ far field
// A (3 n_dir x 2N, row-major): with v_n = int f_n(y) exp(-ik xh.y) dy,
//   A[3d + c, n] = -ik (xh x v_n)_c,  A[3d + c, N + n] = -ik ((I - xh xh^T) v_n)_c,
// from E_sc = -E_k m - H_k j outside (Section II-C); one thread per (triangle, direction).
__global__ void pmchwt_farfield_kernel(DevMesh m, double k, const double* dirs, int64_t n_dir, double* A) {
  const int64_t gid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gid >= m.nt * n_dir) return;
  const int64_t t = gid / n_dir, d = gid % n_dir;
  const int64_t N = m.ne, ld = 2 * m.ne;
  const double u[3] = {dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2]};
  double Jr[3][3] = {}, Ji[3][3] = {};
  for (int qp = 0; qp < 6; ++qp) {
    const double* y = m.tri_qp + 18 * t + 3 * qp;
    double sn, cs;
    sincos(-k * (u[0] * y[0] + u[1] * y[1] + u[2] * y[2]), &sn, &cs);
    for (int i = 0; i < 3; ++i) {
      const int pv = m.tris[3 * t + i];
      for (int c = 0; c < 3; ++c) {
        const double f = (y[c] - m.verts[3 * pv + c]) * m.tri_coef[3 * t + i] * c_pm_w[qp];
        Jr[i][c] += f * cs;
        Ji[i][c] += f * sn;
      }
    }
  }
  const double At = m.tri_area[t];
  for (int i = 0; i < 3; ++i) {
    const double uJr = u[0] * Jr[i][0] + u[1] * Jr[i][1] + u[2] * Jr[i][2];
    const double uJi = u[0] * Ji[i][0] + u[1] * Ji[i][1] + u[2] * Ji[i][2];
    const int64_t n = m.tri_edge[3 * t + i];
    for (int c = 0; c < 3; ++c) {
      const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
      const double Xr = (u[c1] * Jr[i][c2] - u[c2] * Jr[i][c1]) * At, Xi = (u[c1] * Ji[i][c2] - u[c2] * Ji[i][c1]) * At;
      const double Tr = (Jr[i][c] - u[c] * uJr) * At, Ti = (Ji[i][c] - u[c] * uJi) * At;
      // -ik (a + i b) = k b - i k a
      atomic_add_z(A + 2 * ((3 * d + c) * ld + n), k * Xi, -k * Xr);
      atomic_add_z(A + 2 * ((3 * d + c) * ld + N + n), k * Ti, -k * Tr);
    }
  }
}

inline unsigned pm_blocks(int64_t n, int bs) { return unsigned((n + bs - 1) / bs); }

cudaError_t assemble_pmchwt_one_k(const DevMesh& d, double k, int nss, int arith, double* ZT, double* ZK,
                                  int64_t ldz, cudaStream_t s) {
  {
    ProfScope prof("pmchwt_regular", s, 36.0 * (double(d.nt) * double(d.nt) - double(2 * d.ntouch - d.nt)));
    cudaError_t e;
    if (arith == FOSB_ASM_FF) {
      e = launch_pmchwt_regular_ff(d, k, ZT, ZK, ldz, s);
    } else {
      dim3 grid(pm_blocks(d.nt, 32), pm_blocks(d.nt, 8));
      pmchwt_regular_kernel<<<grid, 256, 0, s>>>(d, k, ZT, ZK, ldz);
      e = launched();
    }
    if (e != cudaSuccess) return e;
  }
  if (d.ntouch == 0) return cudaSuccess;
  ProfScope prof("pmchwt_singular", s, double(d.ntouch));
  pmchwt_singular_kernel<<<pm_blocks(d.ntouch, 4), 128, 0, s>>>(d, k, nss, ZT, ZK, ldz);
  return launched();
}

}  // namespace

void upload_rules_pmchwt(const Rules& r) {
  cudaMemcpyToSymbol(c_pm_bary, r.bary, sizeof(r.bary));
  cudaMemcpyToSymbol(c_pm_w, r.w, sizeof(r.w));
  cudaMemcpyToSymbol(c_pm_glx, r.glx, sizeof(r.glx));
  cudaMemcpyToSymbol(c_pm_glw, r.glw, sizeof(r.glw));
}

}  // namespace fosb

using namespace fosb;

extern "C" {

fosb_status fosb_assemble_pmchwt(fosb_mesh mesh, double k0, double eps_r, double mu_r, const fosb_quad_opts* opts,
                                 void* Z, int64_t ldz, const double* inc, int64_t n_inc, void* b, int64_t ldb,
                                 void* stream) {
  if (!mesh || !Z) return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_pmchwt: NULL mesh or Z");
  const int64_t N = mesh->d.ne;
  if (!(k0 > 0.0) || !std::isfinite(k0)) return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_pmchwt: k0 must be > 0");
  if (!(eps_r > 0.0) || !std::isfinite(eps_r) || !(mu_r > 0.0) || !std::isfinite(mu_r))
    return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_pmchwt: eps_r and mu_r must be finite and > 0");
  if (ldz < 2 * N) return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_pmchwt: ldz < 2N");
  if (n_inc < 0 || (n_inc > 0 && (!inc || !b || ldb < n_inc)))
    return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_pmchwt: bad incidence arguments");
  const int nss = opts && opts->n_ss > 0 ? opts->n_ss : 5;
  if (nss > 12) return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_pmchwt: n_ss must be in 1..12");
  const int arith = opts ? opts->arith : FOSB_ASM_FP64;
  if (arith != FOSB_ASM_FP64 && arith != FOSB_ASM_FF)
    return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_pmchwt: arith must be FOSB_ASM_FP64 or FOSB_ASM_FF");
  if (mesh->d.nt > int64_t(65535) * 4) return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_pmchwt: too many triangles");
  for (int64_t s = 0; s < n_inc; ++s)
    for (int c = 0; c < 9; ++c)
      if (!std::isfinite(inc[9 * s + c])) return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_pmchwt: non-finite incidence");
  FOSB_TRY(ensure_rules_for(nss));
  const double k1 = k0 * std::sqrt(eps_r * mu_r), eta = std::sqrt(mu_r / eps_r);
  if (arith == FOSB_ASM_FF && std::max(k0, k1) * mesh->d.diameter >= ff_max_phase())
    return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_pmchwt: max(k0, k1) * mesh diameter = " +
                                          std::to_string(std::max(k0, k1) * mesh->d.diameter) +
                                          " exceeds the float-float phase range " + std::to_string(ff_max_phase()) +
                                          "; use FOSB_ASM_FP64");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* z = static_cast<double*>(Z);
  double* z11 = z;
  double* z12 = z + 2 * N;
  double* z22 = z + 2 * (N * ldz + N);
  FOSB_CUDA(cudaMemset2DAsync(Z, ldz * 16, 0, 2 * N * 16, 2 * N, s));
  FOSB_CUDA(assemble_pmchwt_one_k(mesh->d, k0, nss, arith, z12, z11, ldz, s));
  FOSB_CUDA(assemble_pmchwt_one_k(mesh->d, k1, nss, arith, z22, z11, ldz, s));
  pmchwt_combine_kernel<<<pm_blocks(N * N, 256), 256, 0, s>>>(N, eta, static_cast<double2*>(Z), ldz);
  FOSB_CUDA(launched());
  if (n_inc > 0) {
    // rows d, Re p, Im p for the Dirichlet data and d, Re(d x p), Im(d x p) for the Neumann
    // data (curl E_inc / (ik0) = (d x p) exp(ik0 d.x)); a pageable copy of our own, so the
    // call needs no synchronisation whatever memory `inc` is in
    std::vector<double> h(18 * n_inc);
    for (int64_t i = 0; i < n_inc; ++i) {
      const double* c = inc + 9 * i;
      double* a = h.data() + 9 * i;
      double* bb = h.data() + 9 * (n_inc + i);
      for (int t = 0; t < 9; ++t) a[t] = c[t];
      bb[0] = c[0];
      bb[1] = c[1];
      bb[2] = c[2];
      for (int part = 0; part < 2; ++part) {
        const double* p = c + 3 + 3 * part;
        double* o = bb + 3 + 3 * part;
        o[0] = c[1] * p[2] - c[2] * p[1];
        o[1] = c[2] * p[0] - c[0] * p[2];
        o[2] = c[0] * p[1] - c[1] * p[0];
      }
    }
    Scratch dinc(s);
    FOSB_CUDA(dinc.alloc(sizeof(double) * h.size()));
    FOSB_CUDA(cudaMemcpyAsync(dinc.p, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, s));
    FOSB_CUDA(cudaMemset2DAsync(b, ldb * 16, 0, n_inc * 16, 2 * N, s));
    FOSB_CUDA(launch_rhs(mesh->d, k0, dinc.as<double>(), n_inc, false, b, ldb, s));
    FOSB_CUDA(launch_rhs(mesh->d, k0, dinc.as<double>() + 9 * n_inc, n_inc, false,
                         static_cast<double*>(b) + 2 * N * ldb, ldb, s));
  }
  return FOSB_OK;
}

fosb_status fosb_farfield_pmchwt(fosb_mesh mesh, double k0, const double* dirs, int64_t n_dir, const void* X,
                                 int64_t ldx, int64_t ncols, double weight, void* out, int64_t ldo, int accumulate,
                                 void* stream) {
  if (!mesh || !dirs || !X || !out || n_dir <= 0 || ncols <= 0)
    return fail(FOSB_ERR_INVALID_ARG, "fosb_farfield_pmchwt: NULL argument or empty size");
  if (!(k0 > 0.0) || !std::isfinite(k0)) return fail(FOSB_ERR_INVALID_ARG, "fosb_farfield_pmchwt: k0 must be > 0");
  if (ldx < ncols || ldo < ncols) return fail(FOSB_ERR_INVALID_ARG, "fosb_farfield_pmchwt: bad leading dimension");
  for (int64_t i = 0; i < 3 * n_dir; ++i)
    if (!std::isfinite(dirs[i])) return fail(FOSB_ERR_INVALID_ARG, "fosb_farfield_pmchwt: non-finite direction");
  FOSB_TRY(ensure_rules_for(5));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t N2 = 2 * mesh->d.ne, nd3 = 3 * n_dir;
  Scratch ddirs(s), a(s);
  FOSB_CUDA(ddirs.alloc(sizeof(double) * 3 * n_dir));
  FOSB_CUDA(cudaMemcpyAsync(ddirs.p, dirs, sizeof(double) * 3 * n_dir, cudaMemcpyHostToDevice, s));
  FOSB_CUDA(a.alloc(16 * nd3 * N2));
  FOSB_CUDA(cudaMemsetAsync(a.p, 0, 16 * nd3 * N2, s));
  pmchwt_farfield_kernel<<<pm_blocks(mesh->d.nt * n_dir, 128), 128, 0, s>>>(mesh->d, k0, ddirs.as<double>(), n_dir,
                                                                           a.as<double>());
  FOSB_CUDA(launched());
  FOSB_CUDA(gemm<double>(OP_N, OP_N, nd3, ncols, N2, weight, 0.0, a.p, N2, X, ldx, accumulate ? 1.0 : 0.0, out, ldo, s));
  FOSB_CUDA(cudaStreamSynchronize(s));
  return FOSB_OK;
}

}  // extern "C"
