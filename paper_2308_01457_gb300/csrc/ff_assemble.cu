// Regular-pair EFIE assembly in float-float arithmetic on the FP32 pipe.
//
// GB300 issues FP64 at about 1/70 of its FP32 rate, so the FP64 kernel of assemble.cu is
// bound by the FP64 pipe.  Here every quantity of the point-pair loop is an unevaluated
// sum hi + lo of two floats (about 48 significant bits) built from error-free
// transformations (two-sum, FMA two-product); no FP64 instruction remains in the loop.
//
// Per point pair (x_p on the test triangle, y_q on the trial triangle):
//   d = (o1 - o2) + (x_p - o1) - (y_q - o2);  r = |d| (rsqrt seed + one Newton step);
//   1/r (Newton step on the seed); theta = k r;
//   exp(i theta): theta = j pi/64 + delta (Cody-Waite with a 3-part pi/64, j < 1024),
//   sin/cos(delta) by Taylor series to delta^7 (|delta| <= pi/128) in float-float for
//   the leading terms, combined with a 128-entry table of sin/cos(j pi/64);
//   G0 = exp(i theta)/r.
// The pair's 3 x 3 barycentric moment matrix
//   mu_ab = sum_pq w_p w_q lambda_pa beta_qb G0(x_p, y_q)
// determines the RWG block exactly (with P_a, Q_b the vertices):
//   Z_ij = (s_i l_i s'_j l'_j / (4 pi)) [ -(ik/4) sum_ab mu_ab (P_a - P_i).(Q_b - Q_j) + (i/k) sum_ab mu_ab ],
// which is formed in float-float and added to the complex128 Z with FP64 atomics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fosb_internal.h"

namespace fosb {
namespace {

struct ff {
  float h, l;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {  // accurate
  ff s = two_sum(a.h, b.h);
  ff t = two_sum(a.l, b.l);
  s.l += t.h;
  s = fast_two_sum(s.h, s.l);
  s.l += t.l;
  return fast_two_sum(s.h, s.l);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }
__device__ __forceinline__ ff ff_add_fast(ff a, ff b) {  // sloppy: fine without cancellation
  ff s = two_sum(a.h, b.h);
  s.l += a.l + b.l;
  return fast_two_sum(s.h, s.l);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  float p = a.h * b;
  float e = fmaf(a.h, b, -p);
  e = fmaf(a.l, b, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_sqr(ff a) {
  float p = a.h * a.h;
  float e = fmaf(a.h, a.h, -p);
  e = fmaf(2.0f * a.h, a.l, e);
  return fast_two_sum(p, e);
}
// acc += a * c (compensated; acc is renormalised by the caller when read)
__device__ __forceinline__ void acc_mul(ff& acc, ff a, ff c) {
  float p = a.h * c.h;
  float pe = fmaf(a.h, c.h, -p);
  pe = fmaf(a.h, c.l, fmaf(a.l, c.h, pe));
  float s = acc.h + p;
  float bb = s - acc.h;
  float e = (acc.h - (s - bb)) + (p - bb);
  acc.h = s;
  acc.l += e + pe;
}
__device__ __forceinline__ ff norm(ff a) { return fast_two_sum(a.h, a.l); }
__device__ __forceinline__ double to_d(ff a) { return double(a.h) + double(a.l); }

struct CFF {
  ff r, i;
};

// constants: sin / cos (j pi / 64), j = 0..127, as (S.h, S.l, C.h, C.l); w_q beta_qb as ff
__constant__ float c_sctab[128][4];
__constant__ float c_wb[6][3][2];

struct FFConst {
  ff k, k4, kinv, inv4pi, sixth;
  float c1, c2, c3, inv_c;  // pi/64 = c1 + c2 + c3 (c1, c2 with <= 14 significant bits); 64/pi
};

__device__ __forceinline__ ff ldff(const float* base, int64_t nt, int f, int64_t t) {
  return {base[int64_t(f) * nt + t], base[int64_t(f + 1) * nt + t]};
}

// exp(i theta) for theta = th + tl >= 0, |j| < 1024, table in shared memory
__device__ __forceinline__ void expi_ff(ff theta, const FFConst& C, const float (*tab)[4], ff& cs, ff& sn) {
  const float jf = rintf(theta.h * C.inv_c);
  const int j = int(jf);
  float a = fmaf(-jf, C.c1, theta.h);  // exact
  ff dl = two_sum(a, -jf * C.c2);      // jf * c2 exact
  dl.l += theta.l - jf * C.c3;
  dl = fast_two_sum(dl.h, dl.l);
  const ff d2 = ff_sqr(dl);
  const float d2h = d2.h;
  // sin(delta) = delta (1 - d2/6 + d2^2/120 - d2^3/5040)
  ff t = ff_mul(d2, C.sixth);
  ff ps = fast_two_sum(1.0f, -t.h);
  ps.l += -t.l + d2h * d2h * (1.0f / 120.0f - d2h * (1.0f / 5040.0f));
  ps = norm(ps);
  const ff sd = ff_mul(dl, ps);
  // cos(delta) = 1 - d2/2 + d2^2/24 - d2^3/720
  ff cd = fast_two_sum(1.0f, -0.5f * d2.h);
  cd.l += -0.5f * d2.l + d2h * d2h * (1.0f / 24.0f - d2h * (1.0f / 720.0f));
  cd = norm(cd);
  const int idx = j & 127;
  const ff S = {tab[idx][0], tab[idx][1]}, Cc = {tab[idx][2], tab[idx][3]};
  sn = ff_add_fast(ff_mul(S, cd), ff_mul(Cc, sd));
  cs = ff_add(ff_mul(Cc, cd), ff_neg(ff_mul(S, sd)));
}

// One regular point pair block: test triangle t1, trial triangle t2 (t1, t2 < m.nt); adds the
// 3 x 3 RWG block into Z unless the triangles touch.  tab: the sin/cos table in shared memory.
// MFIO: also the block of the MFIO of the dielectric (PMCHWT) system, into ZK (same ldz):
//   K_ij = -int int (x - y).(f_j(y) x f_i(x)) g,  g = exp(ikr)(ikr - 1)/(4 pi r^3).
// With a = x - p_i, b = y - q_j, (x - y).(b x a) = (p_i - q_j).(b x a) is bilinear in the
// barycentric coordinates, so the pair's second moment matrix
//   nu_ab = sum_pq w_p w_q lambda_pa beta_qb exp(ikr)(ikr - 1)/r^3
// gives K_ij = -(s_i l_i s'_j l'_j / (16 pi)) sum_ab nu_ab (p_i - q_j).((Q_b - q_j) x (P_a - p_i)).
template <bool MFIO>
__device__ __forceinline__ void regular_ff_pair(const DevMesh& m, const FFConst& C, double* Z, double* ZK,
                                                int64_t ldz, int64_t t1, int64_t t2, const float (*tab)[4]) {
  const int64_t nt = m.nt;
  int v1[3], v2[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    v1[a] = m.tris[3 * t1 + a];
    v2[a] = m.tris[3 * t2 + a];
  }
  bool touch = false;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) touch |= v1[a] == v2[b];
  if (touch) return;
  const float* F = m.tri_ff;
  ff D[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) D[c] = ff_add(ldff(F, nt, 36 + 2 * c, t1), ff_neg(ldff(F, nt, 36 + 2 * c, t2)));
  CFF mu[3][3], nu[MFIO ? 3 : 1][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) mu[a][b] = CFF{{0.f, 0.f}, {0.f, 0.f}};
  if constexpr (MFIO) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) nu[a][b] = CFF{{0.f, 0.f}, {0.f, 0.f}};
  }
#pragma unroll 1
  for (int p = 0; p < 6; ++p) {
    ff E[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) E[c] = ff_add(D[c], ldff(F, nt, (p * 3 + c) * 2, t1));
    CFF A[3], B[MFIO ? 3 : 1];
#pragma unroll
    for (int b = 0; b < 3; ++b) A[b] = CFF{{0.f, 0.f}, {0.f, 0.f}};
    if constexpr (MFIO) {
#pragma unroll
      for (int b = 0; b < 3; ++b) B[b] = CFF{{0.f, 0.f}, {0.f, 0.f}};
    }
    // two point pairs per iteration: enough independent work per warp, a third of the code
    // of a full unroll (instruction fetch bounded the fully unrolled loop)
#pragma unroll 2
    for (int q = 0; q < 6; ++q) {
      ff dx = ff_add_fast(E[0], ff_neg(ldff(F, nt, (q * 3 + 0) * 2, t2)));
      ff dy = ff_add_fast(E[1], ff_neg(ldff(F, nt, (q * 3 + 1) * 2, t2)));
      ff dz = ff_add_fast(E[2], ff_neg(ldff(F, nt, (q * 3 + 2) * 2, t2)));
      ff r2 = ff_add_fast(ff_add_fast(ff_sqr(dx), ff_sqr(dy)), ff_sqr(dz));
      const float y0 = rsqrtf(r2.h);
      const float s0 = r2.h * y0;
      const float er = fmaf(-s0, s0, r2.h) + r2.l;
      const ff r = fast_two_sum(s0, er * (0.5f * y0));
      const ff rq = ff_mul_f(r, y0);                     // r * y0 ~ 1
      const float corr = ((1.0f - rq.h) - rq.l) * y0;    // 1 - rq.h exact (rq.h ~ 1)
      const ff rinv = fast_two_sum(y0, corr);
      ff cs, sn;
      const ff kr = ff_mul(C.k, r);
      expi_ff(kr, C, tab, cs, sn);
      const CFF G = {ff_mul(cs, rinv), ff_mul(sn, rinv)};
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const ff wb = {c_wb[q][b][0], c_wb[q][b][1]};
        acc_mul(A[b].r, G.r, wb);
        acc_mul(A[b].i, G.i, wb);
      }
      if constexpr (MFIO) {
        // g = G (ikr - 1) / r^2: Re = -(G.r + G.i kr) / r^2, Im = (G.r kr - G.i) / r^2
        const ff rinv2 = ff_sqr(rinv);
        const CFF g = {ff_neg(ff_mul(ff_add(G.r, ff_mul(G.i, kr)), rinv2)),
                       ff_mul(ff_add(ff_mul(G.r, kr), ff_neg(G.i)), rinv2)};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const ff wb = {c_wb[q][b][0], c_wb[q][b][1]};
          acc_mul(B[b].r, g.r, wb);
          acc_mul(B[b].i, g.i, wb);
        }
      }
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      A[b].r = norm(A[b].r);
      A[b].i = norm(A[b].i);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const ff wa = {c_wb[p][a][0], c_wb[p][a][1]};
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        acc_mul(mu[a][b].r, A[b].r, wa);
        acc_mul(mu[a][b].i, A[b].i, wa);
      }
    }
    if constexpr (MFIO) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        B[b].r = norm(B[b].r);
        B[b].i = norm(B[b].i);
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const ff wa = {c_wb[p][a][0], c_wb[p][a][1]};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          acc_mul(nu[a][b].r, B[b].r, wa);
          acc_mul(nu[a][b].i, B[b].i, wa);
        }
      }
    }
  }
  // epilogue: edge vectors e_a = P_{a+1} - P_a (a mod 3), relative to vertex 0
  ff P1[3], P2[3], Q1[3], Q2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    P1[c] = ldff(F, nt, 42 + 2 * c, t1);
    P2[c] = ldff(F, nt, 48 + 2 * c, t1);
    Q1[c] = ldff(F, nt, 42 + 2 * c, t2);
    Q2[c] = ldff(F, nt, 48 + 2 * c, t2);
  }
  ff eP[3][3], eQ[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    eP[0][c] = P1[c];
    eP[1][c] = ff_add(P2[c], ff_neg(P1[c]));
    eP[2][c] = ff_neg(P2[c]);
    eQ[0][c] = Q1[c];
    eQ[1][c] = ff_add(Q2[c], ff_neg(Q1[c]));
    eQ[2][c] = ff_neg(Q2[c]);
  }
  ff DP[3][3];
#pragma unroll
  for (int al = 0; al < 3; ++al)
#pragma unroll
    for (int be = 0; be < 3; ++be) {
      ff s = ff_mul(eP[al][0], eQ[be][0]);
      s = ff_add(s, ff_mul(eP[al][1], eQ[be][1]));
      DP[al][be] = ff_add(s, ff_mul(eP[al][2], eQ[be][2]));
    }
  CFF I0 = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      mu[a][b].r = norm(mu[a][b].r);
      mu[a][b].i = norm(mu[a][b].i);
      I0.r = ff_add(I0.r, mu[a][b].r);
      I0.i = ff_add(I0.i, mu[a][b].i);
    }
  ff sl1[3], sl2[3];
  int e1[3], e2[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    sl1[i] = ldff(F, nt, 54 + 2 * i, t1);
    sl2[i] = ldff(F, nt, 54 + 2 * i, t2);
    e1[i] = m.tri_edge[3 * t1 + i];
    e2[i] = m.tri_edge[3 * t2 + i];
  }
  // (P_a - P_i) = +e_i for a = i+1, -e_{i+2} for a = i+2 (indices mod 3)
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int a1 = (i + 1) % 3, a2 = (i + 2) % 3;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int b1 = (j + 1) % 3, b2 = (j + 2) % 3;
      CFF V = {{0.f, 0.f}, {0.f, 0.f}};
      acc_mul(V.r, mu[a1][b1].r, DP[i][j]);
      acc_mul(V.i, mu[a1][b1].i, DP[i][j]);
      acc_mul(V.r, mu[a1][b2].r, ff_neg(DP[i][b2]));
      acc_mul(V.i, mu[a1][b2].i, ff_neg(DP[i][b2]));
      acc_mul(V.r, mu[a2][b1].r, ff_neg(DP[a2][j]));
      acc_mul(V.i, mu[a2][b1].i, ff_neg(DP[a2][j]));
      acc_mul(V.r, mu[a2][b2].r, DP[a2][b2]);
      acc_mul(V.i, mu[a2][b2].i, DP[a2][b2]);
      V.r = norm(V.r);
      V.i = norm(V.i);
      // -(ik/4) V + (i/k) I0 = [(k/4) V.i - (1/k) I0.i] + i [-(k/4) V.r + (1/k) I0.r]
      const ff zr = ff_add(ff_mul(C.k4, V.i), ff_neg(ff_mul(C.kinv, I0.i)));
      const ff zi = ff_add(ff_mul(C.kinv, I0.r), ff_neg(ff_mul(C.k4, V.r)));
      const ff sig = ff_mul(ff_mul(sl1[i], sl2[j]), C.inv4pi);
      double* dst = Z + 2 * (int64_t(e1[i]) * ldz + e2[j]);
      atomicAdd(dst, to_d(ff_mul(sig, zr)));
      atomicAdd(dst + 1, to_d(ff_mul(sig, zi)));
    }
  }
  if constexpr (MFIO) {
    // X[be][al] = eQ_be x eP_al;  (P_a - p_i) = eP_i (a = i+1), -eP_{i+2} (a = i+2), and the same for Q
    ff X[3][3][3];
#pragma unroll
    for (int be = 0; be < 3; ++be)
#pragma unroll
      for (int al = 0; al < 3; ++al)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
          X[be][al][c] = ff_add(ff_mul(eQ[be][c1], eP[al][c2]), ff_neg(ff_mul(eQ[be][c2], eP[al][c1])));
        }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        nu[a][b].r = norm(nu[a][b].r);
        nu[a][b].i = norm(nu[a][b].i);
      }
    const ff zero = {0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int a1 = (i + 1) % 3, a2 = (i + 2) % 3;
      // p_i - P_0 (vertex i relative to vertex 0 of t1)
      ff pi_[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) pi_[c] = i == 0 ? zero : (i == 1 ? P1[c] : P2[c]);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int b1 = (j + 1) % 3, b2 = (j + 2) % 3;
        // d = p_i - q_j = (P_0 - Q_0) + (p_i - P_0) - (q_j - Q_0)
        ff d[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const ff qj = j == 0 ? zero : (j == 1 ? Q1[c] : Q2[c]);
          d[c] = ff_add(ff_add(D[c], pi_[c]), ff_neg(qj));
        }
        auto dot3 = [&](const ff (&x)[3]) {
          ff r = ff_mul(d[0], x[0]);
          r = ff_add(r, ff_mul(d[1], x[1]));
          return ff_add(r, ff_mul(d[2], x[2]));
        };
        // (a, b) = (a1, b1), (a1, b2), (a2, b1), (a2, b2)
        const ff t[4] = {dot3(X[j][i]), ff_neg(dot3(X[b2][i])), ff_neg(dot3(X[j][a2])), dot3(X[b2][a2])};
        CFF V = {{0.f, 0.f}, {0.f, 0.f}};
        acc_mul(V.r, nu[a1][b1].r, t[0]);
        acc_mul(V.i, nu[a1][b1].i, t[0]);
        acc_mul(V.r, nu[a1][b2].r, t[1]);
        acc_mul(V.i, nu[a1][b2].i, t[1]);
        acc_mul(V.r, nu[a2][b1].r, t[2]);
        acc_mul(V.i, nu[a2][b1].i, t[2]);
        acc_mul(V.r, nu[a2][b2].r, t[3]);
        acc_mul(V.i, nu[a2][b2].i, t[3]);
        V.r = norm(V.r);
        V.i = norm(V.i);
        // K_ij = -(s_i l_i s'_j l'_j / (16 pi)) V
        const ff sig = ff_mul(ff_mul(sl1[i], sl2[j]), C.inv4pi);
        const float q4 = -0.25f;
        double* dst = ZK + 2 * (int64_t(e1[i]) * ldz + e2[j]);
        atomicAdd(dst, to_d(ff_mul(sig, V.r)) * q4);
        atomicAdd(dst + 1, to_d(ff_mul(sig, V.i)) * q4);
      }
    }
  }
}

__global__ void __launch_bounds__(128) efie_regular_ff_kernel(DevMesh m, FFConst C, double* Z, int64_t ldz) {
  __shared__ float tab[128][4];
  for (int e = threadIdx.x; e < 128 * 4; e += blockDim.x) tab[e >> 2][e & 3] = c_sctab[e >> 2][e & 3];
  __syncthreads();
  const int64_t t1 = int64_t(blockIdx.y) * 4 + (threadIdx.x >> 5);
  const int64_t t2 = int64_t(blockIdx.x) * 32 + (threadIdx.x & 31);
  if (t1 >= m.nt || t2 >= m.nt) return;
  regular_ff_pair<false>(m, C, Z, nullptr, ldz, t1, t2, tab);
}

// Dielectric (PMCHWT) system: the EFIO block into ZT and the MFIO block into ZK.
__global__ void __launch_bounds__(128, 3) pmchwt_regular_ff_kernel(DevMesh m, FFConst C, double* ZT, double* ZK,
                                                                int64_t ldz) {
  __shared__ float tab[128][4];
  for (int e = threadIdx.x; e < 128 * 4; e += blockDim.x) tab[e >> 2][e & 3] = c_sctab[e >> 2][e & 3];
  __syncthreads();
  const int64_t t1 = int64_t(blockIdx.y) * 4 + (threadIdx.x >> 5);
  const int64_t t2 = int64_t(blockIdx.x) * 32 + (threadIdx.x & 31);
  if (t1 >= m.nt || t2 >= m.nt) return;
  regular_ff_pair<true>(m, C, ZT, ZK, ldz, t1, t2, tab);
}

// Batched form: one persistent launch over the tiles of many meshes.  Tile w of the batch
// (WARPS test triangles x 32 trial triangles) belongs to the item with the largest
// tile_start <= w; CTAs take tiles from a device ticket until the batch is exhausted, so
// meshes of uneven size share the GPU without per-mesh launches.
struct FFBatchItem {
  DevMesh m;
  FFConst C;
  double* Z;
  int64_t ldz;
  int64_t tiles_x;     // ceil(nt / 32)
  int64_t tile_start;  // first tile of this item in the batch
};

template <int WARPS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB) efie_regular_ff_batched_kernel(const FFBatchItem* __restrict__ items,
                                                                             int nitems, int64_t total_tiles,
                                                                             unsigned long long* ticket) {
  __shared__ float tab[128][4];
  __shared__ FFBatchItem s_item;
  __shared__ long long s_tile;
  __shared__ int s_idx;
  for (int e = threadIdx.x; e < 128 * 4; e += blockDim.x) tab[e >> 2][e & 3] = c_sctab[e >> 2][e & 3];
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long w = static_cast<long long>(atomicAdd(ticket, 1ull));
      int lo = 0, hi = nitems - 1;
      if (w < total_tiles)
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (items[mid].tile_start <= w) lo = mid;
          else hi = mid - 1;
        }
      s_tile = w;
      s_idx = lo;
    }
    __syncthreads();
    const long long w = s_tile;
    const int idx = s_idx;
    if (w >= total_tiles) break;
    if (idx != cur) {  // stage the item's record in shared memory (read by every thread)
      __syncthreads();
      const int* src = reinterpret_cast<const int*>(items + idx);
      int* dst = reinterpret_cast<int*>(&s_item);
      for (int e = threadIdx.x; e < int(sizeof(FFBatchItem) / sizeof(int)); e += blockDim.x) dst[e] = src[e];
      cur = idx;
      __syncthreads();
    }
    const int64_t local = w - s_item.tile_start;
    const int64_t ty = local / s_item.tiles_x, tx = local - ty * s_item.tiles_x;
    const int64_t t1 = ty * WARPS + (threadIdx.x >> 5), t2 = tx * 32 + (threadIdx.x & 31);
    if (t1 < s_item.m.nt && t2 < s_item.m.nt)
      regular_ff_pair<false>(s_item.m, s_item.C, s_item.Z, nullptr, s_item.ldz, t1, t2, tab);
    __syncthreads();  // s_tile / s_item are rewritten by the next ticket
  }
}

inline unsigned cdiv(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }

void split(double x, float& h, float& l) {
  h = float(x);
  l = float(x - double(h));
}
ff split_ff(double x) {
  ff r;
  split(x, r.h, r.l);
  return r;
}
// round a double to a float with at most `bits` significant bits
float truncate_bits(double x, int bits) {
  int e;
  double m = std::frexp(x, &e);  // x = m 2^e, 0.5 <= |m| < 1
  double scale = std::ldexp(1.0, bits);
  return float(std::ldexp(std::nearbyint(m * scale) / scale, e));
}

}  // namespace

void upload_rules_ff(const Rules& r) {
  float tab[128][4];
  for (int j = 0; j < 128; ++j) {
    double th = j * M_PI / 64.0;
    split(std::sin(th), tab[j][0], tab[j][1]);
    split(std::cos(th), tab[j][2], tab[j][3]);
  }
  cudaMemcpyToSymbol(c_sctab, tab, sizeof(tab));
  float wb[6][3][2];
  for (int q = 0; q < 6; ++q)
    for (int b = 0; b < 3; ++b) split(r.w[q] * r.bary[q][b], wb[q][b][0], wb[q][b][1]);
  cudaMemcpyToSymbol(c_wb, wb, sizeof(wb));
}

// k * diameter must stay below kFFMaxPhase: the phase index j = rint(k r 64/pi) then
// stays below 1024, which keeps j * c1 and j * c2 exact in FP32.
double ff_max_phase() { return 48.0; }

namespace {
FFConst make_ff_const(double k) {
  FFConst C;
  C.k = split_ff(k);
  C.k4 = split_ff(k / 4.0);
  C.kinv = split_ff(1.0 / k);
  C.inv4pi = split_ff(1.0 / (4.0 * M_PI));
  C.sixth = split_ff(1.0 / 6.0);
  const double pi64 = M_PI / 64.0;
  C.c1 = truncate_bits(pi64, 14);
  C.c2 = truncate_bits(pi64 - double(C.c1), 14);
  C.c3 = float(pi64 - double(C.c1) - double(C.c2));
  C.inv_c = float(64.0 / M_PI);
  return C;
}
}  // namespace

cudaError_t launch_efie_regular_ff(const DevMesh& m, double k, double* Z, int64_t ldz, cudaStream_t s) {
  if (k * m.diameter >= ff_max_phase()) return cudaErrorInvalidValue;
  const FFConst C = make_ff_const(k);
  dim3 grid(cdiv(m.nt, 32), cdiv(m.nt, 4));
  if (grid.y > 65535u) return cudaErrorInvalidValue;
  efie_regular_ff_kernel<<<grid, 128, 0, s>>>(m, C, Z, ldz);
  return launched();
}

// PMCHWT regular pairs for one wavenumber: EFIO blocks into ZT, MFIO blocks into ZK (FP64
// atomics; both N x N blocks of the 2N x 2N matrix with leading dimension ldz).
cudaError_t launch_pmchwt_regular_ff(const DevMesh& m, double k, double* ZT, double* ZK, int64_t ldz, cudaStream_t s) {
  if (k * m.diameter >= ff_max_phase()) return cudaErrorInvalidValue;
  const FFConst C = make_ff_const(k);
  dim3 grid(cdiv(m.nt, 32), cdiv(m.nt, 4));
  if (grid.y > 65535u) return cudaErrorInvalidValue;
  pmchwt_regular_ff_kernel<<<grid, 128, 0, s>>>(m, C, ZT, ZK, ldz);
  return launched();
}

// Regular pairs of a batch of meshes in one persistent launch (see efie_regular_ff_batched_kernel):
// warps = test triangles per tile (4 or 8), min_ctas = the CTAs per SM the register
// allocation is bounded for (4 warps: 5 or 4; 8 warps: 2 or 1); the grid is every resident
// CTA.  Z[i] must be zeroed; scratch: regular_ff_batched_scratch_bytes(nmesh) device bytes.
cudaError_t launch_efie_regular_ff_batched(const DevMesh* const* meshes, const double* ks, double* const* Z,
                                           const int64_t* ldz, int nmesh, int warps, int min_ctas,
                                           void* scratch, size_t scratch_bytes, cudaStream_t s) {
  void (*kern)(const FFBatchItem*, int, int64_t, unsigned long long*) = nullptr;
  if (warps == 4 && min_ctas == 5) kern = efie_regular_ff_batched_kernel<4, 5>;
  else if (warps == 4 && min_ctas == 4) kern = efie_regular_ff_batched_kernel<4, 4>;
  else if (warps == 8 && min_ctas == 2) kern = efie_regular_ff_batched_kernel<8, 2>;
  else if (warps == 8 && min_ctas == 1) kern = efie_regular_ff_batched_kernel<8, 1>;
  if (!kern) return cudaErrorInvalidValue;
  std::vector<FFBatchItem> items(nmesh);
  int64_t total = 0;
  for (int i = 0; i < nmesh; ++i) {
    const DevMesh& m = *meshes[i];
    if (ks[i] * m.diameter >= ff_max_phase()) return cudaErrorInvalidValue;
    items[i].m = m;
    items[i].C = make_ff_const(ks[i]);
    items[i].Z = Z[i];
    items[i].ldz = ldz[i];
    items[i].tiles_x = (m.nt + 31) / 32;
    items[i].tile_start = total;
    total += items[i].tiles_x * ((m.nt + warps - 1) / warps);
  }
  const size_t need = 256 + sizeof(FFBatchItem) * size_t(nmesh);
  if (scratch_bytes < need) return cudaErrorInvalidValue;
  unsigned long long* ticket = static_cast<unsigned long long*>(scratch);
  FFBatchItem* d_items = reinterpret_cast<FFBatchItem*>(static_cast<char*>(scratch) + 256);
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_items, items.data(), sizeof(FFBatchItem) * nmesh, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, warps * 32, 0);
  double pairs = 0.0;
  for (int i = 0; i < nmesh; ++i) pairs += 36.0 * double(meshes[i]->nt) * double(meshes[i]->nt);
  ProfScope prof("asm_regular", s, pairs);
  kern<<<unsigned(nsm * std::max(occ, 1)), warps * 32, 0, s>>>(d_items, nmesh, total, ticket);
  return launched();
}
size_t regular_ff_batched_scratch_bytes(int nmesh) { return 256 + sizeof(FFBatchItem) * size_t(nmesh); }

}  // namespace fosb
