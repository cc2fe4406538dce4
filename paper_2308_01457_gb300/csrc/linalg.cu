// Dense complex linear algebra for the EFIE systems (row-major, interleaved complex).
//
//   * gemm: C = alpha op(A) op(B) + beta C, complex128 or complex64.  A 64 x 64 tiled SIMT
//     kernel for wide products and a row-per-warp kernel for skinny products
//     (<= 8 right-hand sides), which streams A once at HBM speed (IR residuals).
//   * getrf: blocked right-looking LU.  complex64 factors: 256-column blocks, each factored
//     as four 64-column tournament-pivoting panels (tslu.cu) with K = 64 updates between
//     them (tc_gemm.cu), then one tcgen05 3xTF32 trailing update with K = 256 (tc_update.cu,
//     operands split once per block).  complex128 factors: 64-column panels by a
//     cooperative partial-pivoting kernel whose CTAs own row chunks and meet at a software
//     grid barrier once per column (bounded spin: on time-out the status word is set and
//     the kernel returns), then row swaps, the unit-lower solve of the block row and the
//     trailing update (gemm).
//   * getrs: complex64 factors with up to 1024 right-hand sides run one persistent
//     streaming kernel per sweep (trsv_stream.cu); otherwise forward / backward
//     substitution by diagonal-block solves plus gemm updates.
//   * gemm_c128_ff: FP64-class complex128 products in float-float on the FP32 pipe.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "fosb_internal.h"

namespace fosb {
namespace {

template <typename T>
struct C2;
template <>
struct C2<double> {
  using type = double2;
};
template <>
struct C2<float> {
  using type = float2;
};

template <typename T>
__device__ __forceinline__ typename C2<T>::type cmul(typename C2<T>::type a, typename C2<T>::type b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

template <typename T>
__device__ __forceinline__ typename C2<T>::type load_op(const typename C2<T>::type* P, int64_t r, int64_t c, int64_t ld,
                                                        int op) {
  // element (r, c) of op(P): N -> P[r, c]; T -> P[c, r]; C -> conj(P[c, r])
  typename C2<T>::type v = (op == OP_N) ? P[r * ld + c] : P[c * ld + r];
  if (op == OP_C) v.y = -v.y;
  return v;
}

inline unsigned cdiv(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }

// ------------------------------------------------------------------ tiled GEMM
constexpr int TBM = 64, TBN = 64, TBK = 8;

template <typename T>
__global__ void __launch_bounds__(256) gemm_tiled_kernel(int opA, int opB, int64_t M, int64_t N, int64_t K, T ar, T ai,
                                                         const typename C2<T>::type* __restrict__ A, int64_t lda,
                                                         const typename C2<T>::type* __restrict__ B, int64_t ldb, T beta,
                                                         typename C2<T>::type* __restrict__ C, int64_t ldc) {
  using V = typename C2<T>::type;
  __shared__ V As[TBK][TBM + 1];
  __shared__ V Bs[TBK][TBN + 1];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t row0 = int64_t(blockIdx.y) * TBM, col0 = int64_t(blockIdx.x) * TBN;
  V acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = {T(0), T(0)};
  for (int64_t k0 = 0; k0 < K; k0 += TBK) {
    // A tile: 64 rows x 8 k (2 elements per thread)
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      int e = tid + 256 * l;
      int r, kk;
      if (opA == OP_N) {
        r = e / TBK;
        kk = e % TBK;
      } else {
        kk = e / TBM;
        r = e % TBM;
      }
      int64_t gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < M && gk < K) ? load_op<T>(A, gr, gk, lda, opA) : V{T(0), T(0)};
    }
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      int e = tid + 256 * l;
      int c, kk;
      if (opB == OP_N) {
        kk = e / TBN;
        c = e % TBN;
      } else {
        c = e / TBK;
        kk = e % TBK;
      }
      int64_t gc = col0 + c, gk = k0 + kk;
      Bs[kk][c] = (gc < N && gk < K) ? load_op<T>(B, gk, gc, ldb, opB) : V{T(0), T(0)};
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TBK; ++kk) {
      V a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, acc[i][j].x);
          acc[i][j].x = fma(-a[i].y, b[j].y, acc[i][j].x);
          acc[i][j].y = fma(a[i].x, b[j].y, acc[i][j].y);
          acc[i][j].y = fma(a[i].y, b[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t r = row0 + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t c = col0 + tx + 16 * j;
      if (c >= N) continue;
      V v = {ar * acc[i][j].x - ai * acc[i][j].y, ar * acc[i][j].y + ai * acc[i][j].x};
      if (beta != T(0)) {
        V o = C[r * ldc + c];
        v.x += beta * o.x;
        v.y += beta * o.y;
      }
      C[r * ldc + c] = v;
    }
  }
}

// ------------------------------------------------------------------ FP64 GEMM on DMMA
// Complex128 C = alpha op(A) op(B) + beta C with mma.sync.m8n8k4 f64 (the FP64 tensor
// path): each complex product is four real MMAs (Ar Br, -Ai Bi into the real part,
// Ar Bi, Ai Br into the imaginary part).  CTA tile 64 x 64 (complex), k-tile 16, eight
// warps in a 2 x 4 grid, 32 x 16 per warp (4 x 2 fragments of 8 x 8).  Fragment layout
// of m8n8k4: A[g][t], B[t][g], C[g][2t + i] with g = lane / 4, t = lane % 4.
constexpr int DBM = 64, DBN = 64, DBK = 16, DPA = 4, DPB = 2;

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  int sz = valid ? 16 : 0;  // src-size 0: the 16 bytes are zero-filled, nothing is read
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N));
}

constexpr int DSA = DBM * (DBK + DPA), DSB = DBK * (DBN + DPB);  // elements per buffer
constexpr size_t kDmmaSmem = 2 * size_t(DSA + DSB) * sizeof(double2);

// Split-K: blockIdx.z covers k in [z k_chunk, (z + 1) k_chunk); with ATOMIC the partial
// products are added into C with FP64 atomics (C must already hold beta C).  Tiles are
// copied global -> shared with cp.async into two buffers: the next k-tile is in flight
// while the current one is multiplied.  Conjugation (op C) is applied on fragment load.
template <bool ATOMIC>
__global__ void __launch_bounds__(256, 2) zgemm_dmma_kernel(int opA, int opB, int64_t M, int64_t N, int64_t K,
                                                            double ar, double ai, const double2* __restrict__ A,
                                                            int64_t lda, const double2* __restrict__ B, int64_t ldb,
                                                            double beta, double2* __restrict__ C, int64_t ldc,
                                                            int64_t k_chunk) {
  extern __shared__ double2 dsm[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 2, wn = warp & 3;  // warp tile origin (wm * 32, wn * 16)
  const int g = lane >> 2, t = lane & 3;
  const int64_t row0 = int64_t(blockIdx.y) * DBM, col0 = int64_t(blockIdx.x) * DBN;
  const int64_t k_begin = int64_t(blockIdx.z) * k_chunk, k_end = min(K, k_begin + k_chunk);
  const double sa = opA == OP_C ? -1.0 : 1.0, sb = opB == OP_C ? -1.0 : 1.0;
  double cr[4][2][2], ci[4][2][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) cr[i][j][e] = ci[i][j][e] = 0.0;
  auto issue = [&](int64_t k0, int buf) {
    double2* As = dsm + buf * (DSA + DSB);
    double2* Bs = As + DSA;
#pragma unroll
    for (int l = 0; l < 4; ++l) {  // A tile 64 x 16
      int e = tid + 256 * l;
      int r = (opA == OP_N) ? e / DBK : e % DBM;
      int kk = (opA == OP_N) ? e % DBK : e / DBM;
      int64_t gr = row0 + r, gk = k0 + kk;
      bool ok = gr < M && gk < k_end;
      const double2* src = ok ? (opA == OP_N ? A + gr * lda + gk : A + gk * lda + gr) : A;
      cp_async16(As + r * (DBK + DPA) + kk, src, ok);
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) {  // B tile 16 x 64
      int e = tid + 256 * l;
      int c = (opB == OP_N) ? e % DBN : e / DBK;
      int kk = (opB == OP_N) ? e / DBN : e % DBK;
      int64_t gc = col0 + c, gk = k0 + kk;
      bool ok = gc < N && gk < k_end;
      const double2* src = ok ? (opB == OP_N ? B + gk * ldb + gc : B + gc * ldb + gk) : B;
      cp_async16(Bs + kk * (DBN + DPB) + c, src, ok);
    }
  };
  const int64_t ntile = k_end > k_begin ? (k_end - k_begin + DBK - 1) / DBK : 0;
  if (ntile > 0) {
    issue(k_begin, 0);
    cp_async_commit();
  }
  for (int64_t it = 0; it < ntile; ++it) {
    if (it + 1 < ntile) {
      issue(k_begin + (it + 1) * DBK, int((it + 1) & 1));
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const double2* As = dsm + int(it & 1) * (DSA + DSB);
    const double2* Bs = As + DSA;
#pragma unroll
    for (int ks = 0; ks < DBK; ks += 4) {
      double2 a[4], b[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[(wm * 32 + i * 8 + g) * (DBK + DPA) + ks + t];
        a[i].y *= sa;
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        b[j] = Bs[(ks + t) * (DBN + DPB) + wn * 16 + j * 8 + g];
        b[j].y *= sb;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          dmma(cr[i][j][0], cr[i][j][1], a[i].x, b[j].x);
          dmma(cr[i][j][0], cr[i][j][1], -a[i].y, b[j].y);
          dmma(ci[i][j][0], ci[i][j][1], a[i].x, b[j].y);
          dmma(ci[i][j][0], ci[i][j][1], a[i].y, b[j].x);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t r = row0 + wm * 32 + i * 8 + g;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        int64_t c = col0 + wn * 16 + j * 8 + 2 * t + e;
        if (c >= N) continue;
        double xr = cr[i][j][e], xi = ci[i][j][e];
        double2 v = make_double2(ar * xr - ai * xi, ar * xi + ai * xr);
        if constexpr (ATOMIC) {
          atomicAdd(&C[r * ldc + c].x, v.x);
          atomicAdd(&C[r * ldc + c].y, v.y);
        } else {
          if (beta != 0.0) {
            double2 o = C[r * ldc + c];
            v.x += beta * o.x;
            v.y += beta * o.y;
          }
          C[r * ldc + c] = v;
        }
      }
  }
}

// ------------------------------------------------------------------ float-float complex GEMM
// FP64-class products on the FP32 pipe.  Operands arrive split into (hi, lo) float pairs,
// float4 (re.hi, re.lo, im.hi, im.lo) per complex128 element (split_ff_kernel, once per
// element rather than once per tile that reads it); every real product is formed exactly
// with an FMA two-product, accumulated with a two-sum, and the (hi, lo) accumulators are
// renormalised after each k-tile so the low word never grows.  About 44 FP32 instructions
// per complex MAC against ~1 TFLOP/s of FP64 throughput on this part.  Split-K with FP64
// atomics as in the DMMA kernel.
__device__ __forceinline__ void ff_acc(float& h, float& l, float xh, float xl, float yh, float yl) {
  float p = xh * yh;
  float e = fmaf(xh, yh, -p);
  e = fmaf(xh, yl, fmaf(xl, yh, e));
  float s = h + p;
  float bb = s - h;
  l += ((h - (s - bb)) + (p - bb)) + e;
  h = s;
}

__global__ void split_ff_kernel(const double2* __restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                                float4* __restrict__ dst, int64_t ldd) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t i = e / cols, j = e % cols;
  const double2 v = src[i * lds + j];
  const float rh = float(v.x), ih = float(v.y);
  dst[i * ldd + j] = make_float4(rh, float(v.x - double(rh)), ih, float(v.y - double(ih)));
}

// Few right-hand sides (NC <= 8) on a pre-split A (op N): one warp per row, lanes stride
// over k, float-float accumulation renormalised every 16 steps, then a float-float warp
// reduction.  Streams the (hi, lo) split of A once: HBM-bound, where the FP64 row kernel is
// bound by the FP64 pipe.
__device__ __forceinline__ void ff_norm(float& h, float& l) {
  const float s = h + l;
  l = l - (s - h);
  h = s;
}
__device__ __forceinline__ void ff_add_pair(float& h, float& l, float h2, float l2) {
  const float s = h + h2;
  const float bb = s - h;
  const float e = (h - (s - bb)) + (h2 - bb);
  h = s;
  l = l + l2 + e;
  ff_norm(h, l);
}
template <int NC>
__global__ void __launch_bounds__(256) zgemv_ff_kernel(int64_t M, int64_t K, double ar, double ai,
                                                       const float4* __restrict__ A, int64_t lda,
                                                       const float4* __restrict__ B, double beta,
                                                       double2* __restrict__ C, int64_t ldc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row = int64_t(blockIdx.x) * 8 + warp;
  if (row >= M) return;
  float4 acc[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4* a = A + row * lda;
  int step = 0;
  for (int64_t k = lane; k < K; k += 32) {
    const float4 av = __ldcs(a + k);
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const float4 bv = __ldg(B + k * NC + j);
      float4& c = acc[j];
      ff_acc(c.x, c.y, av.x, av.y, bv.x, bv.y);
      ff_acc(c.x, c.y, -av.z, -av.w, bv.z, bv.w);
      ff_acc(c.z, c.w, av.x, av.y, bv.z, bv.w);
      ff_acc(c.z, c.w, av.z, av.w, bv.x, bv.y);
    }
    if (++step == 16) {
      step = 0;
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        ff_norm(acc[j].x, acc[j].y);
        ff_norm(acc[j].z, acc[j].w);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    ff_norm(acc[j].x, acc[j].y);
    ff_norm(acc[j].z, acc[j].w);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float h1 = __shfl_xor_sync(0xffffffffu, acc[j].x, off), l1 = __shfl_xor_sync(0xffffffffu, acc[j].y, off);
      const float h2 = __shfl_xor_sync(0xffffffffu, acc[j].z, off), l2 = __shfl_xor_sync(0xffffffffu, acc[j].w, off);
      ff_add_pair(acc[j].x, acc[j].y, h1, l1);
      ff_add_pair(acc[j].z, acc[j].w, h2, l2);
    }
  }
  if (lane < NC) {
    float4 c = acc[0];
#pragma unroll
    for (int j = 1; j < NC; ++j)
      if (lane == j) c = acc[j];
    const double xr = double(c.x) + double(c.y), xi = double(c.z) + double(c.w);
    double2 v = make_double2(ar * xr - ai * xi, ar * xi + ai * xr);
    if (beta != 0.0) {
      const double2 o = C[row * ldc + lane];
      v.x += beta * o.x;
      v.y += beta * o.y;
    }
    C[row * ldc + lane] = v;
  }
}

// NJ complex columns per thread: tile 64 x 16 NJ (NJ = 4, or 3 for 33..48 right-hand sides)
template <bool ATOMIC, int NJ>
__global__ void __launch_bounds__(256) zgemm_ff_kernel(int opA, int opB, int64_t M, int64_t N, int64_t K, double ar,
                                                       double ai, const float4* __restrict__ A, int64_t lda,
                                                       const float4* __restrict__ B, int64_t ldb, double beta,
                                                       double2* __restrict__ C, int64_t ldc, int64_t k_chunk) {
  __shared__ float4 As[TBK * 2][TBM + 1];
  constexpr int TN = 16 * NJ;
  __shared__ float4 Bs[TBK * 2][TN + 1];
  constexpr int KT = TBK * 2;  // 16
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t row0 = int64_t(blockIdx.y) * TBM, col0 = int64_t(blockIdx.x) * TN;
  const int64_t k_begin = int64_t(blockIdx.z) * k_chunk, k_end = min(K, k_begin + k_chunk);
  const float sa = opA == OP_C ? -1.f : 1.f, sb = opB == OP_C ? -1.f : 1.f;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 acc[4][NJ];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[i][j] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t k0 = k_begin; k0 < k_end; k0 += KT) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {  // A tile 64 x 16
      int e = tid + 256 * l;
      int r = (opA == OP_N) ? e / KT : e % TBM;
      int kk = (opA == OP_N) ? e % KT : e / TBM;
      int64_t gr = row0 + r, gk = k0 + kk;
      float4 v = (gr < M && gk < k_end) ? (opA == OP_N ? A[gr * lda + gk] : A[gk * lda + gr]) : z4;
      v.z *= sa;
      v.w *= sa;
      As[kk][r] = v;
    }
#pragma unroll
    for (int l = 0; l < NJ; ++l) {  // B tile 16 x TN
      int e = tid + 256 * l;
      int c = (opB == OP_N) ? e % TN : e / KT;
      int kk = (opB == OP_N) ? e / TN : e % KT;
      int64_t gc = col0 + c, gk = k0 + kk;
      float4 v = (gc < N && gk < k_end) ? (opB == OP_N ? B[gk * ldb + gc] : B[gc * ldb + gk]) : z4;
      v.z *= sb;
      v.w *= sb;
      Bs[kk][c] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KT; ++kk) {
      float4 a[4], b[NJ];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < NJ; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          float4& c = acc[i][j];  // (re.h, re.l, im.h, im.l)
          ff_acc(c.x, c.y, a[i].x, a[i].y, b[j].x, b[j].y);
          ff_acc(c.x, c.y, -a[i].z, -a[i].w, b[j].z, b[j].w);
          ff_acc(c.z, c.w, a[i].x, a[i].y, b[j].z, b[j].w);
          ff_acc(c.z, c.w, a[i].z, a[i].w, b[j].x, b[j].y);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < NJ; ++j) {  // renormalise (fast two-sum)
        float4& c = acc[i][j];
        float s = c.x + c.y;
        c.y = c.y - (s - c.x);
        c.x = s;
        s = c.z + c.w;
        c.w = c.w - (s - c.z);
        c.z = s;
      }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t r = row0 + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      int64_t c = col0 + tx + 16 * j;
      if (c >= N) continue;
      double xr = double(acc[i][j].x) + double(acc[i][j].y), xi = double(acc[i][j].z) + double(acc[i][j].w);
      double2 v = make_double2(ar * xr - ai * xi, ar * xi + ai * xr);
      if constexpr (ATOMIC) {
        atomicAdd(&C[r * ldc + c].x, v.x);
        atomicAdd(&C[r * ldc + c].y, v.y);
      } else {
        if (beta != 0.0) {
          double2 o = C[r * ldc + c];
          v.x += beta * o.x;
          v.y += beta * o.y;
        }
        C[r * ldc + c] = v;
      }
    }
  }
}

// ------------------------------------------------------------------ skinny GEMM (op(A) = A)
// One warp per row of A; lanes stride over K; N <= 8 columns of op(B).
template <typename T, int NC>
__global__ void __launch_bounds__(256) gemm_skinny_kernel(int opB, int64_t M, int64_t K, T ar, T ai,
                                                          const typename C2<T>::type* __restrict__ A, int64_t lda,
                                                          const typename C2<T>::type* __restrict__ B, int64_t ldb,
                                                          T beta, typename C2<T>::type* __restrict__ C, int64_t ldc) {
  using V = typename C2<T>::type;
  const int64_t row = int64_t(blockIdx.x) * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= M) return;
  V acc[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) acc[j] = {T(0), T(0)};
  const V* arow = A + row * lda;
  for (int64_t k = lane; k < K; k += 32) {
    V a = arow[k];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      V b = load_op<T>(B, k, j, ldb, opB);
      acc[j].x = fma(a.x, b.x, acc[j].x);
      acc[j].x = fma(-a.y, b.y, acc[j].x);
      acc[j].y = fma(a.x, b.y, acc[j].y);
      acc[j].y = fma(a.y, b.x, acc[j].y);
    }
  }
#pragma unroll
  for (int j = 0; j < NC; ++j) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc[j].x += __shfl_xor_sync(0xffffffffu, acc[j].x, off);
      acc[j].y += __shfl_xor_sync(0xffffffffu, acc[j].y, off);
    }
  }
  if (lane < NC) {
    V s = acc[0];
#pragma unroll
    for (int j = 1; j < NC; ++j)
      if (lane == j) s = acc[j];
    V v = {ar * s.x - ai * s.y, ar * s.y + ai * s.x};
    if (beta != T(0)) {
      V o = C[row * ldc + lane];
      v.x += beta * o.x;
      v.y += beta * o.y;
    }
    C[row * ldc + lane] = v;
  }
}

// ------------------------------------------------------------------ panel factorisation
// Panel scratch header (zeroed before each factorisation): a monotonic arrival counter for
// the grid barrier and a ring of four 64-bit pivot keys (column c uses key[c & 3]).
struct PanelScratch {
  unsigned count;
  unsigned gen;
  unsigned long long key[4];
};
static_assert(sizeof(PanelScratch) <= 256, "the panel header must fit the zeroed 256 bytes");

constexpr int kPanelThreads = 256;
constexpr int kMaxPanelRows = 2048;  // rows per CTA (multipliers kept in shared memory)
constexpr long long kSpinLimit = 1ll << 26;
// Poll limit of the bounded grid-barrier waits on this device (kSpinLimit unless changed by
// fosb_debug_set_wait_limit, which failure-detection tests use to make the waits give up).
__device__ long long g_wait_limit = kSpinLimit;

__device__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned nblocks, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = gen;
    unsigned my_gen = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(count, 1u);
    if (arrived == nblocks - 1) {
      *count = 0;
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      long long spins = 0;
      const long long limit = g_wait_limit;
      while (*vgen == my_gen) {
        if (++spins > limit || *(volatile int*)status == FOSB_ERR_TIMEOUT) {
          atomicExch(status, FOSB_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(20);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Grid barrier on a counter that only grows: every CTA adds one and waits until the count
// reaches target (this launch's base + (column + 1) x CTAs), so no CTA has to reset it.
// Bounded: after g_wait_limit polls the status word is set to FOSB_ERR_TIMEOUT and the CTA
// leaves.
__device__ bool grid_arrive_wait(unsigned* count, unsigned target, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    atomicAdd(count, 1u);
    volatile unsigned* vc = count;
    long long spins = 0;
    const long long limit = g_wait_limit;
    while (int(*vc - target) < 0) {
      if (++spins > limit || *(volatile int*)status == FOSB_ERR_TIMEOUT) {
        atomicExch(status, FOSB_ERR_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(20);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Pivot key: magnitude |Re| + |Im| in the upper 32 bits (float bits for complex64; the top
// 32 bits of the double for complex128, a monotone truncation), ~row in the lower 32 bits,
// so the largest key is the largest magnitude with ties going to the lowest row.
template <typename T>
__device__ __forceinline__ unsigned long long pivot_key(typename C2<T>::type v, int64_t row) {
  unsigned hi;
  if constexpr (sizeof(T) == 4)
    hi = __float_as_uint(fabsf(v.x) + fabsf(v.y));
  else
    hi = unsigned(uint64_t(__double_as_longlong(fabs(v.x) + fabs(v.y))) >> 32);
  return (static_cast<unsigned long long>(hi) << 32) | (0xFFFFFFFFu - static_cast<unsigned>(row));
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long k) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    unsigned long long o = __shfl_xor_sync(0xffffffffu, k, off);
    k = o > k ? o : k;
  }
  return k;
}

// cand_data[2][G][jb], rowj[2][jb]
// One column per step over the CTAs' row blocks of the panel (rows [lo, hi) each), in
// global memory; cand_data[2][G][jb] and rowj[2][jb] carry the candidate rows and row j.
template <typename T>
__global__ void __launch_bounds__(kPanelThreads) panel_kernel(typename C2<T>::type* A, int64_t m, int jb, int64_t lda,
                                                              int32_t* ipiv, int64_t row_base, PanelScratch* scr,
                                                              unsigned bar_base, typename C2<T>::type* cand_data,
                                                              typename C2<T>::type* rowj, int* status) {
  using V = typename C2<T>::type;
  const unsigned G = gridDim.x;
  const int64_t chunk = (m + G - 1) / G;
  const int64_t lo = int64_t(blockIdx.x) * chunk, hi = min(m, lo + chunk);
  __shared__ unsigned long long s_key[kPanelThreads / 32];
  __shared__ V s_l[kMaxPanelRows];
  __shared__ V s_piv[64];
  __shared__ int64_t s_p;
  // identity pivots first: if a barrier wait gives up, the columns not reached keep valid rows
  if (blockIdx.x == 0)
    for (int c = threadIdx.x; c < jb; c += blockDim.x) ipiv[c] = int32_t(row_base + c);
  __syncthreads();
#define ROW(r, c) A[(r) * lda + (c)]
  for (int j = 0; j < jb; ++j) {
    const int par = j & 1;
    // 1. local pivot candidate (largest |Re|+|Im|, ties -> lowest row)
    unsigned long long best = 0ull;
    for (int64_t r = max(lo, int64_t(j)) + threadIdx.x; r < hi; r += blockDim.x) {
      const unsigned long long k = pivot_key<T>(A[r * lda + j], r);
      best = k > best ? k : best;
    }
    best = warp_max_u64(best);
    if ((threadIdx.x & 31) == 0) s_key[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kPanelThreads / 32; ++w) best = s_key[w] > best ? s_key[w] : best;
      s_key[0] = best;
    }
    __syncthreads();
    best = s_key[0];
    const int64_t brow = best != 0ull ? int64_t(0xFFFFFFFFu - unsigned(best & 0xFFFFFFFFull)) : m;
    // 2. publish the candidate's panel row (and, by its owner, row j); fold the key into
    //    this column's slot; wait for every CTA
    for (int c = threadIdx.x; c < jb; c += blockDim.x) {
      cand_data[(int64_t(par) * G + blockIdx.x) * jb + c] = (brow < m) ? ROW(brow, c) : V{T(0), T(0)};
      if (j >= lo && j < hi) rowj[par * jb + c] = ROW(int64_t(j), c);
    }
    if (threadIdx.x == 0 && best != 0ull) atomicMax(&scr->key[(row_base + j) & 3], best);
    __threadfence();
    if (!grid_arrive_wait(&scr->count, bar_base + unsigned(j + 1) * G, status)) return;
    // 3. the winning key names the pivot row and, through the row partition, its CTA
    if (threadIdx.x == 0) {
      const unsigned long long key = *reinterpret_cast<volatile unsigned long long*>(&scr->key[(row_base + j) & 3]);
      // an exactly zero column folds no key: no interchange (status SINGULAR below)
      const int64_t pk = int64_t(0xFFFFFFFFu - unsigned(key & 0xFFFFFFFFull));
      s_p = (key == 0ull || pk >= m) ? int64_t(j) : pk;
      if (blockIdx.x == 0) {
        ipiv[j] = int32_t(row_base + s_p);
        if ((key >> 32) == 0ull) atomicCAS(status, 0, FOSB_ERR_SINGULAR);
        scr->key[(row_base + j + 3) & 3] = 0ull;  // previous column's slot: every CTA has read it
      }
    }
    __syncthreads();
    const int64_t p = s_p;
    const V* pdata = cand_data + (int64_t(par) * G + p / chunk) * jb;
    for (int c = threadIdx.x; c < jb; c += blockDim.x) s_piv[c] = __ldcg(pdata + c);
    __syncthreads();
    // 4. swap rows j and p inside the panel
    if (p != j) {
      if (j >= lo && j < hi)
        for (int c = threadIdx.x; c < jb; c += blockDim.x) A[int64_t(j) * lda + c] = s_piv[c];
      if (p >= lo && p < hi)
        for (int c = threadIdx.x; c < jb; c += blockDim.x) A[p * lda + c] = __ldcg(rowj + par * jb + c);
    }
    __syncthreads();
    // 5. multipliers and rank-1 update of the rows below j owned by this CTA
    const V pv = s_piv[j];
    const T den = pv.x * pv.x + pv.y * pv.y;
    const V inv = den > T(0) ? V{pv.x / den, -pv.y / den} : V{T(0), T(0)};
    const int64_t r0 = max(lo, int64_t(j) + 1);
    for (int64_t r = r0 + threadIdx.x; r < hi; r += blockDim.x) {
      V l = cmul<T>(A[r * lda + j], inv);
      A[r * lda + j] = l;
      s_l[r - lo] = l;
    }
    __syncthreads();
    const int ncols = jb - j - 1;
    if (ncols > 0 && hi > r0) {
      const int64_t total = (hi - r0) * ncols;
      for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
        int64_t r = r0 + e / ncols;
        int c = j + 1 + int(e % ncols);
        V l = s_l[r - lo], u = s_piv[c];
        V a = A[r * lda + c];
        a.x -= l.x * u.x - l.y * u.y;
        a.y -= l.x * u.y + l.y * u.x;
        A[r * lda + c] = a;
      }
    }
    __syncthreads();
  }
#undef ROW
}

// The same panel factorisation with each CTA's row block resident in shared memory
// (rows [lo, hi) x jb, loaded once, written back once); only the pivot candidates, the
// pivot row and row j cross CTAs, through global memory and the bounded grid barrier.
template <typename T>
__global__ void __launch_bounds__(kPanelThreads) panel_smem_kernel(typename C2<T>::type* A, int64_t m, int jb,
                                                                   int64_t lda, int32_t* ipiv, int64_t row_base,
                                                                   PanelScratch* scr, unsigned bar_base,
                                                                   typename C2<T>::type* cand_data,
                                                                   typename C2<T>::type* rowj, int* status) {
  using V = typename C2<T>::type;
  extern __shared__ unsigned char panel_raw[];
  V* sP = reinterpret_cast<V*>(panel_raw);  // (hi - lo) x jb
  const unsigned G = gridDim.x;
  const int64_t chunk = (m + G - 1) / G;
  const int64_t lo = int64_t(blockIdx.x) * chunk, hi = min(m, lo + chunk);
  const int nr = hi > lo ? int(hi - lo) : 0;
  __shared__ unsigned long long s_key[kPanelThreads / 32];
  __shared__ V s_piv[64];
  __shared__ int64_t s_p;
  // identity pivots first: if a barrier wait gives up, the columns not reached keep valid rows
  if (blockIdx.x == 0)
    for (int c = threadIdx.x; c < jb; c += blockDim.x) ipiv[c] = int32_t(row_base + c);
  for (int e = threadIdx.x; e < nr * jb; e += blockDim.x) sP[e] = A[(lo + e / jb) * lda + e % jb];
  __syncthreads();
#define ROW(r, c) sP[((r) - lo) * jb + (c)]
  for (int j = 0; j < jb; ++j) {
    const int par = j & 1;
    unsigned long long best = 0ull;
    for (int r = (j > lo ? int(j - lo) : 0) + threadIdx.x; r < nr; r += blockDim.x) {
      const unsigned long long k = pivot_key<T>(sP[r * jb + j], lo + r);
      best = k > best ? k : best;
    }
    best = warp_max_u64(best);
    if ((threadIdx.x & 31) == 0) s_key[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kPanelThreads / 32; ++w) best = s_key[w] > best ? s_key[w] : best;
      s_key[0] = best;
    }
    __syncthreads();
    best = s_key[0];
    const int64_t brow = best != 0ull ? int64_t(0xFFFFFFFFu - unsigned(best & 0xFFFFFFFFull)) : m;
    // 2. publish the candidate's panel row (and, by its owner, row j); fold the key into
    //    this column's slot; wait for every CTA
    for (int c = threadIdx.x; c < jb; c += blockDim.x) {
      cand_data[(int64_t(par) * G + blockIdx.x) * jb + c] = (brow < m) ? ROW(brow, c) : V{T(0), T(0)};
      if (j >= lo && j < hi) rowj[par * jb + c] = ROW(int64_t(j), c);
    }
    if (threadIdx.x == 0 && best != 0ull) atomicMax(&scr->key[(row_base + j) & 3], best);
    __threadfence();
    if (!grid_arrive_wait(&scr->count, bar_base + unsigned(j + 1) * G, status)) return;
    // 3. the winning key names the pivot row and, through the row partition, its CTA
    if (threadIdx.x == 0) {
      const unsigned long long key = *reinterpret_cast<volatile unsigned long long*>(&scr->key[(row_base + j) & 3]);
      // an exactly zero column folds no key: no interchange (status SINGULAR below)
      const int64_t pk = int64_t(0xFFFFFFFFu - unsigned(key & 0xFFFFFFFFull));
      s_p = (key == 0ull || pk >= m) ? int64_t(j) : pk;
      if (blockIdx.x == 0) {
        ipiv[j] = int32_t(row_base + s_p);
        if ((key >> 32) == 0ull) atomicCAS(status, 0, FOSB_ERR_SINGULAR);
        scr->key[(row_base + j + 3) & 3] = 0ull;  // previous column's slot: every CTA has read it
      }
    }
    __syncthreads();
    const int64_t p = s_p;
    const V* pdata = cand_data + (int64_t(par) * G + p / chunk) * jb;
    for (int c = threadIdx.x; c < jb; c += blockDim.x) s_piv[c] = __ldcg(pdata + c);
    __syncthreads();
    if (p != j) {
      if (j >= lo && j < hi)
        for (int c = threadIdx.x; c < jb; c += blockDim.x) sP[(j - lo) * jb + c] = s_piv[c];
      if (p >= lo && p < hi)
        for (int c = threadIdx.x; c < jb; c += blockDim.x) sP[(p - lo) * jb + c] = __ldcg(rowj + par * jb + c);
    }
    __syncthreads();
    const V pv = s_piv[j];
    const T den = pv.x * pv.x + pv.y * pv.y;
    const V inv = den > T(0) ? V{pv.x / den, -pv.y / den} : V{T(0), T(0)};
    const int r0 = (int64_t(j) + 1 > lo) ? int(int64_t(j) + 1 - lo) : 0;
    for (int r = r0 + threadIdx.x; r < nr; r += blockDim.x) sP[r * jb + j] = cmul<T>(sP[r * jb + j], inv);
    __syncthreads();
    const int ncols = jb - j - 1;
    if (ncols > 0 && nr > r0) {
      const int total = (nr - r0) * ncols;
      for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int r = r0 + e / ncols, c = j + 1 + e % ncols;
        V l = sP[r * jb + j], u = s_piv[c];
        V a = sP[r * jb + c];
        a.x -= l.x * u.x - l.y * u.y;
        a.y -= l.x * u.y + l.y * u.x;
        sP[r * jb + c] = a;
      }
    }
    __syncthreads();
  }
#undef ROW
  for (int e = threadIdx.x; e < nr * jb; e += blockDim.x) A[(lo + e / jb) * lda + e % jb] = sP[e];
}

// Row swaps of the block row [j0, j0 + jb) applied to columns outside the panel.
template <typename T>
__global__ void laswp_kernel(typename C2<T>::type* A, int64_t n, int64_t lda, int64_t j0, int jb,
                             const int32_t* ipiv) {
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= n || (c >= j0 && c < j0 + jb)) return;
  for (int i = 0; i < jb; ++i) {
    int64_t p = ipiv[j0 + i];
    if (p != j0 + i && p >= 0 && p < n) {  // a pivot outside the matrix (never written) is skipped
      auto t = A[(j0 + i) * lda + c];
      A[(j0 + i) * lda + c] = A[p * lda + c];
      A[p * lda + c] = t;
    }
  }
}

// X (nb x ncols block) <- L^{-1} X with L unit lower (unit=1) or U^{-1} X with U upper
// (unit=0), diagonal block of size nb at D (leading dimension ldd).  Thread per column.
template <typename T>
__global__ void trsm_diag_kernel(const typename C2<T>::type* D, int64_t ldd, int nb, int upper,
                                 typename C2<T>::type* X, int64_t ldx, int64_t ncols) {
  using V = typename C2<T>::type;
  int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  if (!upper) {
    for (int i = 1; i < nb; ++i) {
      V s = X[int64_t(i) * ldx + c];
      for (int k = 0; k < i; ++k) {
        V l = D[int64_t(i) * ldd + k], x = X[int64_t(k) * ldx + c];
        s.x -= l.x * x.x - l.y * x.y;
        s.y -= l.x * x.y + l.y * x.x;
      }
      X[int64_t(i) * ldx + c] = s;
    }
  } else {
    for (int i = nb - 1; i >= 0; --i) {
      V s = X[int64_t(i) * ldx + c];
      for (int k = i + 1; k < nb; ++k) {
        V u = D[int64_t(i) * ldd + k], x = X[int64_t(k) * ldx + c];
        s.x -= u.x * x.x - u.y * x.y;
        s.y -= u.x * x.y + u.y * x.x;
      }
      V d = D[int64_t(i) * ldd + i];
      T den = d.x * d.x + d.y * d.y;
      V q = den > T(0) ? V{(s.x * d.x + s.y * d.y) / den, (s.y * d.x - s.x * d.y) / den} : V{T(0), T(0)};
      X[int64_t(i) * ldx + c] = q;
    }
  }
}

// Few right-hand sides: one warp per column, lanes own rows (lane, lane + 32) of the
// nb x nb diagonal block, which is staged transposed in shared memory (conflict-free
// column reads).  Forward (unit lower) or backward (upper, with the diagonal) sweep.
template <typename T>
__global__ void __launch_bounds__(256) trsv_warp_kernel(const typename C2<T>::type* D, int64_t ldd, int nb, int upper,
                                                        typename C2<T>::type* X, int64_t ldx, int64_t ncols) {
  using V = typename C2<T>::type;
  extern __shared__ unsigned char smem_raw[];
  V* Dt = reinterpret_cast<V*>(smem_raw);  // Dt[k * nb + r] = D[r, k]
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int r = e / nb, k = e % nb;
    Dt[k * nb + r] = D[int64_t(r) * ldd + k];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = int64_t(blockIdx.x) * 8 + warp;
  if (c >= ncols) return;
  const V zero = {T(0), T(0)};
  V x0 = lane < nb ? X[int64_t(lane) * ldx + c] : zero;
  V x1 = lane + 32 < nb ? X[int64_t(lane + 32) * ldx + c] : zero;
  auto bcast = [&](int i) {
    V v = i < 32 ? x0 : x1;
    v.x = __shfl_sync(0xffffffffu, v.x, i & 31);
    v.y = __shfl_sync(0xffffffffu, v.y, i & 31);
    return v;
  };
  auto fms = [](V a, V d, V x) {  // a - d x
    a.x -= d.x * x.x - d.y * x.y;
    a.y -= d.x * x.y + d.y * x.x;
    return a;
  };
  if (!upper) {
    for (int i = 0; i < nb - 1; ++i) {
      V xi = bcast(i);
      if (lane > i && lane < nb) x0 = fms(x0, Dt[i * nb + lane], xi);
      if (lane + 32 > i && lane + 32 < nb) x1 = fms(x1, Dt[i * nb + lane + 32], xi);
    }
  } else {
    for (int i = nb - 1; i >= 0; --i) {
      V d = Dt[i * nb + i];
      T den = d.x * d.x + d.y * d.y;
      bool mine0 = i < 32 && lane == i, mine1 = i >= 32 && lane == i - 32;
      if (mine0 || mine1) {
        V v = mine0 ? x0 : x1;
        V q = den > T(0) ? V{(v.x * d.x + v.y * d.y) / den, (v.y * d.x - v.x * d.y) / den} : zero;
        if (mine0) x0 = q; else x1 = q;
      }
      V xi = bcast(i);
      if (lane < i) x0 = fms(x0, Dt[i * nb + lane], xi);
      if (lane + 32 < i) x1 = fms(x1, Dt[i * nb + lane + 32], xi);
    }
  }
  if (lane < nb) X[int64_t(lane) * ldx + c] = x0;
  if (lane + 32 < nb) X[int64_t(lane + 32) * ldx + c] = x1;
}

// Opt the warp-per-column solve into 64 KB of dynamic shared memory (a 64 x 64 complex128 block).
template <typename T>
void enable_trsv_smem() {
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !done[dev]) {
    cudaFuncSetAttribute(trsv_warp_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(64 * 64 * sizeof(typename C2<T>::type)));
    done[dev] = true;
  }
}

template <typename T>
__global__ void gather_rows_kernel(const typename C2<T>::type* X, int64_t ldx, const int32_t* perm, int64_t n,
                                   int64_t nrhs, typename C2<T>::type* Y, int64_t ldy) {
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n * nrhs) return;
  int64_t i = e / nrhs, c = e % nrhs;
  Y[i * ldy + c] = X[int64_t(perm[i]) * ldx + c];
}

__global__ void c128_to_c64_kernel(const double2* s, int64_t rows, int64_t cols, int64_t lds, float2* d, int64_t ldd) {
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  int64_t i = e / cols, j = e % cols;
  double2 v = s[i * lds + j];
  d[i * ldd + j] = make_float2(float(v.x), float(v.y));
}
__global__ void c64_to_c128_kernel(const float2* s, int64_t rows, int64_t cols, int64_t lds, double2* d, int64_t ldd) {
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  int64_t i = e / cols, j = e % cols;
  float2 v = s[i * lds + j];
  d[i * ldd + j] = make_double2(v.x, v.y);
}
__global__ void axpy_kernel(const float2* dlt, int64_t rows, int64_t cols, int64_t ldd, double2* x, int64_t ldx) {
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  int64_t i = e / cols, j = e % cols;
  float2 v = dlt[i * ldd + j];
  x[i * ldx + j].x += v.x;
  x[i * ldx + j].y += v.y;
}

__device__ __forceinline__ void atomic_max_pos(double* p, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(p), __double_as_longlong(v));
}

__global__ void row_norm_kernel(const double2* A, int64_t rows, int64_t cols, int64_t lda, double* out) {
  int64_t r = int64_t(blockIdx.x) * 8 + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (r >= rows) return;
  double s = 0;
  for (int64_t c = lane; c < cols; c += 32) {
    double2 v = A[r * lda + c];
    s += fabs(v.x) + fabs(v.y);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) atomic_max_pos(out, s);
}

// per-column max |Re| + |Im| (out has cols entries)
__global__ void col_absmax_kernel(const double2* A, int64_t rows, int64_t cols, int64_t lda, double* out) {
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  int64_t i = e / cols, j = e % cols;
  double2 v = A[i * lda + j];
  atomic_max_pos(out + j, fabs(v.x) + fabs(v.y));
}

template <typename T>
__global__ void add_mirrored_kernel(const typename C2<T>::type* M, int64_t n, int64_t ldm, int op, T w, int acc,
                                    typename C2<T>::type* out, int64_t ldo) {
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  int64_t i = e / n, j = e % n;
  auto a = M[i * ldm + j], b = M[j * ldm + i];
  if (op == OP_C) b.y = -b.y;
  typename C2<T>::type v = {w * (a.x + b.x), w * (a.y + b.y)};
  if (acc) {
    v.x += out[i * ldo + j].x;
    v.y += out[i * ldo + j].y;
  }
  out[i * ldo + j] = v;
}

template <typename T>
__global__ void copy_kernel(const T* s, int64_t rows, int64_t cols, int64_t lds, T* d, int64_t ldd) {
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  int64_t i = e / cols, j = e % cols;
  d[i * ldd + j] = s[i * lds + j];
}

// Launch one panel factorisation (m x jb at Ap): the shared-memory-resident kernel when
// each CTA's row block fits in 200 KB, otherwise the global-memory kernel.
constexpr int kPanelSmemBudget = 200 * 1024;

template <typename T>
cudaError_t launch_panel(typename C2<T>::type* Ap, int64_t m, int jb, int64_t lda, int32_t* ip, int64_t row_base,
                         PanelScratch* scr, unsigned& arrivals, typename C2<T>::type* cand_data,
                         typename C2<T>::type* rowj, int* d_status, int64_t G_cap, int nsm, cudaStream_t s) {
  using V = typename C2<T>::type;
  ProfScope prof("lu_panel", s, 4.0 * double(m) * jb * jb);
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    cudaFuncSetAttribute(panel_smem_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPanelSmemBudget);
    attr[dev] = true;
  }
  const int64_t rows_cap = kPanelSmemBudget / (int64_t(jb) * int64_t(sizeof(V)));
  int64_t G = std::min<int64_t>(std::min<int64_t>(G_cap, nsm),
                                std::max<int64_t>((m + rows_cap - 1) / rows_cap, (m + 255) / 256));
  G = std::max<int64_t>(G, 1);
  const int64_t chunk = (m + G - 1) / G;
  const size_t smem = size_t(chunk) * jb * sizeof(V);
  int per_sm = 0;
  if (chunk <= rows_cap &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, panel_smem_kernel<T>, kPanelThreads, smem) == cudaSuccess &&
      per_sm >= 1 && G <= int64_t(per_sm) * nsm) {
    unsigned bar_base = arrivals;
    void* args[] = {&Ap, &m, &jb, &lda, &ip, &row_base, &scr, &bar_base, &cand_data, &rowj, &d_status};
    cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(panel_smem_kernel<T>), dim3(unsigned(G)),
                                                dim3(kPanelThreads), args, smem, s);
    arrivals += unsigned(G) * unsigned(jb);  // every CTA arrives once per column
    return e;
  }
  G = std::min<int64_t>(std::min<int64_t>(G_cap, nsm), std::max<int64_t>(1, (m + 255) / 256));
  if ((m + G - 1) / G > kMaxPanelRows) return cudaErrorInvalidValue;
  unsigned bar_base = arrivals;
  void* args[] = {&Ap, &m, &jb, &lda, &ip, &row_base, &scr, &bar_base, &cand_data, &rowj, &d_status};
  cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(panel_kernel<T>), dim3(unsigned(G)),
                                              dim3(kPanelThreads), args, 0, s);
  arrivals += unsigned(G) * unsigned(jb);
  return e;
}

}  // namespace

template <typename T>
cudaError_t gemm(int opA, int opB, int64_t M, int64_t N, int64_t K, double alpha_re, double alpha_im, const void* A,
                 int64_t lda, const void* B, int64_t ldb, double beta, void* C, int64_t ldc, cudaStream_t s) {
  using V = typename C2<T>::type;
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K <= 0) {
    // C = beta C
    if (beta == 0.0) return cudaMemset2DAsync(C, ldc * sizeof(V), 0, N * sizeof(V), M, s);
    return cudaSuccess;
  }
  const V* a = static_cast<const V*>(A);
  const V* b = static_cast<const V*>(B);
  V* c = static_cast<V*>(C);
  if (opA == OP_N && N <= 8) {
    unsigned g = cdiv(M, 8);
#define FOSB_SKINNY(NC) \
  gemm_skinny_kernel<T, NC><<<g, 256, 0, s>>>(opB, M, K, T(alpha_re), T(alpha_im), a, lda, b, ldb, T(beta), c, ldc)
    switch (N) {
      case 1: FOSB_SKINNY(1); break;
      case 2: FOSB_SKINNY(2); break;
      case 3: FOSB_SKINNY(3); break;
      case 4: FOSB_SKINNY(4); break;
      case 5: FOSB_SKINNY(5); break;
      case 6: FOSB_SKINNY(6); break;
      case 7: FOSB_SKINNY(7); break;
      default: FOSB_SKINNY(8); break;
    }
#undef FOSB_SKINNY
    return launched();
  }
  if (cdiv(M, TBM) > 65535u) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 8) {
    // split K when the output tiles alone cannot fill the GPU (tall-K, skinny products such
    // as refinement residuals); partial products meet in C through FP64 atomics
    const int64_t tiles = int64_t(cdiv(N, DBN)) * cdiv(M, DBM);
    int64_t splits = 1;
    if ((beta == 0.0 || beta == 1.0) && tiles < 2 * 152 && K >= 1024)
      splits = std::min<int64_t>((2 * 152 + tiles - 1) / tiles, K / 512);
    int64_t k_chunk = ((K + splits - 1) / splits + DBK - 1) / DBK * DBK;
    splits = (K + k_chunk - 1) / k_chunk;
    dim3 gridd(cdiv(N, DBN), cdiv(M, DBM), unsigned(splits));
    static bool smem_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !smem_set[dev]) {
      cudaFuncSetAttribute(zgemm_dmma_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kDmmaSmem));
      cudaFuncSetAttribute(zgemm_dmma_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kDmmaSmem));
      smem_set[dev] = true;
    }
    if (splits > 1) {
      if (beta == 0.0) {
        cudaError_t e = cudaMemset2DAsync(c, ldc * sizeof(V), 0, N * sizeof(V), M, s);
        if (e != cudaSuccess) return e;
      }
      zgemm_dmma_kernel<true><<<gridd, 256, kDmmaSmem, s>>>(opA, opB, M, N, K, alpha_re, alpha_im, a, lda, b, ldb,
                                                            beta, c, ldc, k_chunk);
    } else {
      zgemm_dmma_kernel<false><<<gridd, 256, kDmmaSmem, s>>>(opA, opB, M, N, K, alpha_re, alpha_im, a, lda, b, ldb,
                                                             beta, c, ldc, k_chunk);
    }
    return launched();
  }
  dim3 grid(cdiv(N, TBN), cdiv(M, TBM));
  gemm_tiled_kernel<T><<<grid, 256, 0, s>>>(opA, opB, M, N, K, T(alpha_re), T(alpha_im), a, lda, b, ldb, T(beta), c, ldc);
  return launched();
}

template cudaError_t gemm<double>(int, int, int64_t, int64_t, int64_t, double, double, const void*, int64_t,
                                  const void*, int64_t, double, void*, int64_t, cudaStream_t);

cudaError_t split_ff(const void* src, int64_t rows, int64_t cols, int64_t lds, void* dst, int64_t ldd,
                     cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  split_ff_kernel<<<cdiv(rows * cols, 256), 256, 0, s>>>(static_cast<const double2*>(src), rows, cols, lds,
                                                         static_cast<float4*>(dst), ldd);
  return launched();
}

cudaError_t gemm_c128_ff(int opA, int opB, int64_t M, int64_t N, int64_t K, double alpha_re, double alpha_im,
                         const void* A, int64_t lda, const void* B, int64_t ldb, double beta, void* C, int64_t ldc,
                         cudaStream_t s, const void* A_split) {
  using V = double2;
  if (M <= 0 || N <= 0) return cudaSuccess;
  // up to 8 right-hand sides: a row-per-warp kernel that streams A once; float-float on the
  // cached split of A when there is one, else FP64 (a 64-wide tile would be mostly padding)
  if (K > 0 && opA == OP_N && opB == OP_N && N <= 8 && A_split) {
    float4* bs = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&bs), size_t(K * N) * sizeof(float4), s);
    if (e == cudaSuccess) e = split_ff(B, K, N, ldb, bs, N, s);
    if (e == cudaSuccess) {
      ProfScope prof("gemm_ff", s, 8.0 * double(M) * double(N) * double(K));
      const float4* a4 = static_cast<const float4*>(A_split);
      double2* c2 = static_cast<double2*>(C);
      const unsigned g = cdiv(M, 8);
#define FOSB_GEMV(NC) zgemv_ff_kernel<NC><<<g, 256, 0, s>>>(M, K, alpha_re, alpha_im, a4, lda, bs, beta, c2, ldc)
      switch (N) {
        case 1: FOSB_GEMV(1); break;
        case 2: FOSB_GEMV(2); break;
        case 3: FOSB_GEMV(3); break;
        case 4: FOSB_GEMV(4); break;
        case 5: FOSB_GEMV(5); break;
        case 6: FOSB_GEMV(6); break;
        case 7: FOSB_GEMV(7); break;
        default: FOSB_GEMV(8); break;
      }
#undef FOSB_GEMV
      e = launched();
    }
    if (bs) cudaFreeAsync(bs, s);
    return e;
  }
  if (K <= 0 || (opA == OP_N && N <= 8))
    return gemm<double>(opA, opB, M, N, K, alpha_re, alpha_im, A, lda, B, ldb, beta, C, ldc, s);
  if (cdiv(M, TBM) > 65535u) return cudaErrorInvalidValue;
  V* c = static_cast<V*>(C);
  // (hi, lo) splits of the operands as stored (A_split: a cached split of A with ld = lda)
  const int64_t ar = opA == OP_N ? M : K, ac = opA == OP_N ? K : M;
  const int64_t br = opB == OP_N ? K : N, bc = opB == OP_N ? N : K;
  float4 *as = nullptr, *bs = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&bs), size_t(br * bc) * sizeof(float4), s);
  if (e == cudaSuccess) e = split_ff(B, br, bc, ldb, bs, bc, s);
  if (e == cudaSuccess && !A_split) {
    e = cudaMallocAsync(reinterpret_cast<void**>(&as), size_t(ar * ac) * sizeof(float4), s);
    if (e == cudaSuccess) e = split_ff(A, ar, ac, lda, as, ac, s);
  }
  const float4* a4 = A_split ? static_cast<const float4*>(A_split) : as;
  const int64_t lda4 = A_split ? lda : ac;
  if (e == cudaSuccess) {
    const bool n48 = N > 32 && N <= 48;  // 48-wide tiles: less padding for 33..48 columns
    const int64_t tn = n48 ? 48 : TBN;
    const int64_t tiles = int64_t(cdiv(N, tn)) * cdiv(M, TBM);
    int64_t splits = 1;
    if ((beta == 0.0 || beta == 1.0) && tiles < 4 * 152 && K >= 1024)
      splits = std::min<int64_t>((4 * 152 + tiles - 1) / tiles, K / 512);
    int64_t k_chunk = ((K + splits - 1) / splits + 15) / 16 * 16;
    splits = (K + k_chunk - 1) / k_chunk;
    dim3 grid(cdiv(N, tn), cdiv(M, TBM), unsigned(splits));
    ProfScope prof("gemm_ff", s, 8.0 * double(M) * double(N) * double(K));
    if (splits > 1 && beta == 0.0) e = cudaMemset2DAsync(c, ldc * sizeof(V), 0, N * sizeof(V), M, s);
#define FOSB_FF(AT, NJ)                                                                                            \
  zgemm_ff_kernel<AT, NJ><<<grid, 256, 0, s>>>(opA, opB, M, N, K, alpha_re, alpha_im, a4, lda4, bs, bc, beta, c, ldc, \
                                               k_chunk)
    if (e == cudaSuccess) {
      if (splits > 1) {
        if (n48) FOSB_FF(true, 3); else FOSB_FF(true, 4);
      } else {
        if (n48) FOSB_FF(false, 3); else FOSB_FF(false, 4);
      }
    }
#undef FOSB_FF
    if (e == cudaSuccess) e = launched();
  }
  if (as) cudaFreeAsync(as, s);
  if (bs) cudaFreeAsync(bs, s);
  return e;
}
template cudaError_t gemm<float>(int, int, int64_t, int64_t, int64_t, double, double, const void*, int64_t,
                                 const void*, int64_t, double, void*, int64_t, cudaStream_t);

template <typename T>
fosb_status getrf(void* Av, int64_t n, int64_t lda, int32_t* ipiv, int* d_status, cudaStream_t s) {
  using V = typename C2<T>::type;
  V* A = static_cast<V*>(Av);
  const int nb = 64;
  int dev = 0, nsm = 0;
  FOSB_CUDA(cudaGetDevice(&dev));
  FOSB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  int per_sm = 0;
  FOSB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, panel_kernel<T>, kPanelThreads, 0));
  if (per_sm < 1) return fail(FOSB_ERR_CUDA, "getrf: panel kernel cannot be resident");
  const int gmax = nsm * per_sm;
  // scratch: barrier/key header + candidate rows + row j (double-buffered)
  size_t G_cap = size_t(std::min<int64_t>(gmax, std::max<int64_t>(1, (n + 63) / 64)));
  size_t bytes = 256 + 2 * G_cap * nb * sizeof(V) + 2 * nb * sizeof(V);
  char* scratch = nullptr;
  FOSB_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&scratch), bytes, s));
  FOSB_CUDA(cudaMemsetAsync(scratch, 0, 256, s));
  PanelScratch* scr = reinterpret_cast<PanelScratch*>(scratch);
  V* cand_data = reinterpret_cast<V*>(scratch + 256);
  V* rowj = cand_data + 2 * G_cap * nb;
  unsigned arrivals = 0;  // grid-barrier arrivals so far (the counter starts at zero)
  fosb_status st = FOSB_OK;
  // complex64: tournament-pivoting panels (no grid-wide waits); complex128: cooperative
  // partial pivoting with one grid barrier per column
  char* tslu_scr = nullptr;
  void* ws_a = nullptr;  // complex64: the trailing update's operands, split once per block
  void* ws_b = nullptr;
  if constexpr (sizeof(T) == 4) {
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&tslu_scr), tslu_scratch_bytes(n), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&ws_a, update_split_a_bytes(n), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&ws_b, update_split_b_bytes(n), s);
    if (e != cudaSuccess) {
      cudaFreeAsync(scratch, s);
      if (tslu_scr) cudaFreeAsync(tslu_scr, s);
      if (ws_a) cudaFreeAsync(ws_a, s);
      return cuda_fail(e, "getrf: panel scratch");
    }
  }
  // one 64-column panel at column j0, then its row interchanges on every other column
  auto panel_step = [&](int64_t j0, int jb) -> cudaError_t {
    cudaError_t e;
    if constexpr (sizeof(T) == 4)
      e = tslu_panel(A + j0 * lda + j0, n - j0, jb, lda, ipiv + j0, j0, tslu_scr, n, d_status, s);
    else
      e = launch_panel<T>(A + j0 * lda + j0, n - j0, jb, lda, ipiv + j0, j0, scr, arrivals, cand_data, rowj,
                          d_status, int64_t(G_cap), nsm, s);
    if (e != cudaSuccess) return e;
    if constexpr (sizeof(T) == 4) {
      return tslu_swap(A, n, lda, j0, jb, tslu_scr, s);  // the panel's permutation as row moves
    } else {
      laswp_kernel<T><<<cdiv(n, 256), 256, 0, s>>>(A, n, lda, j0, jb, ipiv);
      note_launches(2);  // panel + row swaps
      return cudaGetLastError();
    }
  };
  // X (jb rows x ncols, ld lda) := L^{-1} X with L the unit lower jb x jb block at D
  auto trsm_lower = [&](const V* D, int jb, V* X, int64_t ncols) -> cudaError_t {
    if constexpr (sizeof(T) == 4) {
      return tri_lower_unit_cols(D, lda, jb, X, lda, ncols, s);  // a thread per column
    } else {
      enable_trsv_smem<T>();
      trsv_warp_kernel<T><<<cdiv(ncols, 8), 256, size_t(jb) * jb * sizeof(V), s>>>(D, lda, jb, 0, X, lda, ncols);
      return launched();
    }
  };
  if constexpr (sizeof(T) == 4) {
    // complex64 factors: outer blocks of NB = 256 columns, each factored as four 64-column
    // panels (each panel's L updates the block's columns to its right), then the block's U12
    // rows panel by panel, then one tensor-core trailing update with K = 256, so the trailing
    // matrix streams through HBM a quarter as often as 64-column blocking would.
    const int64_t NB = kLuBlock;
    for (int64_t j0 = 0; j0 < n && st == FOSB_OK; j0 += NB) {
      const int jb = int(std::min<int64_t>(NB, n - j0));
      V* Ab = A + j0 * lda + j0;
      cudaError_t e = cudaSuccess;
      for (int p0 = 0; p0 < jb && e == cudaSuccess; p0 += nb) {
        const int pw = std::min(nb, jb - p0), right = jb - p0 - pw;
        e = panel_step(j0 + p0, pw);
        if (e == cudaSuccess && right > 0) {
          V* Dp = Ab + int64_t(p0) * lda + p0;  // the panel's diagonal block
          e = trsm_lower(Dp, pw, Dp + pw, right);
          if (e == cudaSuccess)
            e = cgemm_update_tc(n - j0 - p0 - pw, right, pw, Dp + int64_t(pw) * lda, lda, Dp + pw, lda,
                                Dp + int64_t(pw) * lda + pw, lda, d_status, s, "lu_update64");
        }
      }
      const int64_t rest = n - j0 - jb;
      if (e == cudaSuccess && rest > 0) {
        // U12 = L11^{-1} A12 for the block's rows, one 64-row sweep and its coupling update per panel
        for (int p0 = 0; p0 < jb && e == cudaSuccess; p0 += nb) {
          const int pw = std::min(nb, jb - p0), below = jb - p0 - pw;
          V* Dp = Ab + int64_t(p0) * lda + p0;
          V* Up = Ab + int64_t(p0) * lda + jb;
          e = trsm_lower(Dp, pw, Up, rest);
          if (e == cudaSuccess && below > 0)
            e = cgemm_update_tc(below, rest, pw, Dp + int64_t(pw) * lda, lda, Up, lda, Up + int64_t(pw) * lda, lda,
                                d_status, s, "lu_update64");
        }
        if (e == cudaSuccess)
          e = cgemm_update_tc_split(rest, rest, jb, Ab + int64_t(jb) * lda, lda, Ab + jb, lda,
                                    Ab + int64_t(jb) * lda + jb, lda, d_status, ws_a, ws_b, s);
      }
      if (e != cudaSuccess) st = cuda_fail(e, "getrf: blocked step");
    }
  } else {
    for (int64_t j0 = 0; j0 < n && st == FOSB_OK; j0 += nb) {
      int jb = int(std::min<int64_t>(nb, n - j0));
      V* Ap = A + j0 * lda + j0;
      cudaError_t e = panel_step(j0, jb);
      if (e != cudaSuccess) {
        st = cuda_fail(e, "getrf: cooperative panel launch");
        break;
      }
      int64_t rest = n - j0 - jb;
      if (rest > 0) {
        e = trsm_lower(Ap, jb, Ap + jb, rest);
        if (e == cudaSuccess)
          e = gemm<T>(OP_N, OP_N, rest, rest, jb, -1.0, 0.0, Ap + jb * lda, lda, Ap + jb, lda, 1.0,
                      Ap + jb * lda + jb, lda, s);
        if (e != cudaSuccess) {
          st = cuda_fail(e, "getrf: trailing update");
          break;
        }
      }
    }
  }
  cudaFreeAsync(scratch, s);
  if (tslu_scr) cudaFreeAsync(tslu_scr, s);
  if (ws_a) cudaFreeAsync(ws_a, s);
  if (ws_b) cudaFreeAsync(ws_b, s);
  return st;
}

template fosb_status getrf<double>(void*, int64_t, int64_t, int32_t*, int*, cudaStream_t);
template fosb_status getrf<float>(void*, int64_t, int64_t, int32_t*, int*, cudaStream_t);

size_t getrf_scratch_bytes(int64_t max_ctas, bool c128) {
  const size_t v = c128 ? 16 : 8, nb = 64;
  return 256 + 2 * size_t(max_ctas) * nb * v + 2 * nb * v;
}

// The same blocked factorisation as getrf, with the panel kernel's scratch (barrier
// words and pivot candidates, getrf_scratch_bytes(max_ctas)) supplied by the caller;
// allocates nothing.  The first 256 bytes of `scratch` must be zero on entry.
template <typename T>
fosb_status getrf_external_scratch(void* Av, int64_t n, int64_t lda, int32_t* ipiv, int* d_status, void* scratch,
                                   int64_t max_ctas, cudaStream_t s) {
  using V = typename C2<T>::type;
  V* A = static_cast<V*>(Av);
  const int nb = 64;
  int dev = 0, nsm = 0, per_sm = 0;
  FOSB_CUDA(cudaGetDevice(&dev));
  FOSB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  FOSB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, panel_kernel<T>, kPanelThreads, 0));
  if (per_sm < 1) return fail(FOSB_ERR_CUDA, "getrf: panel kernel cannot be resident");
  const int64_t G_cap = std::min<int64_t>(int64_t(nsm) * per_sm, max_ctas);
  char* base = static_cast<char*>(scratch);
  PanelScratch* scr = reinterpret_cast<PanelScratch*>(base);
  V* cand_data = reinterpret_cast<V*>(base + 256);
  V* rowj = cand_data + 2 * max_ctas * nb;
  unsigned arrivals = 0;
  for (int64_t j0 = 0; j0 < n; j0 += nb) {
    int jb = int(std::min<int64_t>(nb, n - j0));
    int64_t m = n - j0;
    V* Ap = A + j0 * lda + j0;
    int32_t* ip = ipiv + j0;
    FOSB_CUDA(launch_panel<T>(Ap, m, jb, lda, ip, j0, scr, arrivals, cand_data, rowj, d_status, G_cap, nsm, s));
    laswp_kernel<T><<<cdiv(n, 256), 256, 0, s>>>(A, n, lda, j0, jb, ipiv);
    note_launches(2);
    int64_t rest = n - j0 - jb;
    if (rest > 0) {
      enable_trsv_smem<T>();
      trsv_warp_kernel<T><<<cdiv(rest, 8), 256, size_t(jb) * jb * sizeof(V), s>>>(Ap, lda, jb, 0, Ap + jb, lda, rest);
      note_launches(1);
      if constexpr (sizeof(T) == 4)
        FOSB_CUDA(cgemm_update_tc(rest, rest, jb, Ap + jb * lda, lda, Ap + jb, lda, Ap + jb * lda + jb, lda, d_status, s,
                                  "lu_update64"));
      else
        FOSB_CUDA(gemm<T>(OP_N, OP_N, rest, rest, jb, -1.0, 0.0, Ap + jb * lda, lda, Ap + jb, lda, 1.0,
                        Ap + jb * lda + jb, lda, s));
    }
    FOSB_CUDA(cudaGetLastError());
  }
  return FOSB_OK;
}

fosb_status getrf_external_max_n(int64_t max_ctas, int64_t* max_n) {
  int dev = 0, nsm = 0;
  FOSB_CUDA(cudaGetDevice(&dev));
  FOSB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // the first panel holds all n rows in at most min(SMs, max_ctas) CTAs of kMaxPanelRows rows
  *max_n = std::min<int64_t>(nsm, max_ctas) * kMaxPanelRows;
  return FOSB_OK;
}

template fosb_status getrf_external_scratch<double>(void*, int64_t, int64_t, int32_t*, int*, void*, int64_t,
                                                    cudaStream_t);
template fosb_status getrf_external_scratch<float>(void*, int64_t, int64_t, int32_t*, int*, void*, int64_t,
                                                   cudaStream_t);

// X <- Z^{-1} X given the factors (perm = composed row permutation, device).
template <typename T>
cudaError_t getrs(const void* LUv, int64_t n, int64_t ldlu, const int32_t* perm, void* Xv, int64_t nrhs, int64_t ldx,
                  cudaStream_t s, int* status, const void* dinv) {
  using V = typename C2<T>::type;
  const V* LU = static_cast<const V*>(LUv);
  V* X = static_cast<V*>(Xv);
  V* tmp = nullptr;
  ProfScope prof("getrs", s, 8.0 * double(n) * double(n) * double(nrhs));
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&tmp), sizeof(V) * n * nrhs, s);
  if (e != cudaSuccess) return e;
  gather_rows_kernel<T><<<cdiv(n * nrhs, 256), 256, 0, s>>>(X, ldx, perm, n, nrhs, tmp, nrhs);
  if (sizeof(T) == 4 && status && dinv && nrhs <= kTrsvStreamMaxRhs) {
    // one persistent streaming kernel per sweep
    int* flags = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void**>(&flags), sizeof(int) * trsv_stream_scratch_ints(n, nrhs), s);
    if (e == cudaSuccess) e = trsv_stream_c64(LU, n, ldlu, dinv, tmp, nrhs, 0, flags, status, s);
    if (e == cudaSuccess) e = trsv_stream_c64(LU, n, ldlu, dinv, tmp, nrhs, 1, flags, status, s);
    if (flags) cudaFreeAsync(flags, s);
    if (e != cudaSuccess) {
      cudaFreeAsync(tmp, s);
      return e;
    }
    copy_kernel<V><<<cdiv(n * nrhs, 256), 256, 0, s>>>(tmp, n, nrhs, nrhs, X, ldx);
    note_launches(2);  // gather + final copy
    cudaFreeAsync(tmp, s);
    return cudaGetLastError();
  }
  const int nb = 64;
  enable_trsv_smem<T>();
  auto diag = [&](int64_t i0, int ib, int upper) {
    const V* D = LU + i0 * ldlu + i0;
    trsv_warp_kernel<T><<<cdiv(nrhs, 8), 256, size_t(ib) * ib * sizeof(V), s>>>(D, ldlu, ib, upper, tmp + i0 * nrhs,
                                                                               nrhs, nrhs);
    note_launches(1);
  };
  note_launches(2);  // gather + final copy
  // forward: unit lower
  for (int64_t i0 = 0; i0 < n; i0 += nb) {
    int ib = int(std::min<int64_t>(nb, n - i0));
    diag(i0, ib, 0);
    int64_t rest = n - i0 - ib;
    if (rest > 0) {
      if (sizeof(T) == 4 && status && nrhs >= 16)  // wide right-hand sides: tensor cores
        e = cgemm_update_tc(rest, nrhs, ib, LU + (i0 + ib) * ldlu + i0, ldlu, tmp + i0 * nrhs, nrhs,
                            tmp + (i0 + ib) * nrhs, nrhs, status, s, "trsm_update");
      else
        e = gemm<T>(OP_N, OP_N, rest, nrhs, ib, -1.0, 0.0, LU + (i0 + ib) * ldlu + i0, ldlu, tmp + i0 * nrhs, nrhs,
                    1.0, tmp + (i0 + ib) * nrhs, nrhs, s);
      if (e != cudaSuccess) {
        cudaFreeAsync(tmp, s);
        return e;
      }
    }
  }
  // backward: upper
  for (int64_t i1 = n; i1 > 0; i1 -= nb) {
    int64_t i0 = std::max<int64_t>(0, i1 - nb);
    int ib = int(i1 - i0);
    diag(i0, ib, 1);
    if (i0 > 0) {
      if (sizeof(T) == 4 && status && nrhs >= 16)
        e = cgemm_update_tc(i0, nrhs, ib, LU + i0, ldlu, tmp + i0 * nrhs, nrhs, tmp, nrhs, status, s, "trsm_update");
      else
        e = gemm<T>(OP_N, OP_N, i0, nrhs, ib, -1.0, 0.0, LU + i0, ldlu, tmp + i0 * nrhs, nrhs, 1.0, tmp, nrhs, s);
      if (e != cudaSuccess) {
        cudaFreeAsync(tmp, s);
        return e;
      }
    }
  }
  copy_kernel<V><<<cdiv(n * nrhs, 256), 256, 0, s>>>(tmp, n, nrhs, nrhs, X, ldx);
  cudaFreeAsync(tmp, s);
  return cudaGetLastError();
}

template cudaError_t getrs<double>(const void*, int64_t, int64_t, const int32_t*, void*, int64_t, int64_t, cudaStream_t,
                                   int*, const void*);
template cudaError_t getrs<float>(const void*, int64_t, int64_t, const int32_t*, void*, int64_t, int64_t, cudaStream_t,
                                  int*, const void*);

cudaError_t convert_c128_to_c64(const void* src, int64_t rows, int64_t cols, int64_t lds, void* dst, int64_t ldd,
                                cudaStream_t s) {
  if (rows * cols == 0) return cudaSuccess;
  c128_to_c64_kernel<<<cdiv(rows * cols, 256), 256, 0, s>>>(static_cast<const double2*>(src), rows, cols, lds,
                                                            static_cast<float2*>(dst), ldd);
  return launched();
}
cudaError_t convert_c64_to_c128(const void* src, int64_t rows, int64_t cols, int64_t lds, void* dst, int64_t ldd,
                                cudaStream_t s) {
  if (rows * cols == 0) return cudaSuccess;
  c64_to_c128_kernel<<<cdiv(rows * cols, 256), 256, 0, s>>>(static_cast<const float2*>(src), rows, cols, lds,
                                                            static_cast<double2*>(dst), ldd);
  return launched();
}
cudaError_t copy_matrix(const void* src, int64_t rows, int64_t cols, int64_t lds, void* dst, int64_t ldd, size_t elem,
                        cudaStream_t s) {
  return cudaMemcpy2DAsync(dst, ldd * elem, src, lds * elem, cols * elem, rows, cudaMemcpyDeviceToDevice, s);
}
cudaError_t axpy_c64_into_c128(const void* d, int64_t rows, int64_t cols, int64_t ldd, void* x, int64_t ldx,
                               cudaStream_t s) {
  if (rows * cols == 0) return cudaSuccess;
  axpy_kernel<<<cdiv(rows * cols, 256), 256, 0, s>>>(static_cast<const float2*>(d), rows, cols, ldd,
                                                     static_cast<double2*>(x), ldx);
  return launched();
}
cudaError_t add_mirrored(const void* M, int64_t n, int64_t ldm, int op, double w, bool accumulate, bool c64, void* out,
                         int64_t ldo, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (c64)
    add_mirrored_kernel<float><<<cdiv(n * n, 256), 256, 0, s>>>(static_cast<const float2*>(M), n, ldm, op, float(w),
                                                                accumulate, static_cast<float2*>(out), ldo);
  else
    add_mirrored_kernel<double><<<cdiv(n * n, 256), 256, 0, s>>>(static_cast<const double2*>(M), n, ldm, op, w,
                                                                 accumulate, static_cast<double2*>(out), ldo);
  return launched();
}

cudaError_t norm_inf_c128(const void* A, int64_t rows, int64_t cols, int64_t lda, double* d_out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  row_norm_kernel<<<cdiv(rows, 8), 256, 0, s>>>(static_cast<const double2*>(A), rows, cols, lda, d_out);
  return launched();
}
cudaError_t absmax_c128(const void* A, int64_t rows, int64_t cols, int64_t lda, double* d_out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(double) * cols, s);
  if (e != cudaSuccess) return e;
  if (rows * cols == 0) return cudaSuccess;
  col_absmax_kernel<<<cdiv(rows * cols, 256), 256, 0, s>>>(static_cast<const double2*>(A), rows, cols, lda, d_out);
  return launched();
}

// Sets the poll limit of the panel grid-barrier waits on the current device (polls <= 0:
// the default).
cudaError_t set_wait_limit_panels(long long polls) {
  const long long v = polls > 0 ? polls : kSpinLimit;
  return cudaMemcpyToSymbol(g_wait_limit, &v, sizeof(v));
}

}  // namespace fosb
