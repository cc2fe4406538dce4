// Streaming triangular solves with complex64 factors for a few right-hand sides (A6: the
// forward and backward sweeps L y = P b, U x = y of every refined solve).
//
// A blocked sweep that launches one diagonal solve and one panel update per 64-row block
// is latency-bound for one right-hand side (2 x n/64 dependent launches per sweep).  Here
// one persistent kernel does a whole sweep: CTAs take 64-row blocks in order from a ticket
// counter; the CTA of block i accumulates L_ij y_j (U_ij x_j for the backward sweep) over
// the blocks j that precede it in the sweep as each one is published, then solves its
// diagonal block (a 64 x 64 product with its precomputed inverse) and publishes y_i
// through flags[i].  A block
// only waits for blocks that were taken earlier, by CTAs that are running or done, so the
// waits always end; each is bounded anyway and a time-out sets the status word, which every
// waiter polls, so the sweep ends quickly and the host reports FOSB_ERR_TIMEOUT.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "fosb_internal.h"

namespace fosb {
namespace {

constexpr int kTB = 64;                         // rows per block
constexpr long long kFlagSpinLimit = 1ll << 26;

__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {  // acc += a b
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

// Inverse of each 64 x 64 diagonal block of the factors (unit lower L_ii for which = 0,
// upper U_ii for which = 1), row-major in Dinv[i][64][64]: one CTA per block, each warp
// substitutes 8 unit columns.  Used by the streaming sweeps so that the critical path of a
// block is a parallel 64 x 64 matrix-vector product instead of a 64-step substitution.
__global__ void __launch_bounds__(256) tri_block_inverse_kernel(const float2* __restrict__ LU, int64_t n, int64_t ld,
                                                                int which, float2* __restrict__ Dinv) {
  __shared__ float2 sDt[kTB][kTB + 1];  // sDt[k][r] = D[r][k]
  const int64_t ib = blockIdx.x, r0 = ib * kTB;
  const int rows = int(std::min<int64_t>(kTB, n - r0));
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int e = t; e < kTB * kTB; e += blockDim.x) {
    const int rr = e / kTB, kk = e % kTB;
    sDt[kk][rr] = (rr < rows && kk < rows) ? LU[(r0 + rr) * ld + r0 + kk] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2* out = Dinv + ib * kTB * kTB;
  const float2 zero = make_float2(0.f, 0.f);
  for (int cidx = 0; cidx < 8; ++cidx) {
    const int col = warp * 8 + cidx;  // column of the inverse: solve D x = e_col
    float2 x0 = lane == col ? make_float2(1.f, 0.f) : zero;
    float2 x1 = lane + 32 == col ? make_float2(1.f, 0.f) : zero;
    if (col >= rows) {
      x0 = x1 = zero;
    } else if (which == 0) {
      for (int i = 0; i < rows - 1; ++i) {
        float2 xi = i < 32 ? x0 : x1;
        xi.x = __shfl_sync(0xffffffffu, xi.x, i & 31);
        xi.y = __shfl_sync(0xffffffffu, xi.y, i & 31);
        if (lane > i && lane < rows) {
          const float2 d = sDt[i][lane];
          x0.x -= d.x * xi.x - d.y * xi.y;
          x0.y -= d.x * xi.y + d.y * xi.x;
        }
        if (lane + 32 > i && lane + 32 < rows) {
          const float2 d = sDt[i][lane + 32];
          x1.x -= d.x * xi.x - d.y * xi.y;
          x1.y -= d.x * xi.y + d.y * xi.x;
        }
      }
    } else {
      for (int i = rows - 1; i >= 0; --i) {
        const float2 d = sDt[i][i];
        const float den = d.x * d.x + d.y * d.y;
        const bool mine0 = i < 32 && lane == i, mine1 = i >= 32 && lane == i - 32;
        if (mine0 || mine1) {
          const float2 v = mine0 ? x0 : x1;
          const float2 qv =
              den > 0.f ? make_float2((v.x * d.x + v.y * d.y) / den, (v.y * d.x - v.x * d.y) / den) : zero;
          if (mine0) x0 = qv; else x1 = qv;
        }
        float2 xi = i < 32 ? x0 : x1;
        xi.x = __shfl_sync(0xffffffffu, xi.x, i & 31);
        xi.y = __shfl_sync(0xffffffffu, xi.y, i & 31);
        if (lane < i) {
          const float2 dd = sDt[i][lane];
          x0.x -= dd.x * xi.x - dd.y * xi.y;
          x0.y -= dd.x * xi.y + dd.y * xi.x;
        }
        if (lane + 32 < i) {
          const float2 dd = sDt[i][lane + 32];
          x1.x -= dd.x * xi.x - dd.y * xi.y;
          x1.y -= dd.x * xi.y + dd.y * xi.x;
        }
      }
    }
    out[lane * kTB + col] = x0;  // Dinv[row][col]
    out[(lane + 32) * kTB + col] = x1;
  }
}

template <int NR>
__global__ void __launch_bounds__(256) trsv_stream_kernel(const float2* __restrict__ LU, int64_t n, int64_t ld,
                                                          const float2* __restrict__ Dinv, float2* X, int upper,
                                                          int* ticket, int* flags, int* status) {
  __shared__ float2 sY[kTB][NR];          // the published block being consumed
  __shared__ float2 sR[kTB][NR];          // this block's right-hand side after the panel product
  __shared__ float2 sDi[kTB][kTB + 1];    // inverse of this block's diagonal block
  __shared__ long long s_blk;
  __shared__ int s_abort;
  const int t = threadIdx.x;
  const int r = t >> 2, q = t & 3;        // row r of the block, columns q*16 .. q*16+15
  const int64_t nblk = (n + kTB - 1) / kTB;
  for (;;) {
    if (t == 0) {
      s_blk = atomicAdd(ticket, 1);
      s_abort = 0;
    }
    __syncthreads();
    const int64_t b = s_blk;
    if (b >= nblk) break;
    const int64_t ib = upper ? nblk - 1 - b : b;
    const int64_t r0 = ib * kTB;
    const int rows = int(std::min<int64_t>(kTB, n - r0));
    for (int e = t; e < kTB * kTB; e += blockDim.x) sDi[e / kTB][e % kTB] = Dinv[ib * kTB * kTB + e];
    float2 acc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) acc[k] = make_float2(0.f, 0.f);
    const int64_t jcount = upper ? nblk - 1 - ib : ib;
    for (int64_t jj = 0; jj < jcount; ++jj) {
      const int64_t jb = upper ? nblk - 1 - jj : jj;  // in publication order
      const int64_t c0 = jb * kTB;
      const int cols = int(std::min<int64_t>(kTB, n - c0));
      // this thread's 16 factor entries do not depend on the block being waited for
      float2 lreg[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int cc = q * 16 + c;
        lreg[c] = (r < rows && cc < cols) ? __ldg(LU + (r0 + r) * ld + c0 + cc) : make_float2(0.f, 0.f);
      }
      if (t == 0) {
        const volatile int* f = flags + jb;
        long long spins = 0;
        while (*f == 0) {
          if (++spins > kFlagSpinLimit || *(volatile int*)status == FOSB_ERR_TIMEOUT) {
            atomicExch(status, FOSB_ERR_TIMEOUT);
            s_abort = 1;
            break;
          }
          __nanosleep(32);
        }
        __threadfence();
      }
      __syncthreads();  // also: every thread is done with sY of the previous block
      if (s_abort) break;
      for (int e = t; e < cols * NR; e += blockDim.x) sY[e / NR][e % NR] = __ldcg(X + (c0 + e / NR) * NR + e % NR);
      __syncthreads();
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int cc = q * 16 + c;
        if (cc < cols) {
#pragma unroll
          for (int k = 0; k < NR; ++k) cfma(acc[k], lreg[c], sY[cc][k]);
        }
      }
    }
    if (s_abort) {  // every later wait gives up at once; this block stays unpublished
      __syncthreads();
      continue;
    }
    // reduce the four column quarters of each row; right-hand side of the diagonal block
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      acc[k].x += __shfl_xor_sync(0xffffffffu, acc[k].x, 1);
      acc[k].y += __shfl_xor_sync(0xffffffffu, acc[k].y, 1);
      acc[k].x += __shfl_xor_sync(0xffffffffu, acc[k].x, 2);
      acc[k].y += __shfl_xor_sync(0xffffffffu, acc[k].y, 2);
    }
    if (q == 0) {
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        float2 v = make_float2(0.f, 0.f);
        if (r < rows) {
          const float2 x = X[(r0 + r) * NR + k];
          v = make_float2(x.x - acc[k].x, x.y - acc[k].y);
        }
        sR[r][k] = v;
      }
    }
    __syncthreads();
    // y = Dinv r: row r, quarter q of the columns, then the same quarter reduction
    float2 y[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) y[k] = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const float2 d = sDi[r][q * 16 + c];
#pragma unroll
      for (int k = 0; k < NR; ++k) cfma(y[k], d, sR[q * 16 + c][k]);
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      y[k].x += __shfl_xor_sync(0xffffffffu, y[k].x, 1);
      y[k].y += __shfl_xor_sync(0xffffffffu, y[k].y, 1);
      y[k].x += __shfl_xor_sync(0xffffffffu, y[k].x, 2);
      y[k].y += __shfl_xor_sync(0xffffffffu, y[k].y, 2);
    }
    if (q == 0 && r < rows) {
#pragma unroll
      for (int k = 0; k < NR; ++k) X[(r0 + r) * NR + k] = y[k];
    }
    __threadfence();
    __syncthreads();
    if (t == 0) atomicExch(flags + ib, 1);  // publish block ib
  }
}

}  // namespace

size_t trsv_stream_scratch_ints(int64_t n) { return size_t(2 * ((n + kTB - 1) / kTB) + 64); }

cudaError_t tri_block_inverses_c64(const void* LU, int64_t n, int64_t ld, void* Dinv, cudaStream_t s) {
  const int64_t nblk = (n + kTB - 1) / kTB;
  if (nblk <= 0) return cudaSuccess;
  float2* d = static_cast<float2*>(Dinv);
  tri_block_inverse_kernel<<<unsigned(nblk), 256, 0, s>>>(static_cast<const float2*>(LU), n, ld, 0, d);
  tri_block_inverse_kernel<<<unsigned(nblk), 256, 0, s>>>(static_cast<const float2*>(LU), n, ld, 1,
                                                           d + nblk * kTB * kTB);
  return launched(2);
}

size_t tri_block_inverses_bytes(int64_t n) { return size_t(2 * ((n + kTB - 1) / kTB)) * kTB * kTB * sizeof(float2); }

cudaError_t trsv_stream_c64(const void* LU, int64_t n, int64_t ld, const void* Dinv, void* X, int64_t nrhs, int upper,
                            int* scratch, int* status, cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (nrhs > 8) return cudaErrorInvalidValue;
  static int nsm[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!nsm[dev]) cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev);
  const int64_t nblk = (n + kTB - 1) / kTB;
  int* ticket = scratch;
  int* flags = scratch + 32;
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int) * (32 + nblk), s);
  if (e != cudaSuccess) return e;
  const unsigned grid = unsigned(std::min<int64_t>(nblk, int64_t(4) * std::max(nsm[dev], 1)));
  const float2* L = static_cast<const float2*>(LU);
  const float2* D = static_cast<const float2*>(Dinv) + (upper ? nblk * kTB * kTB : 0);
  float2* x = static_cast<float2*>(X);
#define FOSB_TS(NR) trsv_stream_kernel<NR><<<grid, 256, 0, s>>>(L, n, ld, D, x, upper, ticket, flags, status)
  switch (nrhs) {
    case 1: FOSB_TS(1); break;
    case 2: FOSB_TS(2); break;
    case 3: FOSB_TS(3); break;
    case 4: FOSB_TS(4); break;
    case 5: FOSB_TS(5); break;
    case 6: FOSB_TS(6); break;
    case 7: FOSB_TS(7); break;
    default: FOSB_TS(8); break;
  }
#undef FOSB_TS
  return launched();
}

}  // namespace fosb
