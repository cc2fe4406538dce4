// Streaming triangular solves with complex64 factors for a few right-hand sides (A6: the
// forward and backward sweeps L y = P b, U x = y of every refined solve).
//
// A blocked sweep that launches one diagonal solve and one panel update per 64-row block
// is latency-bound for one right-hand side (2 x n/64 dependent launches per sweep).  Here
// one persistent kernel does a whole sweep: CTAs take 64-row blocks in order from a ticket
// counter; the CTA of block i accumulates L_ij y_j (U_ij x_j for the backward sweep) over
// the blocks j that precede it in the sweep as each one is published, then solves its
// diagonal block (one warp per right-hand side) and publishes y_i through flags[i].  A block
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

template <int NR>
__global__ void __launch_bounds__(256) trsv_stream_kernel(const float2* __restrict__ LU, int64_t n, int64_t ld,
                                                          float2* X, int upper, int* ticket, int* flags,
                                                          int* status) {
  __shared__ float2 sY[kTB][NR];          // the published block being consumed
  __shared__ float2 sR[kTB][NR];          // this block's right-hand side after the panel product
  __shared__ float2 sDt[kTB][kTB + 1];    // diagonal block, transposed: sDt[k][r] = D[r][k]
  __shared__ long long s_blk;
  __shared__ int s_abort;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int r = t >> 2, q = t & 3;        // panel product: row r of the block, columns q*16 .. q*16+15
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
    float2 acc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) acc[k] = make_float2(0.f, 0.f);
    const int64_t jcount = upper ? nblk - 1 - ib : ib;
    for (int64_t jj = 0; jj < jcount; ++jj) {
      const int64_t jb = upper ? nblk - 1 - jj : jj;  // in publication order
      const int64_t c0 = jb * kTB;
      const int cols = int(std::min<int64_t>(kTB, n - c0));
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
      __syncthreads();
      if (s_abort) break;
      for (int e = t; e < cols * NR; e += blockDim.x) sY[e / NR][e % NR] = __ldcg(X + (c0 + e / NR) * NR + e % NR);
      __syncthreads();
      if (r < rows) {
        const float2* Lrow = LU + (r0 + r) * ld + c0 + q * 16;
#pragma unroll 4
        for (int c = 0; c < 16; ++c) {
          const int cc = q * 16 + c;
          if (cc < cols) {
            const float2 l = Lrow[c];
#pragma unroll
            for (int k = 0; k < NR; ++k) cfma(acc[k], l, sY[cc][k]);
          }
        }
      }
      __syncthreads();  // sY is rewritten for the next block
    }
    if (s_abort) {  // every later wait gives up at once; this block stays unpublished
      __syncthreads();
      continue;
    }
    // reduce the four column quarters of each row; right-hand side of the diagonal solve
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      acc[k].x += __shfl_xor_sync(0xffffffffu, acc[k].x, 1);
      acc[k].y += __shfl_xor_sync(0xffffffffu, acc[k].y, 1);
      acc[k].x += __shfl_xor_sync(0xffffffffu, acc[k].x, 2);
      acc[k].y += __shfl_xor_sync(0xffffffffu, acc[k].y, 2);
    }
    if (q == 0 && r < rows) {
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        const float2 v = X[(r0 + r) * NR + k];
        sR[r][k] = make_float2(v.x - acc[k].x, v.y - acc[k].y);
      }
    }
    for (int e = t; e < rows * rows; e += blockDim.x) {
      const int rr = e / rows, kk = e % rows;
      sDt[kk][rr] = LU[(r0 + rr) * ld + r0 + kk];
    }
    __syncthreads();
    if (warp < NR) {  // one warp per right-hand side; lanes own rows lane and lane + 32
      const float2 zero = make_float2(0.f, 0.f);
      float2 x0 = lane < rows ? sR[lane][warp] : zero;
      float2 x1 = lane + 32 < rows ? sR[lane + 32][warp] : zero;
      if (!upper) {
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
            const float2 qv = den > 0.f ? make_float2((v.x * d.x + v.y * d.y) / den, (v.y * d.x - v.x * d.y) / den)
                                        : zero;
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
      if (lane < rows) X[(r0 + lane) * NR + warp] = x0;
      if (lane + 32 < rows) X[(r0 + lane + 32) * NR + warp] = x1;
    }
    __threadfence();
    __syncthreads();
    if (t == 0) atomicExch(flags + ib, 1);  // publish block ib
  }
}

}  // namespace

size_t trsv_stream_scratch_ints(int64_t n) { return size_t(2 * ((n + kTB - 1) / kTB) + 64); }

cudaError_t trsv_stream_c64(const void* LU, int64_t n, int64_t ld, void* X, int64_t nrhs, int upper, int* scratch,
                            int* status, cudaStream_t s) {
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
  float2* x = static_cast<float2*>(X);
#define FOSB_TS(NR) trsv_stream_kernel<NR><<<grid, 256, 0, s>>>(L, n, ld, x, upper, ticket, flags, status)
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
