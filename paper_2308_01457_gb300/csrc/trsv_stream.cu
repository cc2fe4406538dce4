// Streaming triangular solves with complex64 factors (A6: the forward and backward sweeps
// L y = P b, U x = y of every refined solve, and of the multi-right-hand-side covariance solves).
//
// A blocked sweep that launches one diagonal solve and one panel update per 64-row block
// is latency-bound (2 x n/64 dependent launches per sweep).  Here one persistent kernel
// does a whole sweep.  The right-hand sides are cut into chunks of at most 16 columns (one
// chunk of the exact width for 1-8); CTAs take (block, chunk) tasks in block-major order
// from a ticket counter.  The CTA of task (i, c) accumulates L_ij y_j (U_ij x_j for the
// backward sweep) over the blocks j that precede i in the sweep as chunk c of each one is
// published, then solves its diagonal block (a 64 x 64 product with its precomputed
// inverse) and publishes chunk c of y_i through flags[i * chunks + c].  A task only waits
// for tasks that were taken earlier, by CTAs that are running or done, so the waits always
// end; each is bounded anyway and a time-out sets the status word, which every waiter
// polls, so the sweep ends quickly and the host reports FOSB_ERR_TIMEOUT.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "fosb_internal.h"

namespace fosb {
namespace {

constexpr int kTB = 64;                         // rows per block
constexpr long long kFlagSpinLimit = 1ll << 26;
// Poll limit of the flag waits on this device (kFlagSpinLimit unless changed by
// fosb_debug_set_wait_limit).
__device__ long long g_flag_wait_limit = kFlagSpinLimit;

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

// Shared tiles of the streaming sweep.  A factor tile (and, after the panel product, the
// inverse of the diagonal block) is 64 x 64 with a row pitch of 72 complex values; the
// published block of the solution is 64 x NR with an odd pitch NRP.  Thread (g, q) of 256
// owns rows g and g + 32 and the columns q, q + 8, ..., q + 56, so in one step of c the 16
// threads of a half-warp read 8 consecutive complex values of two rows 72 apart (every bank
// once) and 8 values of the solution block 2 NRP words apart (distinct banks, NRP odd).
constexpr int kLP = 72;
template <int NR>
struct StreamSmem {
  static constexpr int NRP = NR | 1;
  float2 L[kTB][kLP];
  float2 Y[kTB][NRP];
};

// acc0/acc1 (rows g, g + 32) += T[rows][cols] Y[cols][0..NR) over this thread's 8 columns
template <int NR>
__device__ __forceinline__ void stream_tile_product(const StreamSmem<NR>& sm, int g, int q, float2 (&acc0)[NR],
                                                    float2 (&acc1)[NR]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int cc = q + 8 * c;
    const float2 l0 = sm.L[g][cc], l1 = sm.L[g + 32][cc];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const float2 y = sm.Y[cc][k];
      cfma(acc0[k], l0, y);
      cfma(acc1[k], l1, y);
    }
  }
}
// sum over the 8 column owners q (lanes differing in their low three bits)
template <int NR>
__device__ __forceinline__ void stream_reduce_q(float2 (&a)[NR]) {
#pragma unroll
  for (int k = 0; k < NR; ++k) {
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {
      a[k].x += __shfl_xor_sync(0xffffffffu, a[k].x, off);
      a[k].y += __shfl_xor_sync(0xffffffffu, a[k].y, off);
    }
  }
}

template <int NR>
__global__ void __launch_bounds__(256, 2) trsv_stream_kernel(const float2* __restrict__ LU, int64_t n, int64_t ld,
                                                          const float2* __restrict__ Dinv, float2* X, int64_t ldx,
                                                          int nrhs, int chunks, int upper, int* ticket, int* flags,
                                                          int* status) {
  extern __shared__ float4 stream_raw[];
  StreamSmem<NR>& sm = *reinterpret_cast<StreamSmem<NR>*>(stream_raw);
  __shared__ long long s_task;
  __shared__ int s_abort;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int g = t >> 3, q = t & 7;
  const int64_t nblk = (n + kTB - 1) / kTB;
  for (;;) {
    if (t == 0) {
      s_task = atomicAdd(ticket, 1);
      s_abort = 0;
    }
    __syncthreads();
    const int64_t task = s_task;
    const int64_t b = task / chunks;
    const int ch = int(task % chunks);
    if (b >= nblk) break;
    const int64_t ib = upper ? nblk - 1 - b : b;
    const int64_t r0 = ib * kTB;
    const int rows = int(std::min<int64_t>(kTB, n - r0));
    const int k0 = ch * NR, nc = std::min(NR, nrhs - k0);  // this chunk's columns of X
    float2 acc0[NR], acc1[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) acc0[k] = acc1[k] = make_float2(0.f, 0.f);
    const int64_t jcount = upper ? nblk - 1 - ib : ib;
    // factor tile of block jj in registers: warp w holds rows 8w .. 8w+7, lanes the columns
    // lane and lane + 32 (256 contiguous bytes of a row per load instruction)
    float2 lreg[16];
    auto fetch = [&](int64_t jj) {
      const int64_t c0 = (upper ? nblk - 1 - jj : jj) * kTB;
      const int cols = int(std::min<int64_t>(kTB, n - c0));
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int rr = warp * 8 + i;
        const float2* src = LU + (r0 + rr) * ld + c0;
        lreg[2 * i] = (rr < rows && lane < cols) ? __ldg(src + lane) : make_float2(0.f, 0.f);
        lreg[2 * i + 1] = (rr < rows && lane + 32 < cols) ? __ldg(src + lane + 32) : make_float2(0.f, 0.f);
      }
    };
    if (jcount > 0) fetch(0);
    for (int64_t jj = 0; jj < jcount; ++jj) {
      const int64_t jb = upper ? nblk - 1 - jj : jj;  // in publication order
      const int64_t c0 = jb * kTB;
      const int cols = int(std::min<int64_t>(kTB, n - c0));
      if (t == 0) {
        const volatile int* f = flags + jb * chunks + ch;
        long long spins = 0;
        const long long limit = g_flag_wait_limit;
        while (*f == 0) {
          if (++spins > limit || *(volatile int*)status == FOSB_ERR_TIMEOUT) {
            atomicExch(status, FOSB_ERR_TIMEOUT);
            s_abort = 1;
            break;
          }
          __nanosleep(32);
        }
        __threadfence();
      }
      __syncthreads();  // also: every thread is done with the tiles of the previous block
      if (s_abort) break;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        sm.L[warp * 8 + i][lane] = lreg[2 * i];
        sm.L[warp * 8 + i][lane + 32] = lreg[2 * i + 1];
      }
      for (int e = t; e < kTB * NR; e += blockDim.x) {
        const int rr = e / NR, k = e % NR;
        sm.Y[rr][k] = (rr < cols && k < nc) ? __ldcg(X + (c0 + rr) * ldx + k0 + k) : make_float2(0.f, 0.f);
      }
      if (jj + 1 < jcount) fetch(jj + 1);  // in flight during the product below
      __syncthreads();
      stream_tile_product<NR>(sm, g, q, acc0, acc1);
    }
    if (s_abort) {  // every later wait gives up at once; this task stays unpublished
      __syncthreads();
      continue;
    }
    // right-hand side of the diagonal block: r = x - sum_j L_ij y_j
    stream_reduce_q<NR>(acc0);
    stream_reduce_q<NR>(acc1);
    __syncthreads();  // every thread is done with the last factor tile
    if (q == 0) {
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        float2 v0 = make_float2(0.f, 0.f), v1 = v0;
        if (k < nc) {
          if (g < rows) {
            const float2 x = X[(r0 + g) * ldx + k0 + k];
            v0 = make_float2(x.x - acc0[k].x, x.y - acc0[k].y);
          }
          if (g + 32 < rows) {
            const float2 x = X[(r0 + g + 32) * ldx + k0 + k];
            v1 = make_float2(x.x - acc1[k].x, x.y - acc1[k].y);
          }
        }
        sm.Y[g][k] = v0;
        sm.Y[g + 32][k] = v1;
      }
    }
    const float2* D = Dinv + ib * kTB * kTB;
    for (int e = t; e < kTB * kTB; e += blockDim.x) sm.L[e / kTB][e % kTB] = D[e];
    __syncthreads();
    // y = Dinv r, the same tile product
#pragma unroll
    for (int k = 0; k < NR; ++k) acc0[k] = acc1[k] = make_float2(0.f, 0.f);
    stream_tile_product<NR>(sm, g, q, acc0, acc1);
    stream_reduce_q<NR>(acc0);
    stream_reduce_q<NR>(acc1);
    if (q == 0) {
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        if (k < nc) {
          if (g < rows) X[(r0 + g) * ldx + k0 + k] = acc0[k];
          if (g + 32 < rows) X[(r0 + g + 32) * ldx + k0 + k] = acc1[k];
        }
      }
    }
    __threadfence();
    __syncthreads();
    if (t == 0) atomicExch(flags + ib * chunks + ch, 1);  // publish chunk ch of block ib
  }
}

}  // namespace

// chunk width: the exact width for 1-8 right-hand sides, 16 above
static int trsv_stream_width(int64_t nrhs) { return nrhs <= 8 ? int(nrhs) : 16; }

size_t trsv_stream_scratch_ints(int64_t n, int64_t nrhs) {
  const int64_t w = trsv_stream_width(std::max<int64_t>(nrhs, 1));
  return size_t(((n + kTB - 1) / kTB) * ((nrhs + w - 1) / w) + 64);
}

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
  if (nrhs > kTrsvStreamMaxRhs) return cudaErrorInvalidValue;
  static int nsm[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!nsm[dev]) cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev);
  const int64_t nblk = (n + kTB - 1) / kTB;
  const int w = trsv_stream_width(nrhs);
  const int chunks = int((nrhs + w - 1) / w);
  int* ticket = scratch;
  int* flags = scratch + 32;
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int) * (32 + nblk * chunks), s);
  if (e != cudaSuccess) return e;
  const unsigned grid = unsigned(std::min<int64_t>(nblk * chunks, int64_t(2) * std::max(nsm[dev], 1)));
  const float2* L = static_cast<const float2*>(LU);
  const float2* D = static_cast<const float2*>(Dinv) + (upper ? nblk * kTB * kTB : 0);
  float2* x = static_cast<float2*>(X);
  const int nr = int(nrhs);
#define FOSB_TS(NR)                                                                                      \
  trsv_stream_kernel<NR><<<grid, 256, sizeof(StreamSmem<NR>), s>>>(L, n, ld, D, x, nrhs, nr, chunks, upper, ticket, \
                                                                   flags, status)
  switch (w) {
    case 1: FOSB_TS(1); break;
    case 2: FOSB_TS(2); break;
    case 3: FOSB_TS(3); break;
    case 4: FOSB_TS(4); break;
    case 5: FOSB_TS(5); break;
    case 6: FOSB_TS(6); break;
    case 7: FOSB_TS(7); break;
    case 8: FOSB_TS(8); break;
    default: FOSB_TS(16); break;
  }
#undef FOSB_TS
  return launched();
}

// Sets the poll limit of the sweep flag waits on the current device (polls <= 0: the default).
cudaError_t set_wait_limit_sweeps(long long polls) {
  const long long v = polls > 0 ? polls : kFlagSpinLimit;
  return cudaMemcpyToSymbol(g_flag_wait_limit, &v, sizeof(v));
}

}  // namespace fosb
