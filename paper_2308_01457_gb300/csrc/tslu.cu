// Tournament-pivoting panel factorisation (TSLU) of a complex64 m x jb panel (jb <= 64),
// for the blocked LU of the mixed and FP32 paths.
//
// Partial pivoting needs one grid-wide reduction per column.  Here the pivot rows of the
// whole panel are chosen by a reduction tree instead:
//   1. leaves: every CTA factors a block of up to 256 rows with partial pivoting and
//      nominates the rows it pivoted on (at most jb);
//   2. tree: CTAs merge up to 4 nominee sets (<= 256 rows, original values re-read from
//      the panel) the same way until one set of jb rows remains; its factorisation is
//      L11 \ U11 of the panel in the chosen pivot order;
//   3. apply: one CTA turns the chosen order into row interchanges (ipiv, in the usual
//      "row i was swapped with ipiv[i]" form), writes L11 \ U11 into the top jb rows and
//      moves the displaced rows;
//   4. L21 = A21 U11^{-1}, one warp per row.
// The panel stays untouched in global memory until step 3, so every level reads original
// rows.  Launches are stream-ordered; there is no inter-CTA wait anywhere.
//
// Within a CTA the candidate rows sit in shared memory, one per thread, and are factored
// by blocked partial pivoting in blocks of 8 columns: per step a warp argmax (one reduce
// and one ballot), one barrier, and the elimination of that column inside the block; per
// block the trailing columns of its pivot rows by forward substitution with the block's
// unit lower factor, then one rank-8 update of every remaining row.  This is the same
// factorisation, with the same pivots, as unblocked partial pivoting.  Rows are never
// moved: a row that has served as pivot is marked used, keeps its (L, U) entries and is
// skipped by later updates, so at the end the row chosen at step j holds row j of L \ U.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "fosb_internal.h"

namespace fosb {
namespace {

constexpr int kTsluRows = 256;  // rows per CTA (one per thread)
constexpr int kTsluCols = 64;   // panel width handled (jb <= 64)
constexpr int kTsluFanIn = kTsluRows / kTsluCols;

__device__ __forceinline__ float2 cinv(float2 v) {
  const float den = v.x * v.x + v.y * v.y;
  if (!(den > 0.f)) return make_float2(0.f, 0.f);
  const float r = 1.f / den;
  return make_float2(v.x * r, -v.y * r);
}
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

constexpr int kTsluLd = kTsluCols + 2;  // row pitch in complex values (16-byte aligned rows)
constexpr int kTsluBlk = 8;              // columns per block of the blocked factorisation
constexpr size_t kTsluSmem = size_t(kTsluRows) * kTsluLd * sizeof(float2);

__device__ __forceinline__ void cfms(float2& a, float2 l, float2 u) {  // a -= l u
  a.x -= l.x * u.x - l.y * u.y;
  a.y -= l.x * u.y + l.y * u.x;
}

// Leaf mode (in_idx == nullptr): CTA b factors panel rows [b * 256, min(m, (b + 1) * 256)).
// Tree mode: CTA b factors the nominees of groups [b * 4, min(groups_in, b * 4 + 4)), where
// group g lists in_cnt[g] panel rows at in_idx[g * 64 ...].
// Every CTA writes its pivot rows in order to out_idx[b * 64 ...] and their count to
// out_cnt[b].  A single-CTA launch is the root: it also writes the factored rows
// (L11 \ U11, row-major jb x 64) to top and the chosen panel rows to sel.
__global__ void __launch_bounds__(kTsluRows, 1)
    tslu_gepp_kernel(const float2* __restrict__ A, int64_t lda, int64_t m, int jb, const int* __restrict__ in_idx,
                     const int* __restrict__ in_cnt, int groups_in, int* __restrict__ out_idx, int* __restrict__ out_cnt,
                     float2* __restrict__ top, int* __restrict__ sel) {
  extern __shared__ float4 tslu_raw[];
  float2* sA = reinterpret_cast<float2*>(tslu_raw);  // [kTsluRows][kTsluLd]
  __shared__ int s_rows[kTsluRows];
  __shared__ unsigned long long s_wk[kTsluRows / 32];
  __shared__ int s_piv[kTsluBlk];
  __shared__ int s_nr;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const bool root = gridDim.x == 1;
  // rows of this CTA (panel-row indices)
  if (t == 0) {
    int nr = 0;
    if (in_idx == nullptr) {
      const int64_t lo = int64_t(blockIdx.x) * kTsluRows;
      nr = m - lo < kTsluRows ? int(m - lo) : kTsluRows;
      for (int i = 0; i < nr; ++i) s_rows[i] = int(lo + i);
    } else {
      for (int g = blockIdx.x * kTsluFanIn; g < min(groups_in, int(blockIdx.x) * kTsluFanIn + kTsluFanIn); ++g)
        for (int i = 0; i < in_cnt[g]; ++i) s_rows[nr++] = in_idx[g * kTsluCols + i];
    }
    s_nr = nr;
  }
  __syncthreads();
  const int nr = s_nr;
  const int steps = min(nr, jb);
  // rows into shared memory, a warp per row (256 contiguous bytes per load instruction),
  // eight rows' loads in flight before any store; zero past jb and for missing rows
  constexpr int kWarps = kTsluRows / 32, kBatch = 8;
  for (int r0 = warp; r0 < kTsluRows; r0 += kWarps * kBatch) {
    float2 v[kBatch][2];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const int r = r0 + b * kWarps;
      const float2* src = A + int64_t(r < nr ? s_rows[r] : 0) * lda;
      v[b][0] = (r < nr && lane < jb) ? __ldg(src + lane) : make_float2(0.f, 0.f);
      v[b][1] = (r < nr && lane + 32 < jb) ? __ldg(src + lane + 32) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      float2* dst = sA + (r0 + b * kWarps) * kTsluLd;
      dst[lane] = v[b][0];
      dst[lane + 32] = v[b][1];
      if (lane < kTsluLd - kTsluCols) dst[kTsluCols + lane] = make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  bool used = t >= nr;
  int order = -1;
  float2* my = sA + t * kTsluLd;
  for (int cb = 0; cb < steps; cb += kTsluBlk) {
    const int ce = min(cb + kTsluBlk, steps);  // pivot steps of this block
    const int cbe = min(cb + kTsluBlk, jb);    // columns of this block
    // the eight steps of the block, each compiled for its position JJ inside the block
    auto step = [&](auto jj_tag) {
      constexpr int JJ = decltype(jj_tag)::value;
      const int j = cb + JJ;
      if (j >= ce) return;  // the same for every thread
      // pivot: the largest |Re| + |Im| in column j among unused rows, ties to the lowest row
      unsigned key = 0;
      if (!used) {
        const float2 v = my[j];
        key = __float_as_uint(fabsf(v.x) + fabsf(v.y));
      }
      const unsigned mk = __reduce_max_sync(0xffffffffu, key);
      const unsigned bal = __ballot_sync(0xffffffffu, !used && key == mk);
      if (lane == 0)
        s_wk[warp] = bal ? (static_cast<unsigned long long>(mk) << 32) |
                               (0xFFFFFFFFu - unsigned(warp * 32 + __ffs(bal) - 1))
                         : 0ull;
      __syncthreads();
      unsigned long long best = s_wk[0];
#pragma unroll
      for (int w = 1; w < kTsluRows / 32; ++w) best = s_wk[w] > best ? s_wk[w] : best;
      const int p = int(0xFFFFFFFFu - unsigned(best & 0xFFFFFFFFull));  // an unused row exists: j < nr
      if (t == p) {
        used = true;
        order = j;
      }
      if (t == 0) s_piv[JJ] = p;
      if (!used) {  // eliminate column j inside the block (all loads before the stores)
        constexpr int W = kTsluBlk - JJ;
        const float2* pr = sA + p * kTsluLd;
        float2 pu[W], mv[W];
#pragma unroll
        for (int q = 0; q < W; ++q) {
          if (j + q < cbe) {
            pu[q] = pr[j + q];
            mv[q] = my[j + q];
          }
        }
        const float2 l = cmulf(mv[0], cinv(pu[0]));
        my[j] = l;
#pragma unroll
        for (int q = 1; q < W; ++q) {
          if (j + q < cbe) {
            cfms(mv[q], l, pu[q]);
            my[j + q] = mv[q];
          }
        }
      }
      __syncthreads();  // column j + 1 is up to date; s_wk may be rewritten
    };
    step(std::integral_constant<int, 0>{});
    step(std::integral_constant<int, 1>{});
    step(std::integral_constant<int, 2>{});
    step(std::integral_constant<int, 3>{});
    step(std::integral_constant<int, 4>{});
    step(std::integral_constant<int, 5>{});
    step(std::integral_constant<int, 6>{});
    step(std::integral_constant<int, 7>{});
    if (cbe >= jb) continue;
    const int npiv = ce - cb;
    // trailing columns of the block's pivot rows: U12 = L11^{-1} A12 (L11 unit lower, the
    // multipliers the pivot rows received inside the block), one thread per column
    for (int k = cbe + t; k < jb; k += blockDim.x) {
      for (int i = 0; i < npiv; ++i) {
        float2* ui = sA + s_piv[i] * kTsluLd;
        float2 u = ui[k];
        for (int q = 0; q < i; ++q) cfms(u, ui[cb + q], sA[s_piv[q] * kTsluLd + k]);
        ui[k] = u;
      }
    }
    __syncthreads();
    // rank-npiv update of the rows not chosen yet, two columns per 16-byte access
    if (!used) {
      float2 l[kTsluBlk];
      const float2* pv[kTsluBlk];
#pragma unroll
      for (int q = 0; q < kTsluBlk; ++q) {
        l[q] = q < npiv ? my[cb + q] : make_float2(0.f, 0.f);
        pv[q] = sA + s_piv[q < npiv ? q : 0] * kTsluLd;
      }
      for (int k = cbe; k < jb; k += 2) {
        float4 a = *reinterpret_cast<const float4*>(my + k);
        float4 u[kTsluBlk];
#pragma unroll
        for (int q = 0; q < kTsluBlk; ++q)
          u[q] = q < npiv ? *reinterpret_cast<const float4*>(pv[q] + k) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < kTsluBlk; ++q) {
          a.x -= l[q].x * u[q].x - l[q].y * u[q].y;
          a.y -= l[q].x * u[q].y + l[q].y * u[q].x;
          a.z -= l[q].x * u[q].z - l[q].y * u[q].w;
          a.w -= l[q].x * u[q].w + l[q].y * u[q].z;
        }
        *reinterpret_cast<float4*>(my + k) = a;
      }
    }
    __syncthreads();
  }
  if (order >= 0) {
    out_idx[blockIdx.x * kTsluCols + order] = s_rows[t];
    if (root) {
      sel[order] = s_rows[t];
      for (int c = 0; c < kTsluCols; ++c) top[order * kTsluCols + c] = my[c];
    }
  }
  if (t == 0) out_cnt[blockIdx.x] = steps;
}

// One CTA: chosen order -> interchanges.  Position i receives sel[i]; the row that was at
// position i goes where sel[i] was.  ipiv[i] = row_base + that position.  Only rows from
// the top jb positions and chosen rows from below ever move, and every position >= jb that
// is touched is the original position of a chosen row; so each involved row gets a slot
// (top row p: slot p; chosen row sel[i] >= jb: slot jb + i) and thread 0 replays the
// interchanges in O(jb).  Then the top jb rows become L11 \ U11 and the displaced original
// top rows land in their new positions.  A zero diagonal of U11 sets FOSB_ERR_SINGULAR.
__global__ void __launch_bounds__(256) tslu_apply_kernel(float2* __restrict__ A, int64_t lda, int jb,
                                                         const int* __restrict__ sel, const float2* __restrict__ top,
                                                         int32_t* __restrict__ ipiv, int64_t row_base,
                                                         int* __restrict__ status) {
  __shared__ int s_sel[kTsluCols];
  __shared__ int s_pos_of[2 * kTsluCols], s_qi_of[2 * kTsluCols];  // per slot: position, index of that position in sel
  __shared__ int s_at[kTsluCols], s_atq[kTsluCols];                // slot at top position p / at position sel[i]
  __shared__ float2 s_orig[kTsluCols][kTsluCols + 1];              // original rows at positions < jb
  const int t = threadIdx.x;
  if (t < jb) {
    const int r = sel[t];
    s_sel[t] = r;
    s_at[t] = t;
    s_pos_of[t] = t;
    s_qi_of[t] = -1;
    s_pos_of[jb + t] = r;
    s_qi_of[jb + t] = t;
    s_atq[t] = jb + t;
  }
  for (int e = t; e < jb * kTsluCols; e += blockDim.x) {
    const int r = e / kTsluCols, c = e % kTsluCols;
    s_orig[r][c] = c < jb ? A[int64_t(r) * lda + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  if (t == 0) {
    for (int i = 0; i < jb; ++i) {
      const int r = s_sel[i];
      const int sr = r < jb ? r : jb + i;
      const int q = s_pos_of[sr];
      ipiv[i] = int32_t(row_base + q);
      if (q != i) {
        const int si = s_at[i];
        if (q < jb) {
          s_at[q] = si;
          s_pos_of[si] = q;
        } else {
          const int k = s_qi_of[sr];
          s_atq[k] = si;
          s_qi_of[si] = k;
          s_pos_of[si] = q;
        }
        s_at[i] = sr;
        s_pos_of[sr] = i;
        s_qi_of[sr] = -1;
      }
    }
  }
  __syncthreads();
  // positions sel[i] >= jb now hold original top rows (slot < jb)
  for (int e = t; e < jb * jb; e += blockDim.x) {
    const int i = e / jb, c = e % jb;
    const int pos = s_sel[i], slot = s_atq[i];
    if (pos >= jb && slot >= 0 && slot < jb) A[int64_t(pos) * lda + c] = s_orig[slot][c];
  }
  for (int e = t; e < jb * jb; e += blockDim.x) {
    const int r = e / jb, c = e % jb;
    A[int64_t(r) * lda + c] = top[r * kTsluCols + c];
  }
  if (t < jb) {
    const float2 d = top[t * kTsluCols + t];
    if (!(d.x != 0.f || d.y != 0.f)) atomicCAS(status, 0, FOSB_ERR_SINGULAR);
  }
}

// L21 = A21 U11^{-1} for rows [jb, m): one warp per row, lanes own columns (lane, lane + 32).
__global__ void __launch_bounds__(256) tslu_lsolve_kernel(float2* __restrict__ A, int64_t lda, int64_t m, int jb) {
  __shared__ float2 s_U[kTsluCols][kTsluCols];
  __shared__ float2 s_dinv[kTsluCols];
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    const int r = e / jb, c = e % jb;
    s_U[r][c] = A[int64_t(r) * lda + c];
  }
  __syncthreads();
  if (threadIdx.x < jb) s_dinv[threadIdx.x] = cinv(s_U[threadIdx.x][threadIdx.x]);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  // grid-stride over rows, so U11 is staged once per CTA
  for (int64_t row = jb + int64_t(blockIdx.x) * 8 + (threadIdx.x >> 5); row < m; row += int64_t(gridDim.x) * 8) {
    float2* x = A + row * lda;
    float2 x0 = lane < jb ? x[lane] : make_float2(0.f, 0.f);
    float2 x1 = lane + 32 < jb ? x[lane + 32] : make_float2(0.f, 0.f);
    for (int k = 0; k < jb; ++k) {
      // l_k = (a_k - sum_{i<k} l_i u_ik) / u_kk: the owner lane finishes it, then all
      // later columns subtract l_k u_kc
      float2 v = k < 32 ? x0 : x1;
      v.x = __shfl_sync(0xffffffffu, v.x, k & 31);
      v.y = __shfl_sync(0xffffffffu, v.y, k & 31);
      const float2 l = cmulf(v, s_dinv[k]);
      if (k < 32 && lane == k) x0 = l;
      if (k >= 32 && lane == k - 32) x1 = l;
      if (lane > k && lane < jb) {
        const float2 u = s_U[k][lane];
        x0.x -= l.x * u.x - l.y * u.y;
        x0.y -= l.x * u.y + l.y * u.x;
      }
      if (lane + 32 > k && lane + 32 < jb) {
        const float2 u = s_U[k][lane + 32];
        x1.x -= l.x * u.x - l.y * u.y;
        x1.y -= l.x * u.y + l.y * u.x;
      }
    }
    if (lane < jb) x[lane] = x0;
    if (lane + 32 < jb) x[lane + 32] = x1;
  }
}

inline unsigned cdivu(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }

}  // namespace

size_t tslu_scratch_bytes(int64_t n) {
  const int64_t leaves = (n + kTsluRows - 1) / kTsluRows;
  return size_t(2 * leaves * kTsluCols + 2 * leaves + kTsluCols) * sizeof(int) +
         size_t(kTsluCols * kTsluCols) * sizeof(float2) + 256;
}

cudaError_t tslu_panel(void* Ap, int64_t m, int jb, int64_t lda, int32_t* ipiv, int64_t row_base, void* scratch,
                       int64_t n_max, int* d_status, cudaStream_t s) {
  if (jb <= 0 || jb > kTsluCols || m < jb) return cudaErrorInvalidValue;
  ProfScope prof("lu_panel", s, 4.0 * double(m) * jb * jb);
  float2* A = static_cast<float2*>(Ap);
  const int64_t leaves_max = (n_max + kTsluRows - 1) / kTsluRows;
  char* base = static_cast<char*>(scratch);
  float2* top = reinterpret_cast<float2*>(base);
  int* idx0 = reinterpret_cast<int*>(top + kTsluCols * kTsluCols);
  int* idx1 = idx0 + leaves_max * kTsluCols;
  int* cnt0 = idx1 + leaves_max * kTsluCols;
  int* cnt1 = cnt0 + leaves_max;
  int* sel = cnt1 + leaves_max;
  int groups = int((m + kTsluRows - 1) / kTsluRows);
  if (groups > leaves_max) return cudaErrorInvalidValue;
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(tslu_gepp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               int(kTsluSmem));
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  tslu_gepp_kernel<<<groups, kTsluRows, kTsluSmem, s>>>(A, lda, m, jb, nullptr, nullptr, 0, idx0, cnt0, top, sel);
  uint64_t nl = 1;
  int *in_i = idx0, *in_c = cnt0, *out_i = idx1, *out_c = cnt1;
  while (groups > 1) {
    const int next = (groups + kTsluFanIn - 1) / kTsluFanIn;
    tslu_gepp_kernel<<<next, kTsluRows, kTsluSmem, s>>>(A, lda, m, jb, in_i, in_c, groups, out_i, out_c, top, sel);
    ++nl;
    groups = next;
    int* ti = in_i; in_i = out_i; out_i = ti;
    int* tc = in_c; in_c = out_c; out_c = tc;
  }
  tslu_apply_kernel<<<1, 256, 0, s>>>(A, lda, jb, sel, top, ipiv, row_base, d_status);
  ++nl;
  if (m > jb) {
    static int nsm[64] = {};
    if (!nsm[dev]) cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev);
    const unsigned g = std::min<unsigned>(cdivu(m - jb, 8), unsigned(6 * std::max(nsm[dev], 1)));
    tslu_lsolve_kernel<<<g, 256, 0, s>>>(A, lda, m, jb);
    ++nl;
  }
  return launched(nl);
}

}  // namespace fosb
