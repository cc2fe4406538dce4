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
// Within a CTA the candidate rows sit in shared memory and are factored by blocked partial
// pivoting in blocks of 8 columns: per step a warp argmax (one reduction), one
// barrier among the eight warps that own the rows, an 8-entry argmax across them, and the
// elimination of that column inside the block (in registers); per block the trailing
// columns of its pivot rows by forward substitution with the block's unit lower factor,
// then one rank-8 update of every remaining row by all sixteen warps.  This is the same
// factorisation as unblocked partial pivoting whose pivot magnitudes are compared on 15
// mantissa bits (a candidate within a relative 2^-15 of the largest may win the tie as the
// lower row, so |l| <= 1 + 2^-15).  Rows are never
// moved: a row that has served as pivot is marked used, keeps its (L, U) entries and is
// skipped by later updates, so at the end the row chosen at step j holds row j of L \ U.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "fosb_internal.h"

namespace fosb {
namespace {

constexpr int kTsluRows = 256;  // rows per CTA
constexpr int kTsluCols = 64;   // panel width handled (jb <= 64)
constexpr int kTsluFanIn = kTsluRows / kTsluCols;
constexpr int kTsluSub = 2;                            // threads per row in the block updates
constexpr int kTsluThreads = kTsluRows * kTsluSub;     // 512
constexpr int kTsluStepWarps = kTsluRows / 32;         // warps 0-7 run the pivot steps
constexpr int kTsluPairs = kTsluCols / 2;              // 16-byte column pairs of a row

__device__ __forceinline__ float2 cinv(float2 v) {
  const float den = v.x * v.x + v.y * v.y;
  if (!(den > 0.f)) return make_float2(0.f, 0.f);
  const float r = 1.f / den;
  return make_float2(v.x * r, -v.y * r);
}
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Row pitch in complex values: 544 bytes, so the eight threads of a 16-byte access phase in
// the block updates (four rows x two column pairs) fall in eight distinct bank groups.
constexpr int kTsluLd = 68;
constexpr int kTsluBlk = 8;  // columns per block of the blocked factorisation
constexpr size_t kTsluSmem = size_t(kTsluRows) * kTsluLd * sizeof(float2);

__device__ __forceinline__ void cfms(float2& a, float2 l, float2 u) {  // a -= l u
  a.x -= l.x * u.x - l.y * u.y;
  a.y -= l.x * u.y + l.y * u.x;
}
__device__ __forceinline__ void cfms2(float4& a, float2 l, float4 u) {  // both complex values of a pair
  a.x -= l.x * u.x - l.y * u.y;
  a.y -= l.x * u.y + l.y * u.x;
  a.z -= l.x * u.z - l.y * u.w;
  a.w -= l.x * u.w + l.y * u.z;
}
__device__ __forceinline__ void step_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kTsluRows) : "memory"); }

// Leaf mode (in_idx == nullptr): CTA b factors panel rows [b * 256, min(m, (b + 1) * 256)).
// Tree mode: CTA b factors the nominees of groups [b * 4, min(groups_in, b * 4 + 4)), where
// group g lists in_cnt[g] panel rows at in_idx[g * 64 ...].
// Every CTA writes its pivot rows in order to out_idx[b * 64 ...] and their count to
// out_cnt[b].  A single-CTA launch is the root: it also writes the factored rows
// (L11 \ U11, row-major jb x 64) to top and the chosen panel rows to sel.
//
// The pivot steps of an 8-column block run on warps 0-7 alone, thread t owning row t and
// keeping the row's eight block columns in registers; a step is one warp argmax, one
// 256-thread named barrier and an 8-entry argmax across the warps, each a single 32-bit
// max-reduction.  Each warp's candidate
// stages its block columns in shared memory before the barrier, so the rows read the pivot
// row from there and nothing is written back until the block ends.  The block's trailing
// work (U12 of its pivot rows, the rank-8 update of the other rows) runs on all 512 threads,
// two per row.
__global__ void __launch_bounds__(kTsluThreads, 1)
    tslu_gepp_kernel(const float2* __restrict__ A, int64_t lda, int64_t m, int jb, const int* __restrict__ in_idx,
                     const int* __restrict__ in_cnt, int groups_in, int* __restrict__ out_idx, int* __restrict__ out_cnt,
                     float2* __restrict__ top, int* __restrict__ sel) {
  extern __shared__ float4 tslu_raw[];
  float2* sA = reinterpret_cast<float2*>(tslu_raw);  // [kTsluRows][kTsluLd]
  __shared__ int s_rows[kTsluRows];
  __shared__ int s_used[kTsluRows];
  __shared__ int s_off[kTsluFanIn + 1];
  __shared__ int s_piv[kTsluBlk];
  __shared__ unsigned s_wk[2][kTsluStepWarps];
  __shared__ float2 s_inv[2][kTsluStepWarps];
  __shared__ float4 s_stage[2][kTsluStepWarps][kTsluBlk / 2];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const bool root = gridDim.x == 1;
  // rows of this CTA (panel-row indices)
  int nr;
  if (in_idx == nullptr) {
    const int64_t lo = int64_t(blockIdx.x) * kTsluRows;
    nr = m - lo < kTsluRows ? int(m - lo) : kTsluRows;
    if (t < nr) s_rows[t] = int(lo + t);
  } else {
    const int g0 = blockIdx.x * kTsluFanIn, ng = min(groups_in - g0, kTsluFanIn);
    if (t == 0) {
      int acc = 0;
      for (int g = 0; g < kTsluFanIn; ++g) {
        s_off[g] = acc;
        acc += g < ng ? in_cnt[g0 + g] : 0;
      }
      s_off[kTsluFanIn] = acc;
    }
    __syncthreads();
    nr = s_off[kTsluFanIn];
    if (t < kTsluRows) {
      const int g = t / kTsluCols, i = t % kTsluCols;
      if (g < ng && i < s_off[g + 1] - s_off[g]) s_rows[s_off[g] + i] = in_idx[(g0 + g) * kTsluCols + i];
    }
  }
  if (t < kTsluRows) s_used[t] = t >= nr;
  __syncthreads();
  const int steps = min(nr, jb);
  // rows into shared memory, a warp per row (256 contiguous bytes per load instruction),
  // sixteen rows' loads in flight per warp; zero past jb and for missing rows
  {
    constexpr int kWarps = kTsluThreads / 32, kBatch = kTsluRows / kWarps;
    float2 v[kBatch][2];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const int rr = warp + b * kWarps;
      const float2* src = A + int64_t(rr < nr ? s_rows[rr] : 0) * lda;
      v[b][0] = (rr < nr && lane < jb) ? __ldg(src + lane) : make_float2(0.f, 0.f);
      v[b][1] = (rr < nr && lane + 32 < jb) ? __ldg(src + lane + 32) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      float2* dst = sA + (warp + b * kWarps) * kTsluLd;
      dst[lane] = v[b][0];
      dst[lane + 32] = v[b][1];
    }
  }
  __syncthreads();
  bool used = t >= nr;  // (row threads: warps 0-7)
  int order = -1;
  const int npairs = (jb + 1) >> 1;
  for (int cb = 0; cb < steps; cb += kTsluBlk) {
    const int ce = min(cb + kTsluBlk, steps);  // pivot steps of this block
    const int cbe = min(cb + kTsluBlk, jb);    // columns of this block
    if (warp < kTsluStepWarps) {
      float4* myb = reinterpret_cast<float4*>(sA + t * kTsluLd + cb);
      float2 bv[kTsluBlk];
#pragma unroll
      for (int i = 0; i < kTsluBlk / 2; ++i) {
        const float4 w = myb[i];
        bv[2 * i] = make_float2(w.x, w.y);
        bv[2 * i + 1] = make_float2(w.z, w.w);
      }
      // the eight steps of the block, each compiled for its position JJ inside the block
      auto step = [&](auto jj_tag) {
        constexpr int JJ = decltype(jj_tag)::value, B = JJ & 1;
        const int j = cb + JJ;
        if (j >= ce) return;  // the same for every thread
        // pivot: the largest |Re| + |Im| in column j among unused rows, compared on the top
        // 24 bits of its float pattern (15 mantissa bits), ties to the lowest row.  One
        // 32-bit key per row: bit 31 marks a candidate, the low 8 bits hold 255 - row.
        const float2 vj = bv[JJ];
        const unsigned key =
            used ? 0u
                 : (0x80000000u | (__float_as_uint(fabsf(vj.x) + fabsf(vj.y)) & 0x7FFFFF00u) | unsigned(255 - t));
        const float2 myinv = cinv(vj);  // the inverse as pivot, ready before the argmax ends
        const unsigned mk = __reduce_max_sync(0xffffffffu, key);
        if (lane == 0) s_wk[B][warp] = mk;
        if (key == mk && mk != 0u) {  // this warp's candidate (the row bits make it unique)
#pragma unroll
          for (int i = 0; i < kTsluBlk / 2; ++i)
            s_stage[B][warp][i] = make_float4(bv[2 * i].x, bv[2 * i].y, bv[2 * i + 1].x, bv[2 * i + 1].y);
          s_inv[B][warp] = myinv;
        }
        step_bar();
        const unsigned g = __reduce_max_sync(0xffffffffu, lane < kTsluStepWarps ? s_wk[B][lane] : 0u);
        const int p = 255 - int(g & 255u);  // an unused row exists: j < nr
        if (t == 0) s_piv[JJ] = p;
        if (t == p) {
          used = true;
          order = j;
          s_used[t] = 1;
        }
        if (!used) {  // eliminate column j from my block columns
          const float4* ps = s_stage[B][p >> 5];
          const float2 l = cmulf(vj, s_inv[B][p >> 5]);
          bv[JJ] = l;
#pragma unroll
          for (int qq = JJ + 1; qq < kTsluBlk; ++qq) {
            if (cb + qq < cbe) {
              const float4 uw = ps[qq >> 1];
              cfms(bv[qq], l, (qq & 1) ? make_float2(uw.z, uw.w) : make_float2(uw.x, uw.y));
            }
          }
        }
      };
      step(std::integral_constant<int, 0>{});
      step(std::integral_constant<int, 1>{});
      step(std::integral_constant<int, 2>{});
      step(std::integral_constant<int, 3>{});
      step(std::integral_constant<int, 4>{});
      step(std::integral_constant<int, 5>{});
      step(std::integral_constant<int, 6>{});
      step(std::integral_constant<int, 7>{});
#pragma unroll
      for (int i = 0; i < kTsluBlk / 2; ++i)
        myb[i] = make_float4(bv[2 * i].x, bv[2 * i].y, bv[2 * i + 1].x, bv[2 * i + 1].y);
    }
    if (cbe >= jb) continue;  // the same for every thread
    const int npiv = ce - cb;
    __syncthreads();  // block columns, s_piv and s_used are in shared memory
    // trailing columns of the block's pivot rows: U12 = L11^{-1} A12 (L11 unit lower, the
    // multipliers the pivot rows received inside the block), one thread per column
    if (t < jb - cbe) {
      const int k = cbe + t;
      float2 u[kTsluBlk];
#pragma unroll
      for (int i = 0; i < kTsluBlk; ++i) {
        if (i < npiv) {
          float2* ui = sA + s_piv[i] * kTsluLd;
          float2 a = ui[k];
#pragma unroll
          for (int qq = 0; qq < i; ++qq) cfms(a, ui[cb + qq], u[qq]);
          u[i] = a;
          ui[k] = a;
        }
      }
    }
    __syncthreads();
    // rank-npiv update of the rows not chosen yet over their column pairs right of the
    // block, thread (r, h) taking the pairs P with P % 2 == h
    {
      const int r = t >> 1, h = t & 1;
      if (!s_used[r]) {
        const float2* my = sA + r * kTsluLd;
        float2 l[kTsluBlk];
        const float4* pv[kTsluBlk];
#pragma unroll
        for (int i = 0; i < kTsluBlk; i += 2) {
          const float4 v = reinterpret_cast<const float4*>(my)[(cb + i) >> 1];
          l[i] = make_float2(v.x, v.y);
          l[i + 1] = make_float2(v.z, v.w);
        }
#pragma unroll
        for (int i = 0; i < kTsluBlk; ++i) pv[i] = reinterpret_cast<const float4*>(sA + s_piv[i < npiv ? i : 0] * kTsluLd);
        float4* myw = reinterpret_cast<float4*>(const_cast<float2*>(my));
        int P = (cbe >> 1) + h;
        for (; P + kTsluSub < npairs; P += 2 * kTsluSub) {  // two pairs per pass: more loads in flight
          float4 a0 = myw[P], a1 = myw[P + kTsluSub];
          float4 u0[kTsluBlk], u1[kTsluBlk];
#pragma unroll
          for (int i = 0; i < kTsluBlk; ++i) {
            if (i < npiv) {
              u0[i] = pv[i][P];
              u1[i] = pv[i][P + kTsluSub];
            }
          }
#pragma unroll
          for (int i = 0; i < kTsluBlk; ++i) {
            if (i < npiv) {
              cfms2(a0, l[i], u0[i]);
              cfms2(a1, l[i], u1[i]);
            }
          }
          myw[P] = a0;
          myw[P + kTsluSub] = a1;
        }
        if (P < npairs) {
          float4 a = myw[P];
#pragma unroll
          for (int i = 0; i < kTsluBlk; ++i)
            if (i < npiv) cfms2(a, l[i], pv[i][P]);
          myw[P] = a;
        }
      }
    }
    __syncthreads();
  }
  if (order >= 0) {  // a row thread whose row was chosen at step `order`
    out_idx[blockIdx.x * kTsluCols + order] = s_rows[t];
    if (root) {
      sel[order] = s_rows[t];
      // every value of the row was last written by this thread or before a CTA barrier
      const float4* src = reinterpret_cast<const float4*>(sA + t * kTsluLd);
      float4* dst = reinterpret_cast<float4*>(top + order * kTsluCols);
#pragma unroll 8
      for (int P = 0; P < kTsluPairs; ++P) dst[P] = src[P];
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
                                                         int* __restrict__ status, int2* __restrict__ moves) {
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
  // (fixed trip counts: all sixteen loads of a thread are in flight together)
#pragma unroll
  for (int k = 0; k < kTsluCols * kTsluCols / 256; ++k) {
    const int e = t + 256 * k, r = e / kTsluCols, c = e % kTsluCols;
    s_orig[r][c] = (r < jb && c < jb) ? A[int64_t(r) * lda + c] : make_float2(0.f, 0.f);
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
  // the same permutation as (source, destination) positions for the other columns: position
  // i takes the row from sel[i]; a displaced original top row goes to its slot's position
  if (t < jb) {
    const int pos = s_sel[t], slot = s_atq[t];
    moves[t] = pos != t ? make_int2(pos, t) : make_int2(-1, -1);
    moves[jb + t] = (pos >= jb && slot >= 0 && slot < jb) ? make_int2(slot, pos) : make_int2(-1, -1);
  }
  // positions sel[i] >= jb now hold original top rows (slot < jb)
#pragma unroll
  for (int k = 0; k < kTsluCols * kTsluCols / 256; ++k) {
    const int e = t + 256 * k, i = e / kTsluCols, c = e % kTsluCols;
    if (i < jb && c < jb) {
      const int pos = s_sel[i], slot = s_atq[i];
      if (pos >= jb && slot >= 0 && slot < jb) A[int64_t(pos) * lda + c] = s_orig[slot][c];
    }
  }
#pragma unroll
  for (int k = 0; k < kTsluCols * kTsluCols / 256; ++k) {
    const int e = t + 256 * k, r = e / kTsluCols, c = e % kTsluCols;
    if (r < jb && c < jb) A[int64_t(r) * lda + c] = top[r * kTsluCols + c];
  }
  if (t < jb) {
    const float2 d = top[t * kTsluCols + t];
    if (!(d.x != 0.f || d.y != 0.f)) atomicCAS(status, 0, FOSB_ERR_SINGULAR);
  }
}

// Triangular substitution on per-thread vectors of 64 complex values held transposed in
// shared memory (element k of this thread's vector at xs[k * ldx]): for k = 0 .. 63,
// x_k *= dinv_k (kScale) and x_c -= x_k M[k][c] for c > k, the right-looking order of
// forward substitution.  The vector is taken 8 elements at a time: the 8 live in registers
// while the chunk is solved, then one rank-8 update reaches every later element (the same
// operations in the same order as one element at a time).  M is in shared memory and read
// by every thread alike (broadcast).
template <bool kScale>
__device__ __forceinline__ void tri_chunked(float2* xs, int ldx, const float2 (*M)[kTsluCols], const float2* dinv) {
#pragma unroll 1
  for (int k0 = 0; k0 < kTsluCols; k0 += 8) {
    float2 x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = xs[(k0 + i) * ldx];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (kScale) x[i] = cmulf(x[i], dinv[k0 + i]);
#pragma unroll
      for (int q = i + 1; q < 8; ++q) cfms(x[q], x[i], M[k0 + i][k0 + q]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) xs[(k0 + i) * ldx] = x[i];
#pragma unroll 4
    for (int c = k0 + 8; c < kTsluCols; ++c) {
      float2 y = xs[c * ldx];
#pragma unroll
      for (int i = 0; i < 8; ++i) cfms(y, x[i], M[k0 + i][c]);
      xs[c * ldx] = y;
    }
  }
}

constexpr int kLsRows = 64;  // rows (threads) per CTA of the L21 solve
constexpr int kLsLd = kLsRows + 1;
constexpr size_t kLsSmem = size_t(kTsluCols) * kTsluCols * sizeof(float2) + kTsluCols * sizeof(float2) +
                           size_t(kTsluCols) * kLsLd * sizeof(float2);

// L21 = A21 U11^{-1} for rows [jb, m), U11 the upper triangle (with the diagonal) of the top
// jb rows: a thread per row.  The CTA's 64 rows are loaded with coalesced row reads, 8 rows
// in flight per warp, into a transposed shared tile; U11 is staged identity-padded to
// 64 x 64, so a ragged panel (jb < 64) needs no other case.
__global__ void __launch_bounds__(kLsRows) tslu_lsolve_kernel(float2* __restrict__ A, int64_t lda, int64_t m, int jb) {
  extern __shared__ float4 ls_raw[];
  auto sM = reinterpret_cast<float2 (*)[kTsluCols]>(ls_raw);
  float2* s_dinv = reinterpret_cast<float2*>(ls_raw) + kTsluCols * kTsluCols;
  float2* xs = s_dinv + kTsluCols;  // [64][kLsLd]
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  constexpr int kWarps = kLsRows / 32, kBatch = 8;
  for (int e = t; e < kTsluCols * kTsluCols; e += kLsRows) {
    const int r = e / kTsluCols, c = e % kTsluCols;
    sM[r][c] = (r < jb && c < jb && c >= r) ? A[int64_t(r) * lda + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  s_dinv[t] = t < jb ? cinv(sM[t][t]) : make_float2(1.f, 0.f);
  const int64_t r0 = jb + int64_t(blockIdx.x) * kLsRows;
  for (int b0 = warp; b0 < kLsRows; b0 += kWarps * kBatch) {
    float2 v[kBatch][2];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const int rr = b0 + b * kWarps;
      const int64_t row = r0 + rr;
      const bool ok = rr < kLsRows && row < m;
      v[b][0] = (ok && lane < jb) ? A[row * lda + lane] : make_float2(0.f, 0.f);
      v[b][1] = (ok && lane + 32 < jb) ? A[row * lda + lane + 32] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const int rr = b0 + b * kWarps;
      if (rr < kLsRows) {
        xs[lane * kLsLd + rr] = v[b][0];
        xs[(lane + 32) * kLsLd + rr] = v[b][1];
      }
    }
  }
  __syncthreads();
  tri_chunked<true>(xs + t, kLsLd, sM, s_dinv);
  __syncthreads();
  for (int rr = warp; rr < kLsRows; rr += kWarps) {
    const int64_t row = r0 + rr;
    if (row >= m) break;
    if (lane < jb) A[row * lda + lane] = xs[lane * kLsLd + rr];
    if (lane + 32 < jb) A[row * lda + lane + 32] = xs[(lane + 32) * kLsLd + rr];
  }
}

constexpr int kLcCols = 64;  // columns (threads) per CTA of the unit-lower column solve
constexpr int kLcLd = kLcCols + 1;
constexpr size_t kLcSmem = size_t(kTsluCols) * kTsluCols * sizeof(float2) + size_t(kTsluCols) * kLcLd * sizeof(float2);

// X (jb x ncols, leading dimension ldx) := L^{-1} X with L the unit lower jb x jb block at
// D (leading dimension ldd): a thread per column, M[k][c] = L[c][k] staged zero-padded.
__global__ void __launch_bounds__(kLcCols) tri_lower_unit_cols_kernel(const float2* __restrict__ D, int64_t ldd, int jb,
                                                                      float2* __restrict__ X, int64_t ldx,
                                                                      int64_t ncols) {
  extern __shared__ float4 lc_raw[];
  auto sM = reinterpret_cast<float2 (*)[kTsluCols]>(lc_raw);
  float2* xs = reinterpret_cast<float2*>(lc_raw) + kTsluCols * kTsluCols;  // [64][kLcLd]
  const int t = threadIdx.x;
  for (int e = t; e < kTsluCols * kTsluCols; e += kLcCols) {
    const int k = e / kTsluCols, c = e % kTsluCols;
    sM[k][c] = (k < jb && c < jb && c > k) ? D[int64_t(c) * ldd + k] : make_float2(0.f, 0.f);
  }
  const int64_t col = int64_t(blockIdx.x) * kLcCols + t;
  const bool ok = col < ncols;
  constexpr int kBatch = 16;
  for (int k0 = 0; k0 < kTsluCols; k0 += kBatch) {
    float2 v[kBatch];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) v[b] = (ok && k0 + b < jb) ? X[int64_t(k0 + b) * ldx + col] : make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < kBatch; ++b) xs[(k0 + b) * kLcLd + t] = v[b];
  }
  __syncthreads();
  tri_chunked<false>(xs + t, kLcLd, sM, nullptr);
  if (!ok) return;
  for (int k = 0; k < jb; ++k) X[int64_t(k) * ldx + col] = xs[k * kLcLd + t];
}

// The panel's row permutation on the columns outside it (left: earlier L columns; right:
// the trailing matrix).  Row j0 + dst takes the old values of row j0 + src for every move
// (at most 2 jb rows, each a source once and a destination once).  A CTA covers 32 columns:
// lanes run along a row (256-byte accesses), the 8 warps split the moves, and every read of
// the CTA's columns happens before any write.
__global__ void __launch_bounds__(256) tslu_swap_kernel(float2* __restrict__ A, int64_t n, int64_t lda, int64_t j0,
                                                        int jb, const int2* __restrict__ moves) {
  __shared__ int2 s_mv[2 * kTsluCols];
  const int t = threadIdx.x;
  if (t < 2 * jb) s_mv[t] = moves[t];
  __syncthreads();
  const int tx = t & 31, ty = t >> 5;
  const int64_t c = int64_t(blockIdx.x) * 32 + tx;
  const bool col_ok = c < n && (c < j0 || c >= j0 + jb);
  constexpr int kPer = 2 * kTsluCols / 8;
  float2 v[kPer];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int mi = ty + 8 * k;
    if (col_ok && mi < 2 * jb && s_mv[mi].x >= 0) v[k] = A[(j0 + s_mv[mi].x) * lda + c];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int mi = ty + 8 * k;
    if (col_ok && mi < 2 * jb && s_mv[mi].x >= 0) A[(j0 + s_mv[mi].y) * lda + c] = v[k];
  }
}

inline unsigned cdivu(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }

}  // namespace

size_t tslu_scratch_bytes(int64_t n) {
  const int64_t leaves = (n + kTsluRows - 1) / kTsluRows;
  return size_t(2 * leaves * kTsluCols + 2 * leaves + kTsluCols) * sizeof(int) +
         size_t(kTsluCols * kTsluCols) * sizeof(float2) + size_t(2 * kTsluCols) * sizeof(int2) + 256;
}

cudaError_t tslu_panel(void* Ap, int64_t m, int jb, int64_t lda, int32_t* ipiv, int64_t row_base, void* scratch,
                       int64_t n_max, int* d_status, cudaStream_t s) {
  if (jb <= 0 || jb > kTsluCols || m < jb) return cudaErrorInvalidValue;
  ProfScope prof("lu_panel", s, 4.0 * double(m) * jb * jb);
  float2* A = static_cast<float2*>(Ap);
  const int64_t leaves_max = (n_max + kTsluRows - 1) / kTsluRows;
  char* base = static_cast<char*>(scratch);
  float2* top = reinterpret_cast<float2*>(base);
  int2* moves = reinterpret_cast<int2*>(top + kTsluCols * kTsluCols);
  int* idx0 = reinterpret_cast<int*>(moves + 2 * kTsluCols);
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
  tslu_gepp_kernel<<<groups, kTsluThreads, kTsluSmem, s>>>(A, lda, m, jb, nullptr, nullptr, 0, idx0, cnt0, top, sel);
  uint64_t nl = 1;
  int *in_i = idx0, *in_c = cnt0, *out_i = idx1, *out_c = cnt1;
  while (groups > 1) {
    const int next = (groups + kTsluFanIn - 1) / kTsluFanIn;
    tslu_gepp_kernel<<<next, kTsluThreads, kTsluSmem, s>>>(A, lda, m, jb, in_i, in_c, groups, out_i, out_c, top, sel);
    ++nl;
    groups = next;
    int* ti = in_i; in_i = out_i; out_i = ti;
    int* tc = in_c; in_c = out_c; out_c = tc;
  }
  tslu_apply_kernel<<<1, 256, 0, s>>>(A, lda, jb, sel, top, ipiv, row_base, d_status, moves);
  ++nl;
  if (m > jb) {
    static bool ls_attr[64] = {};
    if (!ls_attr[dev]) {
      const cudaError_t e = cudaFuncSetAttribute(tslu_lsolve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 int(kLsSmem));
      if (e != cudaSuccess) return e;
      ls_attr[dev] = true;
    }
    tslu_lsolve_kernel<<<cdivu(m - jb, kLsRows), kLsRows, kLsSmem, s>>>(A, lda, m, jb);
    ++nl;
  }
  return launched(nl);
}

cudaError_t tri_lower_unit_cols(const void* D, int64_t ldd, int jb, void* X, int64_t ldx, int64_t ncols,
                                cudaStream_t s) {
  if (jb <= 0 || jb > kTsluCols) return cudaErrorInvalidValue;
  if (ncols <= 0) return cudaSuccess;
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr[dev]) {
    const cudaError_t e =
        cudaFuncSetAttribute(tri_lower_unit_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kLcSmem));
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  tri_lower_unit_cols_kernel<<<cdivu(ncols, kLcCols), kLcCols, kLcSmem, s>>>(static_cast<const float2*>(D), ldd, jb,
                                                                            static_cast<float2*>(X), ldx, ncols);
  return launched();
}

cudaError_t tslu_swap(void* A, int64_t n, int64_t lda, int64_t j0, int jb, const void* scratch, cudaStream_t s) {
  if (jb <= 0 || jb > kTsluCols) return cudaErrorInvalidValue;
  const int2* moves = reinterpret_cast<const int2*>(static_cast<const float2*>(scratch) + kTsluCols * kTsluCols);
  tslu_swap_kernel<<<cdivu(n, 32), 256, 0, s>>>(static_cast<float2*>(A), n, lda, j0, jb, moves);
  return launched();
}

}  // namespace fosb
