// FP64-class complex GEMM C <- beta C + alpha Z X on the bf16 tensor cores by exact digit
// splitting, for the refinement residuals of multi-right-hand-side solves (A6, A9).
//
// Every row i of Z is scaled by a power of two sigma_i > its largest |Re|, |Im| and written
// as seven signed base-256 digits:  Z_ik = sigma_i 2^-7 sum_{s=0..6} 2^{-8s} d_s[i,k] up to
// 2^-56 sigma_i (the balanced base-256 form of Z_ik 2^55 / sigma_i rounded to an integer),
// |d_s| <= 128, so each digit is exact in bf16; the same
// for every column j of X with tau_j and digits e_t.  Then
//   (Z X)_ij = sigma_i tau_j 2^-14 sum_{s,t} 2^{-8(s+t)} sum_k d_s[i,k] e_t[k,j],
// and a digit product is an integer of at most 2^14, so sums of the same order g = s+t over
// 64 values of k are exact in the FP32 accumulators of the tensor cores
// ((g+1) x 2 x 64 x 2^14 < 2^24 for g <= 6).  Orders g <= 6 (28 digit pairs) are kept:
// the dropped terms are below 2^-56 of sigma_i tau_j per product.  After every 64 values
// of k the seven order accumulators (Re, Im) are read out of TMEM: orders 0-3 are added
// exactly into a 64-bit integer sum per output, orders 4-6 (below 2^-32 of them) into an
// FP32 sum; the result is scaled by sigma_i tau_j 2^-14.
//
// Kernel roles (one CTA per SM, persistent over 128 x 32 output tiles): warp 0 lane 0 moves
// the pre-tiled digit tiles of a 16-wide k step (14 A tiles of 4 KB, 14 B tiles of 1 KB)
// into a 3-stage shared ring with bulk copies; warp 1 lane 0 issues 112 MMAs per step
// (tcgen05.mma kind::f16, bf16, M = 128, N = 32, K = 16; the minus of Im Z Im X via the
// negate-B bit; the MMAs that share an A tile and an instruction descriptor run back to
// back and keep it in the A collector, so an A tile is read from shared memory once or
// twice per step) into the 14 order
// accumulators; warps 2-9 read the accumulators after every
// 64 values of k and hold the sums (two warps per TMEM lane group, 16 columns each).  All
// waits are bounded.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "fosb_internal.h"

namespace fosb {
namespace {

constexpr int OZ_TM = 128, OZ_TN = 32, OZ_KS = 16, OZ_ND = 7;  // tile rows, tile columns, k step, digits
constexpr int OZ_KCH = 4;                                      // k steps per exact chunk (64 values)
constexpr int OZ_ATILE = OZ_TM * OZ_KS * 2;                    // 4096 B
constexpr int OZ_BTILE = OZ_TN * OZ_KS * 2;                    // 1024 B
constexpr int OZ_NT = OZ_ND * 2;                               // digit x part tiles per operand and step
constexpr int OZ_STAGE = OZ_NT * (OZ_ATILE + OZ_BTILE);        // 71680 B
constexpr int OZ_STAGES = 3;
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE + 1024;
constexpr int OZ_THREADS = 10 * 32;                            // producer, MMA, 8 flush warps
constexpr int OZ_FLUSH = 8 * 32;
constexpr int OZ_HN = OZ_TN / 2;                               // columns per flush thread
constexpr int OZ_TMEM_COLS = 512;                              // 7 orders x (Re, Im) x 32 columns = 448 used
constexpr long long kOzSpinLimit = 1ll << 24;
static_assert(OZ_SMEM <= 227 * 1024, "digit stages do not fit shared memory");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// canonical no-swizzle K-major offset of element (row, k), k < 16, 2-byte elements:
// 8 x 16-byte core matrices, 128 B apart along k, 256 B between 8-row groups
__host__ __device__ __forceinline__ int oz_off(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ uint64_t oz_desc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = 256;
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}
// kind::f16 instruction descriptor: D f32 (bits 4-5 = 1), A and B bf16 (bits 7-9, 10-12 = 1),
// K-major A and B, N >> 3 at bits 17-22, M >> 4 at bits 24-28, optional negate-B (bit 14)
__host__ __device__ constexpr uint32_t oz_idesc(bool neg_b) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (neg_b ? (1u << 14) : 0u) | (uint32_t(OZ_TN >> 3) << 17) |
         (uint32_t(OZ_TM >> 4) << 24);
}
// One MMA; CU says what the A collector does: 0 = fill (read A, keep it), 1 = use the kept A,
// 2 = use it for the last time.  Consecutive MMAs on the same A tile read it from shared
// memory once.
__device__ __forceinline__ void oz_mma_once(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}
template <int CU>
__device__ __forceinline__ void oz_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  if constexpr (CU == 0)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
  else if constexpr (CU == 1)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ bool oz_wait(uint32_t mbar, uint32_t parity) {
  for (long long spins = 0; spins < kOzSpinLimit; ++spins) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
    if (done) return true;
    __nanosleep(32);
  }
  return false;
}
__device__ __forceinline__ void oz_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}
__device__ __forceinline__ void oz_arrive(uint32_t a) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(a));
}
__device__ __forceinline__ void oz_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(a), "r"(bytes));
}
__device__ __forceinline__ void oz_bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void oz_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}
__device__ __forceinline__ void oz_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// ---------------------------------------------------------------- digit splitting
// |x| as an ordered integer: the bit pattern with the sign cleared (non-negative doubles
// compare like their bit patterns), so the maxima below run on the integer pipe.
__device__ __forceinline__ unsigned long long oz_abs_bits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull;
}
// the smallest e with |x| < 2^e for the largest |x| of a row or column (bit pattern mb),
// e = 0 for zero: m = f 2^e with f in [0.5, 1)
__device__ __forceinline__ int oz_exponent(unsigned long long mb) {
  int e = 0;
  if (mb) frexp(__longlong_as_double(static_cast<long long>(mb)), &e);
  return e;
}
__device__ __forceinline__ unsigned long long oz_umax(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}
// Power-of-two scale exponent per row of a complex128 matrix (rows x cols, ld), the max
// over Re and Im parts.  One warp per row.
__global__ void oz_row_exp_kernel(const double2* __restrict__ A, int64_t rows, int64_t cols, int64_t ld,
                                  int* __restrict__ ex) {
  const int64_t row = int64_t(blockIdx.x) * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  unsigned long long m = 0;
  const double2* a = A + row * ld;
#pragma unroll 4
  for (int64_t k = lane; k < cols; k += 32) {
    const double2 v = a[k];
    m = oz_umax(m, oz_umax(oz_abs_bits(v.x), oz_abs_bits(v.y)));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = oz_umax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if (lane == 0) ex[row] = oz_exponent(m);
}
// the same per column of a matrix stored rows x cols (exponent per column)
__global__ void oz_col_exp_kernel(const double2* __restrict__ A, int64_t rows, int64_t cols, int64_t ld,
                                  int* __restrict__ ex) {
  const int64_t col = blockIdx.x;
  __shared__ unsigned long long red[8];
  unsigned long long m = 0;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) {
    const double2 v = A[r * ld + col];
    m = oz_umax(m, oz_umax(oz_abs_bits(v.x), oz_abs_bits(v.y)));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = oz_umax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < int(blockDim.x >> 5); ++w) m = oz_umax(m, red[w]);
    ex[col] = oz_exponent(m);
  }
}
// x 2^(55 - e) rounded to an integer (|x| < 2^e, so |F| <= 2^55), from the bit pattern:
// x = M 2^(b - 1075) with the 53-bit significand M (b the biased exponent; subnormals have
// b = 1 and no hidden bit), so F = M 2^(b - 1020 - e), a left shift of at most 2 or a right
// shift rounded to nearest (ties away from zero).  Everything below 2^-1 of the last digit
// is dropped here, the same truncation as seven successive digit roundings.
__device__ __forceinline__ long long oz_fixed(double x, int e) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
  int b = int((bits >> 52) & 0x7FF);
  unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
  if (b) m |= 1ull << 52;
  else b = 1;
  const int sh = b - 1020 - e;
  unsigned long long f;
  if (sh >= 0) f = m << sh;
  else if (sh >= -60) f = (m + (1ull << (-sh - 1))) >> (-sh);
  else f = 0;
  return (bits >> 63) ? -static_cast<long long>(f) : static_cast<long long>(f);
}
// bf16 bit pattern of (byte - 128) for an integer byte in [0, 256]: the float 2^23 + byte
// minus 2^23 + 128 is exact, and a float holding an integer of magnitude <= 256 has its
// nonzero bits in the top 16
__device__ __forceinline__ uint32_t oz_bf16_bits(uint32_t byte) {
  return __float_as_uint(__uint_as_float(0x4B000000u | byte) - 8388736.0f) >> 16;
}
// Digit tiles of a matrix read as rows x K elements (element (r, k) at A[r * rs + k * ks]),
// one power-of-two exponent per row, zero-padded to whole tiles of TR rows x 16 k:
// tile (rt, kc, s, p) of TR x 16 bf16 at byte offset (((rt * KC + kc) * 7 + s) * 2 + p) * TR * 32.
// Z (rs = ld, ks = 1, TR = 128) and X read by columns (rs = 1, ks = ld, TR = 32) both land here.
// Digits: F = x 2^(55 - e) rounded (above) is written in balanced base 256,
// F = sum_{s=0..6} d_s 256^(6-s) with d_1..d_6 in [-128, 127] and |d_0| <= 128: adding 128 in
// each of the seven byte positions turns every digit into a plain byte (the carries of the
// balanced form are those of the addition), so d_s = byte_{6-s}(F + 0x80...80) - 128.
// A thread owns 8 consecutive k of one row, one 16-byte row of a core matrix, and writes it
// for every digit and part with one vector store; a warp covers 8 rows x 4 such groups, so
// each store instruction fills two whole 256-byte segments.
template <int TR>
__global__ void oz_split_kernel(const double2* __restrict__ A, int64_t rows, int64_t K, int64_t rs, int64_t ks,
                                const int* __restrict__ ex, int64_t KC, unsigned char* __restrict__ out) {
  constexpr int TILE = TR * OZ_KS * 2;
  constexpr unsigned long long BIAS = 0x0080808080808080ull;
  const int lane = threadIdx.x & 31;
  const int64_t row = int64_t(blockIdx.y) * 8 + (lane & 7);
  const int64_t kg = (int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 4 + (lane >> 3);
  if (kg >= KC * 2) return;
  const int e = row < rows ? ex[row] : 0;
  unsigned long long gr[8], gi[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int64_t k = kg * 8 + j;
    gr[j] = gi[j] = BIAS;
    if (row < rows && k < K) {
      const double2 v = A[row * rs + k * ks];
      gr[j] = static_cast<unsigned long long>(oz_fixed(v.x, e)) + BIAS;
      gi[j] = static_cast<unsigned long long>(oz_fixed(v.y, e)) + BIAS;
    }
  }
  const int64_t rt = row / TR, kc = kg >> 1;
  unsigned char* base = out + ((rt * KC + kc) * OZ_NT) * TILE + oz_off(int(row % TR), int(kg & 1) * 8);
#pragma unroll
  for (int s = 0; s < OZ_ND; ++s) {
    const int sh = 8 * (6 - s);
    uint32_t pr[4], pi[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      // byte 6 (digit 0) may be 256: take it with the bits above
      const uint32_t msk = s == 0 ? 0x1FFu : 0xFFu;
      pr[j] = oz_bf16_bits(uint32_t(gr[2 * j] >> sh) & msk) | (oz_bf16_bits(uint32_t(gr[2 * j + 1] >> sh) & msk) << 16);
      pi[j] = oz_bf16_bits(uint32_t(gi[2 * j] >> sh) & msk) | (oz_bf16_bits(uint32_t(gi[2 * j + 1] >> sh) & msk) << 16);
    }
    *reinterpret_cast<uint4*>(base + (s * 2 + 0) * TILE) = make_uint4(pr[0], pr[1], pr[2], pr[3]);
    *reinterpret_cast<uint4*>(base + (s * 2 + 1) * TILE) = make_uint4(pi[0], pi[1], pi[2], pi[3]);
  }
}
constexpr int OZ_SPLIT_WARPS = 8;  // a block covers 8 rows x 8 warps x 4 groups x 8 k = 8 x 256

// ---------------------------------------------------------------- the product
__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_gemm_kernel(int64_t M, int64_t N, int64_t KC, const unsigned char* __restrict__ Ad,
                   const int* __restrict__ aex, const unsigned char* __restrict__ Bd, const int* __restrict__ bex,
                   double alpha_re, double alpha_im, double beta, double2* __restrict__ C, int64_t ldc, int* status) {
  extern __shared__ unsigned char oz_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(oz_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t bar_full[OZ_STAGES], bar_empty[OZ_STAGES], bar_accf, bar_acce, bar_drain;
  __shared__ uint32_t tmem_sh;
  __shared__ volatile int abort_sh;
  __shared__ volatile int fl_stop;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t RT = (M + OZ_TM - 1) / OZ_TM, CT = (N + OZ_TN - 1) / OZ_TN, tiles = RT * CT;
  const int64_t nch = (KC + OZ_KCH - 1) / OZ_KCH;  // exact chunks per tile
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                 "r"(OZ_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < OZ_STAGES; ++i) {
      oz_init(smem_u32(&bar_full[i]), 1);
      oz_init(smem_u32(&bar_empty[i]), 1);
    }
    oz_init(smem_u32(&bar_accf), 1);
    oz_init(smem_u32(&bar_acce), OZ_FLUSH);
    oz_init(smem_u32(&bar_drain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_sh = 0;
    fl_stop = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_sh;
  auto fail = [&]() {
    abort_sh = 1;
    atomicExch(status, FOSB_ERR_TIMEOUT);
  };

  if (warp == 0) {
    // ---------------------------------------------------------- producer
    if (lane == 0) {
      int64_t it = 0;
      for (int64_t tile = blockIdx.x; tile < tiles && !abort_sh; tile += gridDim.x) {
        const int64_t rt = tile / CT, ct = tile % CT;
        for (int64_t kc = 0; kc < KC; ++kc, ++it) {
          const int st = int(it % OZ_STAGES);
          const int64_t use = it / OZ_STAGES;
          if (use > 0 && !oz_wait(smem_u32(&bar_empty[st]), uint32_t((use - 1) & 1))) {
            fail();
            break;
          }
          unsigned char* sa = smem + st * OZ_STAGE;
          unsigned char* sb = sa + OZ_NT * OZ_ATILE;
          const uint32_t fb = smem_u32(&bar_full[st]);
          oz_expect_tx(fb, OZ_STAGE);
          const unsigned char* ga = Ad + ((rt * KC + kc) * OZ_NT) * OZ_ATILE;
          const unsigned char* gb = Bd + ((ct * KC + kc) * OZ_NT) * OZ_BTILE;
          for (int q = 0; q < OZ_NT; ++q) {
            oz_bulk_load(smem_u32(sa + q * OZ_ATILE), ga + q * OZ_ATILE, OZ_ATILE, fb);
            oz_bulk_load(smem_u32(sb + q * OZ_BTILE), gb + q * OZ_BTILE, OZ_BTILE, fb);
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t id = oz_idesc(false), idn = oz_idesc(true);
      int64_t it = 0, chunks = 0;
      for (int64_t tile = blockIdx.x; tile < tiles && !abort_sh; tile += gridDim.x) {
        for (int64_t c = 0; c < nch && !abort_sh; ++c, ++chunks) {
          // the order accumulators are free once the flush warps have read the last chunk
          if (chunks > 0 && !oz_wait(smem_u32(&bar_acce), uint32_t((chunks - 1) & 1))) {
            fail();
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const int64_t k0 = c * OZ_KCH, k1 = std::min<int64_t>(KC, k0 + OZ_KCH);
          for (int64_t kc = k0; kc < k1; ++kc, ++it) {
            const int st = int(it % OZ_STAGES);
            const int64_t use = it / OZ_STAGES;
            if (!oz_wait(smem_u32(&bar_full[st]), uint32_t(use & 1))) {
              fail();
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            // descriptors of the stage's first A and B tiles; a tile at byte offset X adds
            // X >> 4 to the address field (shared addresses stay below 2^18, no carry)
            const uint32_t a0 = smem_u32(smem + st * OZ_STAGE), b0 = a0 + OZ_NT * OZ_ATILE;
            const uint64_t da = oz_desc(a0), db = oz_desc(b0);
            // the first product into an order's accumulator in a chunk overwrites it
            const uint32_t first = kc == k0 ? 0u : 1u;
            // Each A tile meets its B digits t = 0 .. 6 - s in consecutive MMAs that keep it in
            // the A collector, so it is read from shared memory once per group.  A group must
            // keep one instruction descriptor, so digit s of Re Z is one group (Re and Im of
            // every order), digit s of Im Z two: -Im Z Im X into Re (negate-B), Im Z Re X into Im.
#pragma unroll
            for (int s = 0; s < OZ_ND; ++s) {
              const uint64_t ar = da + uint64_t((s * 2 + 0) * (OZ_ATILE >> 4));
              const uint64_t ai = da + uint64_t((s * 2 + 1) * (OZ_ATILE >> 4));
              const uint32_t acc = s == 0 ? first : 1u;  // s == 0 holds the first pair of each order
              const int T = OZ_ND - s;  // B digits met by this A digit (a constant once unrolled)
#pragma unroll
              for (int t = 0; t < T; ++t) {
                const int g = s + t;
                const uint64_t br = db + uint64_t((t * 2 + 0) * (OZ_BTILE >> 4));
                const uint64_t bi = db + uint64_t((t * 2 + 1) * (OZ_BTILE >> 4));
                const uint32_t dre = tmem + uint32_t(g * 2 + 0) * OZ_TN, dim = tmem + uint32_t(g * 2 + 1) * OZ_TN;
                if (t == 0) oz_mma<0>(dre, ar, br, id, acc);
                else oz_mma<1>(dre, ar, br, id, acc);
                if (t == T - 1) oz_mma<2>(dim, ar, bi, id, acc);
                else oz_mma<1>(dim, ar, bi, id, acc);
              }
#pragma unroll
              for (int half = 0; half < 2; ++half) {
#pragma unroll
                for (int t = 0; t < T; ++t) {
                  const int g = s + t;
                  const uint64_t b = db + uint64_t((t * 2 + (half == 0 ? 1 : 0)) * (OZ_BTILE >> 4));
                  const uint32_t d = tmem + uint32_t(g * 2 + half) * OZ_TN;
                  const uint32_t idd = half == 0 ? idn : id;
                  if (T == 1) oz_mma_once(d, ai, b, idd, 1u);
                  else if (t == 0) oz_mma<0>(d, ai, b, idd, 1u);
                  else if (t == T - 1) oz_mma<2>(d, ai, b, idd, 1u);
                  else oz_mma<1>(d, ai, b, idd, 1u);
                }
              }
            }
            oz_commit(smem_u32(&bar_empty[st]));
          }
          if (abort_sh) break;
          oz_commit(smem_u32(&bar_accf));
        }
      }
      oz_commit(smem_u32(&bar_drain));  // completes once every MMA above has finished
      if (!oz_wait(smem_u32(&bar_drain), 0u)) fail();
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------- flush and epilogue (warps 2-9)
    // TMEM lane group warp % 4 (rows), column half (warp - 2) / 4 of the tile
    const int lane_base = (warp & 3) * 32;
    const int c0 = ((warp - 2) >> 2) * OZ_HN;
    const int r_local = lane_base + lane;
    int64_t chunks = 0;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
      const int64_t rt = tile / CT, ct = tile % CT;
      // orders 0-3: exact integer sum a = sum_g V_g 2^{24-8g} (V_g the integer order sums);
      // orders 4-6 (below 2^-32 of the leading terms): FP32 sum t in the same units, so its
      // rounding stays near 2^-50 of the result; the value is 2^-24 (a + t)
      long long ar_[OZ_HN], ai_[OZ_HN];
      float tr[OZ_HN], ti[OZ_HN];
#pragma unroll
      for (int j = 0; j < OZ_HN; ++j) {
        ar_[j] = ai_[j] = 0ll;
        tr[j] = ti[j] = 0.f;
      }
      for (int64_t c = 0; c < nch; ++c, ++chunks) {
        if (!oz_wait(smem_u32(&bar_accf), uint32_t(chunks & 1))) {
          fail();
          fl_stop = 1;
        }
        asm volatile("bar.sync 1, 256;");  // the stop decision is the same in all eight warps
        if (fl_stop) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
        for (int g = 0; g < OZ_ND; ++g) {
          // both parts of order g in flight together, one wait
          uint32_t v[16], w[16];
          oz_ld16(tmem + (uint32_t(lane_base) << 16) + uint32_t(g * 2 + 0) * OZ_TN + c0, v);
          oz_ld16(tmem + (uint32_t(lane_base) << 16) + uint32_t(g * 2 + 1) * OZ_TN + c0, w);
          asm volatile("tcgen05.wait::ld.sync.aligned;");
          if (g <= 3) {
            const int sh = 24 - 8 * g;
#pragma unroll
            for (int j = 0; j < OZ_HN; ++j) {
              ar_[j] += (long long)__float2int_rn(__uint_as_float(v[j])) << sh;
              ai_[j] += (long long)__float2int_rn(__uint_as_float(w[j])) << sh;
            }
          } else {
            const float sc = __int_as_float((127 + 24 - 8 * g) << 23);  // 2^{24-8g}
#pragma unroll
            for (int j = 0; j < OZ_HN; ++j) {
              tr[j] = fmaf(__uint_as_float(v[j]), sc, tr[j]);
              ti[j] = fmaf(__uint_as_float(w[j]), sc, ti[j]);
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        oz_arrive(smem_u32(&bar_acce));
      }
      if (fl_stop) break;
      const int64_t row = rt * OZ_TM + r_local;
      if (row < M) {
        const double srow = ldexp(1.0, aex[row] - 14);
#pragma unroll
        for (int j = 0; j < OZ_HN; ++j) {
          const int64_t col = ct * OZ_TN + c0 + j;
          if (col < N) {
            const double sc = srow * ldexp(1.0, bex[col]);
            const double xr = ldexp(double(ar_[j]) + double(tr[j]), -24) * sc;
            const double xi = ldexp(double(ai_[j]) + double(ti[j]), -24) * sc;
            double2 v = make_double2(alpha_re * xr - alpha_im * xi, alpha_re * xi + alpha_im * xr);
            if (beta != 0.0) {
              const double2 o = C[row * ldc + col];
              v.x += beta * o.x;
              v.y += beta * o.y;
            }
            C[row * ldc + col] = v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS));
}

inline unsigned oz_cdiv(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }

}  // namespace

size_t oz_a_bytes(int64_t M, int64_t K) {
  return size_t((M + OZ_TM - 1) / OZ_TM) * size_t((K + OZ_KS - 1) / OZ_KS) * OZ_NT * OZ_ATILE;
}

cudaError_t oz_prepare_a(const void* A, int64_t M, int64_t K, int64_t lda, void* digits, int* ex, cudaStream_t s) {
  if (M <= 0 || K <= 0) return cudaSuccess;
  const int64_t KC = (K + OZ_KS - 1) / OZ_KS, MP = ((M + OZ_TM - 1) / OZ_TM) * OZ_TM;
  if (MP / 8 > 65535) return cudaErrorInvalidValue;
  ProfScope prof("oz_prep", s, 44.0 * double(M) * double(K));  // bytes read + written
  oz_row_exp_kernel<<<oz_cdiv(M, 8), 256, 0, s>>>(static_cast<const double2*>(A), M, K, lda, ex);
  oz_split_kernel<OZ_TM><<<dim3(oz_cdiv(KC * 2, OZ_SPLIT_WARPS * 4), unsigned(MP / 8)), OZ_SPLIT_WARPS * 32, 0, s>>>(
      static_cast<const double2*>(A), M, K, lda, 1, ex, KC, static_cast<unsigned char*>(digits));
  return launched(2);
}

cudaError_t oz_gemm(int64_t M, int64_t N, int64_t K, double alpha_re, double alpha_im, const void* a_digits,
                    const int* a_ex, const void* B, int64_t ldb, double beta, void* C, int64_t ldc, int* status,
                    cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  static bool attr[64] = {};
  static int nsm[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  const int64_t KC = (K + OZ_KS - 1) / OZ_KS, CT = (N + OZ_TN - 1) / OZ_TN;
  if (CT * OZ_TN / 8 > 65535) return cudaErrorInvalidValue;
  const size_t bbytes = size_t(CT) * size_t(KC) * OZ_NT * OZ_BTILE;
  unsigned char* bd = nullptr;
  int* bex = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&bd), bbytes, s);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&bex), sizeof(int) * size_t(N), s);
  if (e == cudaSuccess) {
    oz_col_exp_kernel<<<unsigned(N), 256, 0, s>>>(static_cast<const double2*>(B), K, N, ldb, bex);
    oz_split_kernel<OZ_TN><<<dim3(oz_cdiv(KC * 2, OZ_SPLIT_WARPS * 4), unsigned(CT * OZ_TN / 8)), OZ_SPLIT_WARPS * 32,
                             0, s>>>(static_cast<const double2*>(B), N, K, 1, ldb, bex, KC, bd);
    const int64_t tiles = ((M + OZ_TM - 1) / OZ_TM) * CT;
    const unsigned grid = unsigned(std::min<int64_t>(tiles, std::max(nsm[dev], 1)));
    ProfScope prof("gemm_oz", s, 8.0 * double(M) * double(N) * double(K));
    oz_gemm_kernel<<<grid, OZ_THREADS, OZ_SMEM, s>>>(M, N, KC, static_cast<const unsigned char*>(a_digits), a_ex, bd,
                                                      bex, alpha_re, alpha_im, beta, static_cast<double2*>(C), ldc,
                                                      status);
    e = launched(3);
  }
  if (bd) cudaFreeAsync(bd, s);
  if (bex) cudaFreeAsync(bex, s);
  return e;
}

}  // namespace fosb

extern "C" fosb_status fosb_zgemm_fp64class(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B,
                                            int64_t ldb, void* C, int64_t ldc, int method, void* stream) {
  using namespace fosb;
  if (M < 0 || N < 0 || K < 0 || (M > 0 && N > 0 && (!A || !B || !C)) || lda < K || ldb < N || ldc < N)
    return fail(FOSB_ERR_INVALID_ARG, "fosb_zgemm_fp64class: bad arguments");
  if (method != 0 && method != 1) return fail(FOSB_ERR_INVALID_ARG, "fosb_zgemm_fp64class: method must be 0 or 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (M == 0 || N == 0) return FOSB_OK;
  if (K == 0) {
    FOSB_CUDA(cudaMemset2DAsync(C, ldc * 16, 0, N * 16, M, s));
    return FOSB_OK;
  }
  if (method == 1) {
    FOSB_CUDA(gemm_c128_ff(OP_N, OP_N, M, N, K, 1.0, 0.0, A, lda, B, ldb, 0.0, C, ldc, s));
    return FOSB_OK;
  }
  Scratch dig(s), ex(s), st(s);
  FOSB_CUDA(dig.alloc(oz_a_bytes(M, K)));
  FOSB_CUDA(ex.alloc(sizeof(int) * size_t(M)));
  FOSB_CUDA(st.alloc(sizeof(int)));
  FOSB_CUDA(cudaMemsetAsync(st.p, 0, sizeof(int), s));
  FOSB_CUDA(oz_prepare_a(A, M, K, lda, dig.p, ex.as<int>(), s));
  FOSB_CUDA(oz_gemm(M, N, K, 1.0, 0.0, dig.p, ex.as<int>(), B, ldb, 0.0, C, ldc, st.as<int>(), s));
  int status = 0;
  FOSB_CUDA(cudaMemcpyAsync(&status, st.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FOSB_CUDA(cudaStreamSynchronize(s));
  if (status == FOSB_ERR_TIMEOUT) return fail(FOSB_ERR_TIMEOUT, "fosb_zgemm_fp64class: tensor-core wait timed out");
  return FOSB_OK;
}

