// Trailing update C -= A B of the blocked complex64 LU on the tcgen05 tensor cores, fed by
// bulk copies of operands split once per block (3xTF32: x = x_b + x_s, x_b = tf32(x),
//   x y ~ x_b y_b + x_b y_s + x_s y_b).
//
// Split once, copied many times.  A (L21, M x K) and B (U12, K x N) are each split by one
// pass per column block (K <= 256) into the exact shared-memory image the MMAs read: for every
// 128-row (or 128-column) tile and 8-wide k-slab, 4 KB "parts" in the canonical no-swizzle
// K-major layout (8-row x 16-byte core matrices; 128 B between the two core matrices of a
// slab, 256 B between 8-row groups).  Per slab, A has 4 parts (Re_b, Re_s, Im_b, Im_s) and
// B has 6: big [Br_b | Bi_b | -Br_b] then small [Br_s | Bi_s | -Br_s].  A tile's stage is
// then two plain cp.async.bulk copies (16 KB + 24 KB): no per-CTA split, no scattered
// shared-memory stores, and a 3-deep ring that hides the L2 latency.
//
// Complex product with N = 256 MMAs.  The accumulator holds [Re | Im] of a 128 x 128 complex
// tile in 256 TMEM columns, and B is read through two 256-row windows of the contiguous
// parts:  [Br | Bi] (at Br) and [Bi | -Br] (at Bi), so
//   D += A_r [Br | Bi] + (-A_i) [Bi | -Br] = [Ar Br - Ai Bi | Ar Bi + Ai Br]
// (the -A_i by the instruction's negate-A bit): 6 MMAs of 128 x 256 x 8 per slab instead of
// 12 of 128 x 128 x 8, with half the B-operand reads per useful flop.
//
// Roles (persistent, one CTA per SM, tiles in super-rows of 16 row tiles for L2 reuse):
//   warp 0  producer: per slab waits empty[s], expect_tx 40 KB, two bulk copies;
//   warp 1  MMA issuer: waits full[s], 6 MMAs into accumulator buffer b, commits empty[s];
//           after a tile's last slab commits tfull[b];
//   warps 2-5 epilogue (TMEM lane quarters 2, 3, 0, 1): per 64-column half, C is prefetched
//           by cp.async into a padded shared tile, the accumulator row of each thread is
//           subtracted in place, and the half is stored with coalesced 16-byte writes.
// Every wait is bounded; a time-out sets the status word and an abort flag, the MMA thread
// drains its MMAs and the producer waits for its copies in flight before TMEM is freed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "fosb_internal.h"

namespace fosb {
namespace {

constexpr int U_TM = 128, U_TN = 128;          // tile: 128 rows x 128 complex columns
constexpr int U_KB = kLuBlock;                 // largest k extent of a split block (32 slabs)
constexpr int U_SLABS = U_KB / 8;
constexpr int U_PART = 4096;                   // one 128 x 8 tf32 part
constexpr int U_ABYTES = 4 * U_PART;           // A parts of one slab
constexpr int U_BBYTES = 6 * U_PART;           // B parts of one slab
constexpr int U_STAGE = U_ABYTES + U_BBYTES;   // 40 KB
constexpr int U_STAGES = 3;
constexpr int U_EPI_LD = 66;                   // padded float2 row of the 64-column tile (16-byte rows)
constexpr int U_EPI_BYTES = U_TM * U_EPI_LD * 8;
constexpr int U_EPI_OFF = U_STAGES * U_STAGE;
constexpr int U_SMEM = U_EPI_OFF + U_EPI_BYTES + 1024;  // + alignment slack
constexpr int U_THREADS = 6 * 32;
constexpr int U_GROUP = 16;                    // row tiles per super-row
constexpr long long U_SPIN = 1ll << 24;
static_assert(U_SMEM <= 227 * 1024, "stages and drain tile exceed shared memory");

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ float tf32r(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// byte offset of element (row, k8) of a part: 8-row groups 256 B apart, k halves 128 B apart
__host__ __device__ __forceinline__ int part_off(int row, int k8) {
  return (row >> 3) * 256 + (k8 >> 2) * 128 + (row & 7) * 16 + (k8 & 3) * 4;
}
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t(128 >> 4) << 16) | (uint64_t(256 >> 4) << 32) |
         (uint64_t(1) << 46);
}
// kind::tf32: D f32, A/B tf32, K-major, N = 256, M = 128, optional negate-A (bit 13)
__host__ __device__ constexpr uint32_t u_idesc(bool neg_a) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (neg_a ? (1u << 13) : 0u) | (uint32_t(256 >> 3) << 17) |
         (uint32_t(U_TM >> 4) << 24);
}
__device__ __forceinline__ void u_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ bool u_wait(uint32_t mbar, uint32_t parity) {
  for (long long i = 0; i < U_SPIN; ++i) {
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
__device__ __forceinline__ void u_init(uint32_t a, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(n));
}
__device__ __forceinline__ void u_arrive(uint32_t a) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(a));
}
__device__ __forceinline__ void u_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(a), "r"(bytes));
}
__device__ __forceinline__ void u_bulk(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void u_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}
__device__ __forceinline__ void u_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void u_bar(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n)); }
// 16-byte global -> shared copy that bypasses the registers; bytes < 16 zero-fills the rest
__device__ __forceinline__ void u_cp16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
// float2 index of the 16-byte piece holding columns (2 j, 2 j + 1) of row r in the 64-column
// drain tile; the 528-byte row pitch keeps 8 consecutive rows reading piece j in 8 different
// bank groups (row-per-thread phase) and a row's 32 pieces contiguous (coalesced phases)
__device__ __forceinline__ int u_piece(int r, int j) { return r * U_EPI_LD + (j << 1); }
__device__ __forceinline__ void u_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void u_cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// ---------------------------------------------------------------- splits
// A (M x K, lda), K <= 256 in nslab = ceil(K / 8) slabs: out[(rt * nslab + s) * 16 KB + p * 4 KB +
// part_off(r, k8)], parts Re_b, Re_s, Im_b, Im_s; zero outside M x K.  One thread per (row, k)
// of the padded tile grid.
__global__ void split_a_kernel(int64_t M, int K, int nslab, const float2* __restrict__ A, int64_t lda,
                               float* __restrict__ out, int64_t rows_pad) {
  const int kp = nslab * 8;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= rows_pad * kp) return;
  const int64_t row = e / kp;
  const int k = int(e % kp);
  const float2 v = (row < M && k < K) ? A[row * lda + k] : make_float2(0.f, 0.f);
  const float rb = tf32r(v.x), ib = tf32r(v.y);
  float* base = out + ((row / U_TM) * nslab + k / 8) * (U_ABYTES / 4) + part_off(int(row % U_TM), k & 7) / 4;
  base[0 * U_PART / 4] = rb;
  base[1 * U_PART / 4] = tf32r(v.x - rb);
  base[2 * U_PART / 4] = ib;
  base[3 * U_PART / 4] = tf32r(v.y - ib);
}
// B (K x N, ldb), K <= 256: out[(ct * nslab + s) * 24 KB + p * 4 KB + part_off(c, k8)], parts
// Br_b, Bi_b, -Br_b, Br_s, Bi_s, -Br_s; zero outside K x N.  Threads run along N (coalesced).
__global__ void split_b_kernel(int64_t N, int K, int nslab, const float2* __restrict__ B, int64_t ldb,
                               float* __restrict__ out, int64_t cols_pad) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= cols_pad * nslab * 8) return;
  const int k = int(e / cols_pad);
  const int64_t col = e % cols_pad;
  const float2 v = (col < N && k < K) ? B[int64_t(k) * ldb + col] : make_float2(0.f, 0.f);
  const float rb = tf32r(v.x), ib = tf32r(v.y);
  const float rs = tf32r(v.x - rb), is = tf32r(v.y - ib);
  float* base = out + ((col / U_TN) * nslab + k / 8) * (U_BBYTES / 4) + part_off(int(col % U_TN), k & 7) / 4;
  base[0 * U_PART / 4] = rb;
  base[1 * U_PART / 4] = ib;
  base[2 * U_PART / 4] = -rb;
  base[3 * U_PART / 4] = rs;
  base[4 * U_PART / 4] = is;
  base[5 * U_PART / 4] = -rs;
}

// tile index -> (row tile, column tile): super-rows of U_GROUP row tiles, columns inside
__device__ __forceinline__ void tile_rc(int64_t tile, int64_t RT, int64_t CT, int64_t& rt, int64_t& ct) {
  const int64_t g = tile / (int64_t(U_GROUP) * CT);
  const int64_t local = tile - g * U_GROUP * CT;
  const int64_t gr = min(int64_t(U_GROUP), RT - g * U_GROUP);
  ct = local / gr;
  rt = g * U_GROUP + local % gr;
}

// ---------------------------------------------------------------- the update
__global__ void __launch_bounds__(U_THREADS, 1)
    cgemm_update_split_kernel(int64_t M, int64_t N, int nslab, const unsigned char* __restrict__ As,
                              const unsigned char* __restrict__ Bs, float2* __restrict__ C, int64_t ldc, int* status,
                              int vec_ok) {
  extern __shared__ unsigned char u_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(u_raw) + 1023) & ~uintptr_t(1023));
  float2* sE = reinterpret_cast<float2*>(smem + U_EPI_OFF);
  __shared__ uint64_t bar_full[U_STAGES], bar_empty[U_STAGES], bar_tfull[2], bar_tempty[2], bar_drain;
  __shared__ uint32_t tmem_sh;
  __shared__ volatile int abort_sh;
  __shared__ volatile int epi_stop;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t RT = (M + U_TM - 1) / U_TM, CT = (N + U_TN - 1) / U_TN, tiles = RT * CT;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_sh)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < U_STAGES; ++i) {
      u_init(su32(&bar_full[i]), 1);
      u_init(su32(&bar_empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      u_init(su32(&bar_tfull[i]), 1);
      u_init(su32(&bar_tempty[i]), 128);
    }
    u_init(su32(&bar_drain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_sh = 0;
    epi_stop = 0;
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
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int64_t it = 0;
      for (int64_t tile = blockIdx.x; tile < tiles && !abort_sh; tile += gridDim.x) {
        int64_t rt, ct;
        tile_rc(tile, RT, CT, rt, ct);
        for (int s = 0; s < nslab; ++s, ++it) {
          const int st = int(it % U_STAGES);
          const int64_t use = it / U_STAGES;
          if (use > 0 && !u_wait(su32(&bar_empty[st]), uint32_t((use - 1) & 1))) {
            fail();
            break;
          }
          unsigned char* sa = smem + st * U_STAGE;
          const uint32_t fb = su32(&bar_full[st]);
          u_expect_tx(fb, U_STAGE);
          u_bulk(su32(sa), As + (rt * nslab + s) * int64_t(U_ABYTES), U_ABYTES, fb);
          u_bulk(su32(sa + U_ABYTES), Bs + (ct * nslab + s) * int64_t(U_BBYTES), U_BBYTES, fb);
        }
      }
      // wait for every copy issued here that the MMA thread may not have consumed
      for (int64_t j = it > U_STAGES ? it - U_STAGES : 0; j < it; ++j)
        if (!u_wait(su32(&bar_full[int(j % U_STAGES)]), uint32_t((j / U_STAGES) & 1))) fail();
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id = u_idesc(false), idn = u_idesc(true);
      int64_t it = 0, tcount = 0;
      for (int64_t tile = blockIdx.x; tile < tiles && !abort_sh; tile += gridDim.x, ++tcount) {
        const int b = int(tcount & 1);
        const int64_t ub = tcount >> 1;
        if (ub > 0 && !u_wait(su32(&bar_tempty[b]), uint32_t((ub - 1) & 1))) {
          fail();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t d = tmem + uint32_t(b) * 256;
        for (int s = 0; s < nslab; ++s, ++it) {
          const int st = int(it % U_STAGES);
          const int64_t use = it / U_STAGES;
          if (!u_wait(su32(&bar_full[st]), uint32_t(use & 1))) {
            fail();
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t a0 = su32(smem + st * U_STAGE), b0 = a0 + U_ABYTES;
          const uint64_t arb = sdesc(a0), ars = sdesc(a0 + U_PART), aib = sdesc(a0 + 2 * U_PART),
                         ais = sdesc(a0 + 3 * U_PART);
          // B windows: [Br | Bi] at part 0 (big) / 3 (small); [Bi | -Br] at part 1 / 4
          const uint64_t w1b = sdesc(b0), w1s = sdesc(b0 + 3 * U_PART);
          const uint64_t w2b = sdesc(b0 + U_PART), w2s = sdesc(b0 + 4 * U_PART);
          const uint32_t acc0 = s > 0 ? 1u : 0u;
          u_mma(d, arb, w1b, id, acc0);
          u_mma(d, arb, w1s, id, 1u);
          u_mma(d, ars, w1b, id, 1u);
          u_mma(d, aib, w2b, idn, 1u);
          u_mma(d, aib, w2s, idn, 1u);
          u_mma(d, ais, w2b, idn, 1u);
          u_commit(su32(&bar_empty[st]));
        }
        if (abort_sh) break;
        u_commit(su32(&bar_tfull[b]));
      }
      u_commit(su32(&bar_drain));  // completes once every MMA issued above has finished
      if (!u_wait(su32(&bar_drain), 0u)) fail();
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue (warps 2-5)
    // Per 64-column half of a tile: the C half-tile is copied into the padded shared tile by
    // cp.async (4096 16-byte pieces in flight; for the first half issued before the
    // accumulator wait), thread r subtracts its TMEM row (lane r) in place, and the half is
    // stored with coalesced 16-byte writes.  Without 16-byte alignment of C the tile takes
    // the negated accumulator and C is updated element by element.
    const int et = tid - 2 * 32;             // 0..127
    const int lane_base = (warp & 3) * 32;   // TMEM lane quarter of this warp
    const int r_local = lane_base + lane;
    int64_t tcount = 0;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++tcount) {
      const int b = int(tcount & 1);
      const int64_t ub = tcount >> 1;
      int64_t rt, ct;
      tile_rc(tile, RT, CT, rt, ct);
      const int64_t row0 = rt * U_TM, col0 = ct * U_TN;
      const uint32_t d = tmem + uint32_t(b) * 256 + (uint32_t(lane_base) << 16);
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        if (vec_ok) {
#pragma unroll 8
          for (int q = 0; q < 32; ++q) {
            const int e = et + 128 * q;  // 0 .. 4095 pairs of complex
            const int r = e >> 5, c = (e & 31) * 2;
            const int64_t gr = row0 + r, gc = col0 + h * 64 + c;
            const int bytes = gr < M ? (gc + 1 < N ? 16 : (gc < N ? 8 : 0)) : 0;
            u_cp16(su32(&sE[u_piece(r, c >> 1)]), bytes ? static_cast<const void*>(C + gr * ldc + gc) : C, bytes);
          }
          u_cp_commit();
        }
        if (h == 0) {
          // the stop decision must be the same in all four warps (they share named barriers)
          if (!u_wait(su32(&bar_tfull[b]), uint32_t(ub & 1))) {
            fail();
            epi_stop = 1;
          }
          u_bar(1, 128);
          if (epi_stop) {
            u_cp_wait_all();  // no copy may land after the kernel has left
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
        }
        if (vec_ok) {
          u_cp_wait_all();
          u_bar(1, 128);  // every thread's pieces of C are in the tile
        }
#pragma unroll 1
        for (int cs = 0; cs < 2; ++cs) {
          uint32_t vr[32], vi[32];
          u_ld32(d + h * 64 + cs * 32, vr);
          u_ld32(d + 128 + h * 64 + cs * 32, vi);
          asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
          for (int j = 0; j < 32; j += 2) {
            float4* p = reinterpret_cast<float4*>(&sE[u_piece(r_local, cs * 16 + (j >> 1))]);
            float4 c4 = vec_ok ? *p : make_float4(0.f, 0.f, 0.f, 0.f);
            c4.x -= __uint_as_float(vr[j]);
            c4.y -= __uint_as_float(vi[j]);
            c4.z -= __uint_as_float(vr[j + 1]);
            c4.w -= __uint_as_float(vi[j + 1]);
            *p = c4;
          }
        }
        if (h == 1) {  // every accumulator value of this buffer has been read
          asm volatile("tcgen05.fence::before_thread_sync;");
          u_arrive(su32(&bar_tempty[b]));
        }
        u_bar(1, 128);
        if (vec_ok) {
#pragma unroll 8
          for (int q = 0; q < 32; ++q) {
            const int e = et + 128 * q;
            const int r = e >> 5, c = (e & 31) * 2;
            const int64_t gr = row0 + r, gc = col0 + h * 64 + c;
            if (gr < M && gc + 1 < N) {
              *reinterpret_cast<float4*>(C + gr * ldc + gc) = *reinterpret_cast<const float4*>(&sE[u_piece(r, c >> 1)]);
            } else if (gr < M && gc < N) {
              C[gr * ldc + gc] = sE[u_piece(r, c >> 1)];
            }
          }
        } else {
#pragma unroll 4
          for (int q = 0; q < 64; ++q) {
            const int e = et + 128 * q;  // 0 .. 8191
            const int r = e >> 6, c = e & 63;
            const int64_t gr = row0 + r, gc = col0 + h * 64 + c;
            if (gr < M && gc < N) {  // the tile holds -D here: C += it
              const float2 dd = sE[u_piece(r, c >> 1) + (c & 1)];
              float2 o = C[gr * ldc + gc];
              o.x += dd.x;
              o.y += dd.y;
              C[gr * ldc + gc] = o;
            }
          }
        }
        u_bar(1, 128);  // the tile is free for the next half's copies
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

inline unsigned ucdiv(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }

}  // namespace

size_t update_split_a_bytes(int64_t M) { return size_t((M + U_TM - 1) / U_TM) * U_SLABS * U_ABYTES; }
size_t update_split_b_bytes(int64_t N) { return size_t((N + U_TN - 1) / U_TN) * U_SLABS * U_BBYTES; }

// C (M x N) -= A (M x K) B (K x N), complex64 row-major, K <= kLuBlock: split A and B once into
// the workspaces (update_split_a_bytes(M), update_split_b_bytes(N) bytes, 16-byte aligned),
// then the bulk-copy-fed tcgen05 update.
cudaError_t cgemm_update_tc_split(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B,
                                  int64_t ldb, void* C, int64_t ldc, int* status, void* ws_a, void* ws_b,
                                  cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  if (K > U_KB) return cudaErrorInvalidValue;
  static bool attr[64] = {};
  static int nsm[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(cgemm_update_split_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, U_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  const int64_t RT = (M + U_TM - 1) / U_TM, CT = (N + U_TN - 1) / U_TN;
  const int64_t rows_pad = RT * U_TM, cols_pad = CT * U_TN;
  ProfScope prof("lu_update", s, 8.0 * double(M) * double(N) * double(K));  // the splits are part of it
  const int nslab = int((K + 7) / 8);  // tiles packed with exactly nslab slabs each
  split_a_kernel<<<ucdiv(rows_pad * nslab * 8, 256), 256, 0, s>>>(M, int(K), nslab, static_cast<const float2*>(A), lda,
                                                                static_cast<float*>(ws_a), rows_pad);
  split_b_kernel<<<ucdiv(cols_pad * nslab * 8, 256), 256, 0, s>>>(N, int(K), nslab, static_cast<const float2*>(B), ldb,
                                                                static_cast<float*>(ws_b), cols_pad);
  note_launches(2);
  const unsigned grid = unsigned(std::min<int64_t>(RT * CT, std::max(nsm[dev], 1)));
  const int vec_ok = (reinterpret_cast<uintptr_t>(C) % 16 == 0) && (ldc % 2 == 0);
  cgemm_update_split_kernel<<<grid, U_THREADS, U_SMEM, s>>>(M, N, nslab, static_cast<const unsigned char*>(ws_a),
                                                          static_cast<const unsigned char*>(ws_b),
                                                          static_cast<float2*>(C), ldc, status, vec_ok);
  return launched();
}

}  // namespace fosb
