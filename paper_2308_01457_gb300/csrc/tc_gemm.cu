// Complex64 rank-k update C -= A B on the 5th-generation tensor cores (tcgen05, TF32),
// with 3xTF32 splitting for FP32-class accuracy: x = x_b + x_s (x_b = tf32(x)), and
//   x y ~ x_b y_b + x_b y_s + x_s y_b.
// Re(C) -= Ar Br - Ai Bi and Im(C) -= Ar Bi + Ai Br give 12 MMAs (M = 128, N = 128,
// K = 8) per k-slab of 8; the minus sign of Ai Bi uses the instruction's negate-A bit.
//
// Output tile 128 x 128 complex; accumulators Re and Im in TMEM (128 lanes x 128 fp32
// columns each).  K is consumed in chunks of 16, stored split in the canonical no-swizzle
// K-major layout (8 x 16-byte core matrices; LBO = 128 B between the two core matrices of a
// k-slab, SBO = 256 B between 8-row groups).
#include <cuda_runtime.h>

#include <algorithm>

#include <cstdint>

#include "fosb_internal.h"

namespace fosb {
namespace {

constexpr int TC_M = 128, TC_N = 128, TC_KC = 16;       // tile rows, tile complex columns, k-chunk
constexpr int SLAB = 128 * 8 * 4;                        // bytes per k-slab of one 128-row operand part
constexpr int PART = SLAB * (TC_KC / 8);                 // 8192 bytes per part per chunk
constexpr int SMEM_A = 4 * PART, SMEM_B = 4 * PART;      // parts: re_b, re_s, im_b, im_s
constexpr int EPI_LD = 66;                               // padded float2 row stride of the epilogue tile (16-B rows)
constexpr int SMEM_EPI = TC_M * EPI_LD * 8;              // 67584 bytes (epilogue tile)
constexpr int TMEM_COLS = 256;
constexpr long long kMmaSpinLimit = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// canonical K-major no-swizzle offset of element (row, k) inside one k-slab
__device__ __forceinline__ int kmajor_off(int row, int k8) {
  return (row >> 3) * 256 + (k8 >> 2) * 128 + (row & 7) * 16 + (k8 & 3) * 4;
}
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = 256;
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}
// kind::tf32 instruction descriptor: D f32 (bits 4-5 = 1), A/B tf32 (bits 7-9, 10-12 = 2),
// K-major A and B, N >> 3 at bits 17-22, M >> 4 at bits 24-28, optional negate-A (bit 13).
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N, bool neg_a) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (neg_a ? (1u << 13) : 0u) | (uint32_t(N >> 3) << 17) |
         (uint32_t(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}
// Non-blocking probe + short sleep: at most kMmaSpinLimit probes (about 2 s) in total.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long spins = 0; spins < kMmaSpinLimit; ++spins) {
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
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
// split x into the tf32 pair and store both parts of re and im at `off` of the 4 parts
__device__ __forceinline__ void store_split(unsigned char* base, int off, float2 v) {
  const float rb = tf32_round(v.x), ib = tf32_round(v.y);
  *reinterpret_cast<float*>(base + 0 * PART + off) = rb;
  *reinterpret_cast<float*>(base + 1 * PART + off) = tf32_round(v.x - rb);
  *reinterpret_cast<float*>(base + 2 * PART + off) = ib;
  *reinterpret_cast<float*>(base + 3 * PART + off) = tf32_round(v.y - ib);
}

// ---------------------------------------------------------------------------------------
// Persistent, warp-specialised form of the same update (one CTA per SM, tiles strided over
// the grid).  Roles:
//   warps 0-7  producers: global -> registers -> 3xTF32 split -> stage s of a 2-stage
//              shared-memory ring (64 KB per stage), then arrive on full[s];
//   warp 8     MMA issuer: per chunk waits full[s], issues the 24 MMAs into accumulator
//              buffer b (two buffers x 256 TMEM columns), commits to empty[s]; after a
//              tile's last chunk commits to tmem_full[b];
//   warps 9-12 epilogue (TMEM lane groups 1, 2, 3, 0): wait tmem_full[b], drain the
//              accumulators, release the buffer on tmem_empty[b], then update C through a
//              padded shared tile with coalesced 16-byte read-modify-writes.
// So the C traffic of tile i overlaps the MMAs of tile i + 1, and staging overlaps MMAs.
// Every wait is bounded; a time-out sets the status word, raises an abort flag that all
// roles poll, and the MMA thread drains its outstanding MMAs before TMEM is freed.
constexpr int WS_STAGES = 2;
constexpr int WS_STAGE_BYTES = SMEM_A + SMEM_B;                       // 64 KB
constexpr int WS_EPI_OFF = WS_STAGES * WS_STAGE_BYTES;                // 128 KB
constexpr int WS_SMEM = WS_EPI_OFF + SMEM_EPI + 1024;                 // + alignment slack
constexpr int WS_THREADS = 13 * 32;
constexpr int WS_PRODUCERS = 256;
static_assert(WS_SMEM <= 227 * 1024, "warp-specialised tile does not fit shared memory");

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(a));
}
__device__ __forceinline__ void named_bar(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n)); }
// 16-byte global -> shared copy that bypasses the registers; bytes < 16 zero-fills the rest
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__global__ void __launch_bounds__(WS_THREADS, 1)
    cgemm_update_tc_ws_kernel(int64_t M, int64_t N, int64_t K, const float2* __restrict__ A, int64_t lda,
                              const float2* __restrict__ B, int64_t ldb, float2* __restrict__ C, int64_t ldc,
                              int* status, int vec_ok) {
  extern __shared__ unsigned char tc_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
  float2* sE = reinterpret_cast<float2*>(smem + WS_EPI_OFF);
  __shared__ uint64_t bar_full[WS_STAGES], bar_empty[WS_STAGES], bar_tfull[2], bar_tempty[2], bar_drain;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_sh;
  __shared__ volatile int epi_stop;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t tiles_n = (N + TC_N - 1) / TC_N, tiles = tiles_n * ((M + TC_M - 1) / TC_M);
  const int64_t nchunk = (K + TC_KC - 1) / TC_KC;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(2 * TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < WS_STAGES; ++i) {
      mbar_init(smem_u32(&bar_full[i]), WS_PRODUCERS);
      mbar_init(smem_u32(&bar_empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&bar_tfull[i]), 1);
      mbar_init(smem_u32(&bar_tempty[i]), 128);
    }
    mbar_init(smem_u32(&bar_drain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_sh = 0;
    epi_stop = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_sh;
  auto fail = [&]() {
    abort_sh = 1;
    atomicExch(status, FOSB_ERR_TIMEOUT);
  };

  if (warp < 8) {
    // ------------------------------------------------------------ producers
    const int k3 = lane & 3, rc = lane >> 2;
    float2 va[8], vb[8];
    auto load_chunk = [&](int64_t row0, int64_t col0, int64_t k0) {
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int w = warp + 8 * it;
        const int khi = w & 3, rg = w >> 2;
        const int r = rg * 8 + rc, kk = (khi >> 1) * 8 + (khi & 1) * 4 + k3;
        const int64_t gr = row0 + r, gk = k0 + kk;
        va[it] = (gr < M && gk < K) ? A[gr * lda + gk] : make_float2(0.f, 0.f);
        const int cg = w & 15, kb = w >> 4;
        const int c = cg * 8 + rc, kkb = (kb >> 1) * 8 + (kb & 1) * 4 + k3;
        const int64_t gc = col0 + c, gkb = k0 + kkb;
        vb[it] = (gc < N && gkb < K) ? B[gkb * ldb + gc] : make_float2(0.f, 0.f);
      }
    };
    int64_t it_glob = 0;
    bool have = false;
    int64_t tile = blockIdx.x;
    if (tile < tiles) {
      load_chunk((tile / tiles_n) * TC_M, (tile % tiles_n) * TC_N, 0);
      have = true;
    }
    for (; tile < tiles && have; tile += gridDim.x) {
      const int64_t row0 = (tile / tiles_n) * TC_M, col0 = (tile % tiles_n) * TC_N;
      for (int64_t ch = 0; ch < nchunk; ++ch, ++it_glob) {
        const int st = int(it_glob % WS_STAGES);
        const int64_t use = it_glob / WS_STAGES;
        if (use > 0 && !mbar_wait(smem_u32(&bar_empty[st]), uint32_t((use - 1) & 1))) fail();
        if (abort_sh) {
          have = false;
          break;
        }
        unsigned char* sA = smem + st * WS_STAGE_BYTES;
        unsigned char* sB = sA + SMEM_A;
#pragma unroll
        for (int it = 0; it < 8; ++it) {
          const int w = warp + 8 * it;
          const int khi = w & 3, rg = w >> 2;
          const int r = rg * 8 + rc, k8 = (khi & 1) * 4 + k3;
          store_split(sA, (khi >> 1) * SLAB + kmajor_off(r, k8), va[it]);
          const int cg = w & 15, kb = w >> 4;
          const int c = cg * 8 + rc, k8b = (kb & 1) * 4 + k3;
          store_split(sB, (kb >> 1) * SLAB + kmajor_off(c, k8b), vb[it]);
        }
        asm volatile("fence.proxy.async.shared::cta;");
        mbar_arrive(smem_u32(&bar_full[st]));
        // prefetch the next chunk (this tile's or the next tile's first) while MMAs run
        if (ch + 1 < nchunk) {
          load_chunk(row0, col0, (ch + 1) * TC_KC);
        } else if (tile + gridDim.x < tiles) {
          const int64_t nt = tile + gridDim.x;
          load_chunk((nt / tiles_n) * TC_M, (nt % tiles_n) * TC_N, 0);
        }
      }
    }
  } else if (warp == 8) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id = idesc_tf32(TC_M, TC_N, false), idn = idesc_tf32(TC_M, TC_N, true);
      int64_t it_glob = 0, tcount = 0;
      for (int64_t tile = blockIdx.x; tile < tiles && !abort_sh; tile += gridDim.x, ++tcount) {
        const int b = int(tcount & 1);
        const int64_t ub = tcount >> 1;
        if (ub > 0 && !mbar_wait(smem_u32(&bar_tempty[b]), uint32_t((ub - 1) & 1))) {
          fail();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t d_re = tmem + uint32_t(b) * TMEM_COLS, d_im = d_re + TC_N;
        for (int64_t ch = 0; ch < nchunk; ++ch, ++it_glob) {
          const int st = int(it_glob % WS_STAGES);
          const int64_t use = it_glob / WS_STAGES;
          if (!mbar_wait(smem_u32(&bar_full[st]), uint32_t(use & 1))) {
            fail();
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t a0 = smem_u32(smem + st * WS_STAGE_BYTES), b0 = a0 + SMEM_A;
#pragma unroll
          for (int sl = 0; sl < TC_KC / 8; ++sl) {
            const uint64_t arb = smem_desc(a0 + 0 * PART + sl * SLAB), ars = smem_desc(a0 + 1 * PART + sl * SLAB);
            const uint64_t aib = smem_desc(a0 + 2 * PART + sl * SLAB), ais = smem_desc(a0 + 3 * PART + sl * SLAB);
            const uint64_t brb = smem_desc(b0 + 0 * PART + sl * SLAB), brs = smem_desc(b0 + 1 * PART + sl * SLAB);
            const uint64_t bib = smem_desc(b0 + 2 * PART + sl * SLAB), bis = smem_desc(b0 + 3 * PART + sl * SLAB);
            const uint32_t acc0 = (ch > 0 || sl > 0) ? 1u : 0u;
            mma_tf32(d_re, arb, brb, id, acc0);
            mma_tf32(d_re, arb, brs, id, 1u);
            mma_tf32(d_re, ars, brb, id, 1u);
            mma_tf32(d_re, aib, bib, idn, 1u);
            mma_tf32(d_re, aib, bis, idn, 1u);
            mma_tf32(d_re, ais, bib, idn, 1u);
            mma_tf32(d_im, arb, bib, id, acc0);
            mma_tf32(d_im, arb, bis, id, 1u);
            mma_tf32(d_im, ars, bib, id, 1u);
            mma_tf32(d_im, aib, brb, id, 1u);
            mma_tf32(d_im, aib, brs, id, 1u);
            mma_tf32(d_im, ais, brb, id, 1u);
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&bar_empty[st])));
        }
        if (abort_sh) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&bar_tfull[b])));
      }
      // drain: completes once every MMA issued above has finished
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&bar_drain)));
      if (!mbar_wait(smem_u32(&bar_drain), 0u)) fail();
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue (128 threads)
    // Per 64-column half of a tile: (1) the C half-tile goes to the padded shared tile by
    // cp.async, all 4096 16-byte pieces in flight at once and, for the first half, issued
    // before the accumulator is waited for; (2) thread r subtracts its TMEM row (lane r) in
    // place; (3) coalesced 16-byte stores.  Without 16-byte alignment of C the tile takes the
    // accumulator and C is updated element by element.
    const int et = tid - 9 * 32;              // 0..127
    const int lane_base = (warp & 3) * 32;    // TMEM lane group of this warp
    const int r_local = lane_base + lane;
    int64_t tcount = 0;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++tcount) {
      const int b = int(tcount & 1);
      const int64_t ub = tcount >> 1;
      const int64_t row0 = (tile / tiles_n) * TC_M, col0 = (tile % tiles_n) * TC_N;
      const uint32_t d_re = tmem + uint32_t(b) * TMEM_COLS, d_im = d_re + TC_N;
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        if (vec_ok) {
#pragma unroll 8
          for (int q = 0; q < 32; ++q) {
            const int e = et + 128 * q;  // 0 .. 4095 pairs of complex
            const int r = e >> 5, c = (e & 31) * 2;
            const int64_t gr = row0 + r, gc = col0 + h * 64 + c;
            const int bytes = gr < M ? (gc + 1 < N ? 16 : (gc < N ? 8 : 0)) : 0;
            cp_async16(smem_u32(&sE[r * EPI_LD + c]), bytes ? static_cast<const void*>(C + gr * ldc + gc) : C, bytes);
          }
          cp_async_commit();
        }
        if (h == 0) {
          // the stop decision must be the same in all four epilogue warps (they share named
          // barriers): a flag written before and read after one
          if (!mbar_wait(smem_u32(&bar_tfull[b]), uint32_t(ub & 1))) {
            fail();
            epi_stop = 1;
          }
          named_bar(1, 128);
          if (epi_stop) {
            cp_async_wait_all();  // no copy may land after the kernel has left
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
        }
        if (vec_ok) {
          cp_async_wait_all();
          named_bar(1, 128);  // every thread's pieces of C are in the tile
        }
#pragma unroll 1
        for (int cs = 0; cs < 2; ++cs) {
          uint32_t vr[32], vi[32];
          tmem_ld32(d_re + (uint32_t(lane_base) << 16) + h * 64 + cs * 32, vr);
          tmem_ld32(d_im + (uint32_t(lane_base) << 16) + h * 64 + cs * 32, vi);
          asm volatile("tcgen05.wait::ld.sync.aligned;");
          float2* row = sE + r_local * EPI_LD + cs * 32;
          if (vec_ok) {
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
              float4 c4 = *reinterpret_cast<float4*>(row + j);
              c4.x -= __uint_as_float(vr[j]);
              c4.y -= __uint_as_float(vi[j]);
              c4.z -= __uint_as_float(vr[j + 1]);
              c4.w -= __uint_as_float(vi[j + 1]);
              *reinterpret_cast<float4*>(row + j) = c4;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) row[j] = make_float2(__uint_as_float(vr[j]), __uint_as_float(vi[j]));
          }
        }
        if (h == 1) {  // every accumulator value of this buffer has been read
          asm volatile("tcgen05.fence::before_thread_sync;");
          mbar_arrive(smem_u32(&bar_tempty[b]));
        }
        named_bar(1, 128);
        if (vec_ok) {
#pragma unroll 8
          for (int q = 0; q < 32; ++q) {
            const int e = et + 128 * q;
            const int r = e >> 5, c = (e & 31) * 2;
            const int64_t gr = row0 + r, gc = col0 + h * 64 + c;
            if (gr < M && gc + 1 < N) {
              *reinterpret_cast<float4*>(C + gr * ldc + gc) = *reinterpret_cast<const float4*>(&sE[r * EPI_LD + c]);
            } else if (gr < M && gc < N) {
              C[gr * ldc + gc] = sE[r * EPI_LD + c];
            }
          }
        } else {
#pragma unroll 4
          for (int q = 0; q < 64; ++q) {
            const int e = et + 128 * q;  // 0 .. 8191
            const int r = e >> 6, c = e & 63;
            const int64_t gr = row0 + r, gc = col0 + h * 64 + c;
            if (gr < M && gc < N) {
              const float2 d = sE[r * EPI_LD + c];
              float2 o = C[gr * ldc + gc];
              o.x -= d.x;
              o.y -= d.y;
              C[gr * ldc + gc] = o;
            }
          }
        }
        named_bar(1, 128);  // the tile is free for the next half's copies
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TMEM_COLS));
}

inline unsigned cdiv(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }

}  // namespace

// C (M x N) -= A (M x K) B (K x N), complex64 row-major, on tcgen05 (3xTF32).
cudaError_t cgemm_update_tc(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B, int64_t ldb,
                            void* C, int64_t ldc, int* status, cudaStream_t s, const char* family) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  static bool attr[64] = {};
  static int nsm[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(cgemm_update_tc_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, WS_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  const int64_t tiles = int64_t(cdiv(N, TC_N)) * cdiv(M, TC_M);
  const unsigned grid = unsigned(std::min<int64_t>(tiles, std::max(nsm[dev], 1)));  // persistent: one CTA per SM
  // 16-byte epilogue accesses need a 16-byte aligned C with an even leading dimension
  const int vec_ok = (reinterpret_cast<uintptr_t>(C) % 16 == 0) && (ldc % 2 == 0);
  ProfScope prof(family, s, 8.0 * double(M) * double(N) * double(K));
  cgemm_update_tc_ws_kernel<<<grid, WS_THREADS, WS_SMEM, s>>>(M, N, K, static_cast<const float2*>(A), lda,
                                                             static_cast<const float2*>(B), ldb,
                                                             static_cast<float2*>(C), ldc, status, vec_ok);
  return launched();
}

}  // namespace fosb
