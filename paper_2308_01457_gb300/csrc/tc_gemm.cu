// Complex64 rank-k update C -= A B on the 5th-generation tensor cores (tcgen05, TF32),
// with 3xTF32 splitting for FP32-class accuracy: x = x_b + x_s (x_b = tf32(x)), and
//   x y ~ x_b y_b + x_b y_s + x_s y_b.
// Re(C) -= Ar Br - Ai Bi and Im(C) -= Ar Bi + Ai Br give 12 MMAs (M = 128, N = 128,
// K = 8) per k-slab of 8; the minus sign of Ai Bi uses the instruction's negate-A bit.
//
// CTA = 256 threads, output tile 128 x 128 complex; accumulators Re and Im in TMEM
// (128 lanes x 128 fp32 columns each, 256 columns allocated).  K is consumed in chunks of
// 16: the threads load the chunk from global memory (row-major complex64), split it and
// store it in the canonical no-swizzle K-major layout (8 x 16-byte core matrices; LBO =
// 128 B between the two core matrices of a k-slab, SBO = 256 B between 8-row groups); one
// thread issues the MMAs and commits them to an mbarrier; the next chunk overwrites shared
// memory only after that mbarrier completes.  The epilogue moves the accumulators
// TMEM -> registers -> shared memory (padded rows) and updates C with coalesced 16-byte
// read-modify-writes, 64 columns at a time.  Two CTAs per SM (68 KB shared memory each)
// let one CTA's MMAs overlap the other's staging and epilogue.  Every wait is bounded:
// on time-out the status word is set to FOSB_ERR_TIMEOUT, outstanding MMAs get a second
// bounded wait, TMEM is freed and the CTA returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "fosb_internal.h"

namespace fosb {
namespace {

constexpr int TC_M = 128, TC_N = 128, TC_KC = 16;       // tile rows, tile complex columns, k-chunk
constexpr int SLAB = 128 * 8 * 4;                        // bytes per k-slab of one 128-row operand part
constexpr int PART = SLAB * (TC_KC / 8);                 // 8192 bytes per part per chunk
constexpr int SMEM_A = 4 * PART, SMEM_B = 4 * PART;      // parts: re_b, re_s, im_b, im_s
constexpr int EPI_LD = 65;                               // padded float2 row stride of the epilogue tile
constexpr int SMEM_EPI = TC_M * EPI_LD * 8;              // 66560 bytes (aliases the operand buffers)
constexpr int SMEM_BODY = (SMEM_A + SMEM_B) > SMEM_EPI ? (SMEM_A + SMEM_B) : SMEM_EPI;
// 100 KB requested (66.5 KB used + alignment slack) so that at most two CTAs share an SM:
// 2 x 256 TMEM columns fill its 512 exactly and tcgen05.alloc never has to wait.
constexpr int TC_SMEM = 100 * 1024;
static_assert(SMEM_BODY + 1024 <= TC_SMEM, "tile does not fit the shared-memory request");
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

__global__ void __launch_bounds__(256, 2) cgemm_update_tc_kernel(int64_t M, int64_t N, int64_t K, const float2* __restrict__ A,
                                                              int64_t lda, const float2* __restrict__ B, int64_t ldb,
                                                              float2* __restrict__ C, int64_t ldc, int* status,
                                                              int vec_ok) {
  extern __shared__ unsigned char tc_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = smem;           // 4 parts x 2 slabs x 4096
  unsigned char* sB = smem + SMEM_A;  // 4 parts x 2 slabs x 4096
  float2* sE = reinterpret_cast<float2*>(smem);  // epilogue tile (after the last MMA)
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t row0 = int64_t(blockIdx.y) * TC_M, col0 = int64_t(blockIdx.x) * TC_N;
  const uint32_t mbar_addr = smem_u32(&mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_addr));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_sh = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_sh;
  const uint32_t d_re = tmem, d_im = tmem + TC_N;
  uint32_t phase = 0;
  const int64_t nchunk = (K + TC_KC - 1) / TC_KC;
  // Staging maps (per 32-lane group: k3 = lane & 3, rc = lane >> 2): every warp load covers
  // 8 rows x 4 consecutive k (A) or 4 k-rows x 8 consecutive columns (B) -- whole 32-byte
  // sectors -- and the K-major store offsets (rc * 16 + k3 * 4 within a core matrix) hit 32
  // distinct banks.
  const int k3 = lane & 3, rc = lane >> 2;
  float2 va[8], vb[8];
  auto load_chunk = [&](int64_t k0) {
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const int w = warp + 8 * it;                       // 0..63
      const int khi = w & 3, rg = w >> 2;                // A: k-quad, 8-row group
      const int r = rg * 8 + rc, kk = (khi >> 1) * 8 + (khi & 1) * 4 + k3;
      const int64_t gr = row0 + r, gk = k0 + kk;
      va[it] = (gr < M && gk < K) ? A[gr * lda + gk] : make_float2(0.f, 0.f);
      const int cg = w & 15, kb = w >> 4;                // B: 8-column group, k-quad
      const int c = cg * 8 + rc, kkb = (kb >> 1) * 8 + (kb & 1) * 4 + k3;
      const int64_t gc = col0 + c, gkb = k0 + kkb;
      vb[it] = (gc < N && gkb < K) ? B[gkb * ldb + gc] : make_float2(0.f, 0.f);
    }
  };
  if (nchunk > 0) load_chunk(0);
  for (int64_t ch = 0; ch < nchunk; ++ch) {
    // ---- split and store the chunk held in registers (K-major, canonical layout)
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
    asm volatile("fence.proxy.async.shared::cta;");  // generic-proxy stores -> tensor core
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      const uint32_t id = idesc_tf32(TC_M, TC_N, false), idn = idesc_tf32(TC_M, TC_N, true);
#pragma unroll
      for (int s = 0; s < TC_KC / 8; ++s) {
        const uint64_t arb = smem_desc(a0 + 0 * PART + s * SLAB), ars = smem_desc(a0 + 1 * PART + s * SLAB);
        const uint64_t aib = smem_desc(a0 + 2 * PART + s * SLAB), ais = smem_desc(a0 + 3 * PART + s * SLAB);
        const uint64_t brb = smem_desc(b0 + 0 * PART + s * SLAB), brs = smem_desc(b0 + 1 * PART + s * SLAB);
        const uint64_t bib = smem_desc(b0 + 2 * PART + s * SLAB), bis = smem_desc(b0 + 3 * PART + s * SLAB);
        const uint32_t acc0 = (ch > 0 || s > 0) ? 1u : 0u;
        // Re += Ar Br - Ai Bi
        mma_tf32(d_re, arb, brb, id, acc0);
        mma_tf32(d_re, arb, brs, id, 1u);
        mma_tf32(d_re, ars, brb, id, 1u);
        mma_tf32(d_re, aib, bib, idn, 1u);
        mma_tf32(d_re, aib, bis, idn, 1u);
        mma_tf32(d_re, ais, bib, idn, 1u);
        // Im += Ar Bi + Ai Br
        mma_tf32(d_im, arb, bib, id, acc0);
        mma_tf32(d_im, arb, bis, id, 1u);
        mma_tf32(d_im, ars, bib, id, 1u);
        mma_tf32(d_im, aib, brb, id, 1u);
        mma_tf32(d_im, aib, brs, id, 1u);
        mma_tf32(d_im, ais, brb, id, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_addr));
    }
    // the next chunk's global loads are in flight while the MMAs run
    if (ch + 1 < nchunk) load_chunk((ch + 1) * TC_KC);
    // all threads wait for the MMAs (shared memory is reused by the next chunk)
    if (!mbar_wait(mbar_addr, phase)) abort_sh = 1;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (abort_sh) break;
  }
  if (abort_sh) {
    if (tid == 0) {
      atomicExch(status, FOSB_ERR_TIMEOUT);
      mbar_wait(mbar_addr, phase);  // second bounded wait for MMAs still in flight
    }
    __syncthreads();
  } else if (nchunk > 0) {
    // ---- epilogue in two halves of 64 columns: TMEM -> registers -> shared -> C
    const int lane_base = (warp & 3) * 32, csub = (warp >> 2) * 32;
    const int r_local = lane_base + lane;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      uint32_t vr[32], vi[32];
      tmem_ld32(d_re + (uint32_t(lane_base) << 16) + h * 64 + csub, vr);
      tmem_ld32(d_im + (uint32_t(lane_base) << 16) + h * 64 + csub, vi);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int j = 0; j < 32; ++j) sE[r_local * EPI_LD + csub + j] = make_float2(__uint_as_float(vr[j]), __uint_as_float(vi[j]));
      __syncthreads();
      // coalesced update: a warp covers one row's 64 complex (512 B) per pass; all loads
      // are issued before any store
      if (vec_ok) {
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
        float4 o[8];
#pragma unroll
        for (int it = 0; it < 8; ++it) {
          const int e = tid + 256 * (it + 8 * pass);  // 0 .. 4095 pairs of complex
          const int r = e >> 5, c = (e & 31) * 2;
          const int64_t gr = row0 + r, gc = col0 + h * 64 + c;
          o[it] = (gr < M && gc + 1 < N) ? *reinterpret_cast<const float4*>(C + gr * ldc + gc) : make_float4(0, 0, 0, 0);
        }
#pragma unroll
        for (int it = 0; it < 8; ++it) {
          const int e = tid + 256 * (it + 8 * pass);
          const int r = e >> 5, c = (e & 31) * 2;
          const int64_t gr = row0 + r, gc = col0 + h * 64 + c;
          if (gr < M && gc + 1 < N) {
            const float2 d0 = sE[r * EPI_LD + c], d1 = sE[r * EPI_LD + c + 1];
            *reinterpret_cast<float4*>(C + gr * ldc + gc) =
                make_float4(o[it].x - d0.x, o[it].y - d0.y, o[it].z - d1.x, o[it].w - d1.y);
          } else if (gr < M && gc < N) {  // ragged last column
            float2 v = C[gr * ldc + gc];
            const float2 d0 = sE[r * EPI_LD + c];
            C[gr * ldc + gc] = make_float2(v.x - d0.x, v.y - d0.y);
          }
        }
        }
      } else {
#pragma unroll 8
        for (int it = 0; it < 32; ++it) {
          const int e = tid + 256 * it;  // 0 .. 8191
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
      __syncthreads();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

inline unsigned cdiv(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }

}  // namespace

// C (M x N) -= A (M x K) B (K x N), complex64 row-major, on tcgen05 (3xTF32).
cudaError_t cgemm_update_tc(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B, int64_t ldb,
                            void* C, int64_t ldc, int* status, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(cgemm_update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  dim3 grid(cdiv(N, TC_N), cdiv(M, TC_M));
  if (grid.y > 65535u) return cudaErrorInvalidValue;
  // 16-byte epilogue accesses need a 16-byte aligned C with an even leading dimension
  const int vec_ok = (reinterpret_cast<uintptr_t>(C) % 16 == 0) && (ldc % 2 == 0);
  ProfScope prof("lu_update", s, 8.0 * double(M) * double(N) * double(K));
  cgemm_update_tc_kernel<<<grid, 256, TC_SMEM, s>>>(M, N, K, static_cast<const float2*>(A), lda,
                                                   static_cast<const float2*>(B), ldb, static_cast<float2*>(C), ldc,
                                                   status, vec_ok);
  return launched();
}

}  // namespace fosb
