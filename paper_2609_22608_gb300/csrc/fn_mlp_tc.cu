// Fused inference of the duration surrogate on the 5th-generation tensor
// cores: one persistent CTA per SM walks tiles of 128 edges.  Per tile:
//   features (28 scaled boundary-state values, 4 zeros) -> bf16 A operand in
//   shared memory; layer 1 (K = 32) against the resident packed W1;
//   layers 2 and 3 (K = 256) against weight chunks of 64 columns streamed by
//   cp.async.bulk into a 4-deep ring, the accumulator (128 lanes x 256 FP32
//   columns) in tensor memory; after each layer sixteen warps read it back
//   (tcgen05.ld; warp w takes lane quarter w % 4 and 64 of the 256 columns),
//   add the bias, apply ReLU, round to bf16 and write the next A operand;
//   layer 4 (256 -> 2) runs on the CUDA cores in the last epilogue.  Same rounding points as the mma.sync path (bf16
//   operands, FP32 accumulation, bias then ReLU then bf16).
//
// One thread issues the copies and the MMAs; completion is tracked by
// mbarriers (transaction bytes for the copies, tcgen05.commit for the MMAs).
// Every wait is bounded: on a timeout the kernel raises the error flag,
// waits (bounded) for its own copies in flight, frees its tensor memory and
// returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "fn_internal.h"
#include "fn_mlp_tc.h"

namespace fn {

typedef __nv_bfloat16 bf16;

// shared memory map (bytes)
constexpr int kSA = 0;                          // A operand: 128 x 256 bf16 (64 KB)
constexpr int kSB = 65536;                      // weight ring: 4 x 32 KB
constexpr int kSW1 = kSB + 4 * kTcChunkBytes;   // packed W1 (16 KB)
constexpr int kSBias = kSW1 + kTcW1Bytes;       // b1, b2, b3 (3 x 256 f32)
constexpr int kSW4 = kSBias + 3 * 256 * 4;      // W4 [256][2] f32
constexpr int kSBar = kSW4 + 512 * 4;           // mbarriers + TMEM address
constexpr int kSY = kSBar + 128;                // layer-4 partial sums [4][128][2] f32
constexpr int kTcSmem = kSY + 4 * kTcM * 2 * 4;

// 16 warps: warp w reads TMEM lane quarter w % 4 (the tcgen05 access rule)
// and column group w / 4 (64 of the 256 accumulator columns) in the
// epilogues, so that four warps share each scheduler.
constexpr int kTcThreads = 512;

constexpr int kRing = 4;
constexpr int kTmemCols = 256;
constexpr long long kWaitCycles = 2000000000LL;   // ~1 s at 2 GHz

// instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator,
// bf16 A and B, both K-major, N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: canonical K-major layout without swizzle
// (start, leading = K-adjacent core matrices, stride = 8-row groups)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version
  return d;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for phase `parity` of the barrier to complete
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void proxy_fence() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const bf16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// weights [K][256] bf16 -> packed chunks of Kt columns
__global__ void k_mlp_tc_pack(const bf16* __restrict__ W, int K, int Kt, bf16* __restrict__ out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)K * kTcN) return;
  const int k = (int)(i / kTcN), n = (int)(i - (long)k * kTcN);
  const int c = k / Kt, kk = k - c * Kt;
  const long off = (long)c * kTcN * Kt +
                   ((long)((n >> 3) * (Kt >> 3) + (kk >> 3)) * 128 + (n & 7) * 16 + (kk & 7) * 2) / 2;
  out[off] = W[i];
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_mlp_tc(ArmK A, const float* __restrict__ s0, const float* __restrict__ s1, int E,
             const bf16* __restrict__ W1p, const bf16* __restrict__ W23p,
             const float* __restrict__ b1, const float* __restrict__ b2,
             const float* __restrict__ b3, const bf16* __restrict__ W4b,
             const float* __restrict__ b4, float* __restrict__ Y, int* __restrict__ err,
             const int* __restrict__ E_dev) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int lq = warp & 3, cg = warp >> 2;          // TMEM lane quarter, column group
  const int trow = lq * 32 + (tid & 31);            // this thread's row of the tile
  if (E_dev) E = min(E, *E_dev);   // rows counted on the device (at most the launch's E)
  const int ntiles = (E + kTcM - 1) / kTcM;
  if ((int)blockIdx.x >= ntiles) return;   // block-uniform, before any barrier
  const int my_tiles = (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1;
  uint8_t* sA = smem + kSA;
  float* sBias = reinterpret_cast<float*>(smem + kSBias);
  float* sW4 = reinterpret_cast<float*>(smem + kSW4);
  float* sY = reinterpret_cast<float*>(smem + kSY);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kSBar);
  // bars[0..3] chunk arrived, bars[4..7] chunk consumed, bars[8] layer done, bars[9] W1 arrived
  volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(smem + kSBar + 80);
  volatile int* s_fail = reinterpret_cast<volatile int*>(smem + kSBar + 84);
  const uint32_t a_base = su32(sA), b_base = su32(smem + kSB), w1_base = su32(smem + kSW1);
  const uint32_t bar_base = su32(bars);
  auto bar_w = [&](int b) { return bar_base + 8u * b; };
  auto bar_free = [&](int b) { return bar_base + 8u * (4 + b); };
  const uint32_t bar_layer = bar_base + 64u, bar_w1 = bar_base + 72u;

  for (int i = tid; i < 768; i += blockDim.x)
    sBias[i] = i < 256 ? b1[i] : (i < 512 ? b2[i - 256] : b3[i - 512]);
  for (int i = tid; i < 512; i += blockDim.x) sW4[i] = __bfloat162float(W4b[i]);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     su32((const void*)s_tmem)),
                 "r"((uint32_t)kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int b = 0; b < 10; ++b) mbar_init(bar_base + 8u * b, 1);
    *s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t tmem_lane = tmem + ((uint32_t)(lq * 32) << 16);   // this warp's 32 lanes

  const long total = (long)my_tiles * 8;   // streamed chunks (layers 2 and 3 of every tile)
  int issued[kRing] = {0, 0, 0, 0};        // thread 0: copies in flight per slot
  uint32_t ph_w[kRing] = {0, 0, 0, 0}, ph_free[kRing] = {0, 0, 0, 0};
  uint32_t ph_layer = 0;
  long g = 0;                              // next chunk to multiply (thread 0)
  bool fail = false;
  if (tid == 0) {
    mbar_expect_tx(bar_w1, kTcW1Bytes);
    bulk_g2s(w1_base, W1p, kTcW1Bytes, bar_w1);
    for (int c = 0; c < kRing && c < total; ++c) {
      mbar_expect_tx(bar_w(c), kTcChunkBytes);
      bulk_g2s(b_base + c * kTcChunkBytes, W23p + (long)(c % 8) * (kTcChunkBytes / 2),
               kTcChunkBytes, bar_w(c));
      issued[c] = 1;
    }
  }

  for (int it = 0; it < my_tiles; ++it) {
    const long row = ((long)blockIdx.x + (long)it * gridDim.x) * kTcM + trow;
    // ---- features -> A (K = 32 layout: 4 core matrices per 8-row group):
    // warps 0-3, whose thread tid owns row tid (= trow)
    if (tid < kTcM) {
      float f[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) f[j] = 0.f;
      if (row < E) {
        const float* p0 = s0 + 16 * row;
        const float* p1 = s1 + 16 * row;
#pragma unroll
        for (int j = 0; j < 7; ++j) {
          const float c = 0.5f * (A.q_lo[j] + A.q_hi[j]);
          const float h = 0.5f * (A.q_hi[j] - A.q_lo[j]);
          f[j] = (p0[j] - c) / h;
          f[7 + j] = p0[8 + j] / A.qd_max[j];
          f[14 + j] = (p1[j] - c) / h;
          f[21 + j] = p1[8 + j] / A.qd_max[j];
        }
      }
#pragma unroll
      for (int kb = 0; kb < 4; ++kb) {
        uint4 v;
        v.x = pack_bf16x2(f[8 * kb + 0], f[8 * kb + 1]);
        v.y = pack_bf16x2(f[8 * kb + 2], f[8 * kb + 3]);
        v.z = pack_bf16x2(f[8 * kb + 4], f[8 * kb + 5]);
        v.w = pack_bf16x2(f[8 * kb + 6], f[8 * kb + 7]);
        *reinterpret_cast<uint4*>(sA + ((tid >> 3) * 4 + kb) * 128 + (tid & 7) * 16) = v;
      }
    }
    proxy_fence();
    __syncthreads();
    // ---- layer 1
    if (tid == 0 && !fail) {
      tc_fence_after();
      if (it == 0 && !mbar_wait(bar_w1, 0)) fail = true;
      if (!fail) {
#pragma unroll
        for (int s = 0; s < kTcK1 / 16; ++s)
          umma(tmem, sdesc(a_base + s * 256, 128, kTcK1 * 16), sdesc(w1_base + s * 256, 128, kTcK1 * 16),
               s > 0);
        umma_commit(bar_layer);
      }
    }
    for (int layer = 0; layer < 3; ++layer) {
      if (tid == 0 && fail) *s_fail = 1;
      __syncthreads();
      // wait for this layer's accumulator (all threads; a block vote keeps
      // the decision uniform, so no thread is left at a barrier)
      const bool lf = *s_fail || !mbar_wait(bar_layer, ph_layer);
      ph_layer ^= 1;
      tc_fence_after();
      if (__syncthreads_or(lf)) {
        *s_fail = 1;
        break;
      }
      const float* bias = sBias + 256 * layer;
      if (layer < 2) {
        // epilogue: bias, ReLU, bf16 -> A (K = 256 layout: 32 core matrices per
        // 8-row group); this warp's two 32-column blocks of its 32 rows
#pragma unroll 1
        for (int cb = 2 * cg; cb < 2 * cg + 2; ++cb) {
          uint32_t v[32];
          tmem_ld32(tmem_lane + cb * 32, v);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float x[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
              x[j] = fmaxf(__uint_as_float(v[8 * q + j]) + bias[cb * 32 + 8 * q + j], 0.f);
            uint4 o;
            o.x = pack_bf16x2(x[0], x[1]);
            o.y = pack_bf16x2(x[2], x[3]);
            o.z = pack_bf16x2(x[4], x[5]);
            o.w = pack_bf16x2(x[6], x[7]);
            *reinterpret_cast<uint4*>(sA + ((trow >> 3) * 32 + cb * 4 + q) * 128 + (trow & 7) * 16) = o;
          }
        }
        tc_fence_before();
        proxy_fence();
        __syncthreads();
        // ---- layers 2, 3: four streamed chunks of 64 K columns each
        if (tid == 0 && !fail) {
          tc_fence_after();
          for (int c = 0; c < 4 && !fail; ++c, ++g) {
            const int b = (int)(g % kRing);
            if (!mbar_wait(bar_w(b), ph_w[b])) { fail = true; break; }
            ph_w[b] ^= 1;
            issued[b] = 0;
            const uint32_t bb = b_base + b * kTcChunkBytes;
#pragma unroll
            for (int s = 0; s < kTcKc / 16; ++s)
              umma(tmem, sdesc(a_base + (4 * c + s) * 256, 128, 256 * 16), sdesc(bb + s * 256, 128, kTcKc * 16),
                   (c | s) != 0);
            umma_commit(bar_free(b));
            // refill the slot of the previous chunk (its MMAs are queued before
            // this chunk's) with the chunk RING - 1 ahead of this one
            if (g >= 1 && g + kRing - 1 < total) {
              const int pb = (int)((g - 1) % kRing);
              if (!mbar_wait(bar_free(pb), ph_free[pb])) { fail = true; break; }
              ph_free[pb] ^= 1;
              const long nc = g + kRing - 1;
              mbar_expect_tx(bar_w(pb), kTcChunkBytes);
              bulk_g2s(b_base + pb * kTcChunkBytes, W23p + (nc % 8) * (kTcChunkBytes / 2),
                       kTcChunkBytes, bar_w(pb));
              issued[pb] = 1;
            }
          }
          if (!fail) umma_commit(bar_layer);
          else *s_fail = 1;
        }
        __syncthreads();
      } else {
        // last epilogue: h3 = bf16(ReLU(acc + b3)); y = h3 W4 + b4 on the CUDA
        // cores, each warp over its 64 columns, the four groups summed in order
        float y0 = 0.f, y1 = 0.f;
#pragma unroll 1
        for (int cb = 2 * cg; cb < 2 * cg + 2; ++cb) {
          uint32_t v[32];
          tmem_ld32(tmem_lane + cb * 32, v);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int k = cb * 32 + j;
            const float h = __bfloat162float(
                __float2bfloat16_rn(fmaxf(__uint_as_float(v[j]) + bias[k], 0.f)));
            y0 = fmaf(h, sW4[2 * k], y0);
            y1 = fmaf(h, sW4[2 * k + 1], y1);
          }
        }
        sY[(cg * kTcM + trow) * 2] = y0;
        sY[(cg * kTcM + trow) * 2 + 1] = y1;
        tc_fence_before();
        __syncthreads();
        if (cg == 0 && row < E) {
          float z0 = 0.f, z1 = 0.f;
#pragma unroll
          for (int g2 = 0; g2 < 4; ++g2) {
            z0 += sY[(g2 * kTcM + trow) * 2];
            z1 += sY[(g2 * kTcM + trow) * 2 + 1];
          }
          Y[2 * row] = z0 + b4[0];
          Y[2 * row + 1] = z1 + b4[1];
        }
        __syncthreads();
      }
    }
    if (*s_fail) break;
  }
  // ---- exit: on failure, wait (bounded) for this CTA's copies still in flight
  __syncthreads();
  if (*s_fail || fail) {
    if (tid == 0) {
      atomicExch(err, 1);
      for (int b = 0; b < kRing; ++b)
        if (issued[b]) mbar_wait(bar_w(b), ph_w[b]);
    }
    __syncthreads();
  }
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"((uint32_t)kTmemCols)
                 : "memory");
}

// ---------------------------------------------------------------------------
// General BF16 GEMM on the tensor cores for the surrogate's training:
//   C[M][N] = op(A)[M][K] op(B)[K][N] (+ bias, ReLU), FP32 accumulation in
//   tensor memory; op(A) = A [M][K] (row-major, lda) or, TA, A^T with A
//   [K][M]; op(B) = B [K][N] or, TB, B^T with B [N][K].
// A CTA computes a 128 x 128 tile over the K range of its grid z slice:
// 128 threads stage 64-column K chunks of both operands into shared memory
// in the canonical K-major layout with 16-byte loads (stage_tile), two
// stages deep; one thread issues four tcgen05.mma (K = 16) per chunk and commits
// them to the stage's barrier; the epilogue reads the accumulator back
// (warp w: lanes 32w..32w+31) and stores FP32 and / or BF16, or adds FP32
// partial sums atomically when the K range is split.  Waits are bounded as
// in the fused forward.
// ---------------------------------------------------------------------------
constexpr int kGM = 128, kGN = 128, kGK = 64;
constexpr int kGTile = kGM * kGK * 2;               // 16 KB per operand tile
constexpr int kGStage = 2 * kGTile;                 // A and B
constexpr int kGScrW = kGM + 8;                     // transpose scratch row (bf16), padded
constexpr int kGScr = kGK * kGScrW * 2;             // 17 KB
constexpr int kGSmem = 2 * kGStage + kGScr + 64;    // two stages, scratch, barriers
constexpr uint32_t kGIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                             ((uint32_t)(kGN >> 3) << 17) | ((uint32_t)(kGM >> 4) << 24);

__device__ __forceinline__ void umma_g(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kGIdesc), "r"(acc)
      : "memory");
}

// byte offset of element (row, k) of a 128 x 64 tile in the canonical
// K-major layout: 8 x 8 core matrices of 128 B, K-adjacent ones 128 B apart,
// 8-row groups 1024 B apart
__device__ __forceinline__ int g_off(int row, int k) {
  return ((row >> 3) * (kGK / 8) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Stage one 128 x 64 operand tile (rows r0.., columns kc..) into the
// canonical layout at dst.  KC: the source is contiguous along K (element
// (r, k) at src[r * ld + k]): 16-byte vectors are whole core-matrix rows.
// Otherwise (element (r, k) at src[k * ld + r]) 16-byte vectors along r go
// to a padded row-major scratch, and each thread then gathers 8 K values of
// one row into a 16-byte store.  Elements past R rows or k1 columns are 0.
// Rows of 8 elements must be 16-byte aligned (ld % 8 == 0, aligned base).
template <bool KC>
__device__ __forceinline__ void stage_tile(uint8_t* dst, const bf16* __restrict__ src, int ld,
                                           int r0, int R, int kc, int k1, bf16* scr, int tid) {
  constexpr int kPer = kGM * (kGK / 8) / 128;   // 16-byte vectors per thread (8)
  uint4 x[kPer];
  // all loads first, so that the eight are in flight together
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int v = tid + 128 * i;
    int gr, gk, lim;   // the vector's first element and its extent along the contiguous index
    if (KC) {
      gr = r0 + (v >> 3);
      gk = kc + (v & 7) * 8;
    } else {
      gk = kc + (v >> 4);
      gr = r0 + (v & 15) * 8;
    }
    x[i] = make_uint4(0u, 0u, 0u, 0u);
    if (gr < R && gk < k1) {
      const bf16* p = KC ? src + (long)gr * ld + gk : src + (long)gk * ld + gr;
      lim = KC ? k1 - gk : R - gr;
      if (lim >= 8) {
        x[i] = *reinterpret_cast<const uint4*>(p);
      } else {
        alignas(16) bf16 e[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) e[j] = j < lim ? p[j] : __float2bfloat16_rn(0.f);
        x[i] = *reinterpret_cast<const uint4*>(e);
      }
    }
  }
  if (KC) {
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int v = tid + 128 * i;
      *reinterpret_cast<uint4*>(dst + g_off(v >> 3, (v & 7) * 8)) = x[i];
    }
  } else {
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int v = tid + 128 * i;
      *reinterpret_cast<uint4*>(scr + (v >> 4) * kGScrW + (v & 15) * 8) = x[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int v = tid + 128 * i;
      const int r = v & (kGM - 1), k = (v >> 7) * 8;
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        w[q] = (uint32_t)__bfloat16_as_ushort(scr[(k + 2 * q) * kGScrW + r]) |
               ((uint32_t)__bfloat16_as_ushort(scr[(k + 2 * q + 1) * kGScrW + r]) << 16);
      *reinterpret_cast<uint4*>(dst + g_off(r, k)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    __syncthreads();   // the scratch is reused by the next tile
  }
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128, 1)
    k_gemm_tc(int M, int N, int K, int kslice, const bf16* __restrict__ A, int lda,
              const bf16* __restrict__ B, int ldb, const float* __restrict__ bias, int relu,
              int accumulate, int atomic, float* __restrict__ Cf, int ldcf, bf16* __restrict__ Cb,
              int ldcb, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kGM, n0 = blockIdx.x * kGN;
  const int k0 = blockIdx.z * kslice, k1 = min(K, k0 + kslice);
  if (k0 >= k1) return;                              // block-uniform, before any barrier
  bf16* scr = reinterpret_cast<bf16*>(smem + 2 * kGStage);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * kGStage + kGScr);
  volatile uint32_t* s_tmem = reinterpret_cast<volatile uint32_t*>(smem + 2 * kGStage + kGScr + 32);
  volatile int* s_fail = reinterpret_cast<volatile int*>(smem + 2 * kGStage + kGScr + 36);
  const uint32_t base = su32(smem), bar0 = su32(bars);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     su32((const void*)s_tmem)),
                 "r"((uint32_t)kGN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8, 1);
    *s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const bf16 zero = __float2bfloat16_rn(0.f);
  const int nk = (k1 - k0 + kGK - 1) / kGK;
  for (int c = 0; c < nk; ++c) {
    const int st = c & 1;
    // the MMAs that read this stage two chunks ago must be done (a block
    // vote keeps the decision uniform, so no thread is left at a barrier)
    const bool f = c >= 2 && !mbar_wait(bar0 + 8 * st, ((c - 2) >> 1) & 1);
    if (__syncthreads_or(f)) {
      *s_fail = 1;
      break;
    }
    uint8_t* sa = smem + st * kGStage;
    uint8_t* sb = sa + kGTile;
    const int kc = k0 + c * kGK;
    stage_tile<!TA>(sa, A, lda, m0, M, kc, k1, scr, tid);   // (m, k)
    stage_tile<TB>(sb, B, ldb, n0, N, kc, k1, scr, tid);    // (n, k)
    proxy_fence();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a = base + st * kGStage, b = a + kGTile;
#pragma unroll
      for (int j = 0; j < kGK / 16; ++j)
        umma_g(tmem, sdesc(a + j * 256, 128, (kGK / 8) * 128), sdesc(b + j * 256, 128, (kGK / 8) * 128),
               (c | j) != 0);
      umma_commit(bar0 + 8 * st);
    }
  }
  // the last chunk's MMAs (every earlier one completes before it)
  const int last = nk - 1;
  const bool bad = *s_fail || !mbar_wait(bar0 + 8 * (last & 1), (last >> 1) & 1);
  if (__syncthreads_or(bad)) *s_fail = 1;
  tc_fence_after();
  if (!*s_fail) {
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int cb = 0; cb < kGN / 32; ++cb) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + cb * 32, v);
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = n0 + cb * 32 + j;
          if (col >= N) continue;
          float x = __uint_as_float(v[j]) + (bias ? bias[col] : 0.f);
          if (relu) x = fmaxf(x, 0.f);
          if (Cf) {
            float* o = Cf + (long)row * ldcf + col;
            if (atomic) atomicAdd(o, x);
            else *o = accumulate ? *o + x : x;
          }
          if (Cb) Cb[(long)row * ldcb + col] = __float2bfloat16_rn(x);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*s_fail && tid == 0) atomicExch(err, 1);
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"((uint32_t)kGN)
                 : "memory");
}

template <bool TA, bool TB>
void gemm_tc(int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb,
             const float* bias, bool relu, bool accumulate, float* Cf, int ldcf, bf16* Cb,
             int ldcb, int* err, cudaStream_t st) {
  static bool attr[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    cudaFuncSetAttribute(k_gemm_tc<TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmem);
    attr[dev] = true;
  }
  const int gx = (N + kGN - 1) / kGN, gy = (M + kGM - 1) / kGM;
  // split a long K over the grid's z so that every SM gets a CTA; the
  // slices add FP32 partial sums atomically into a zeroed C
  int slices = 1;
  const int want = num_sms() / std::max(1, gx * gy);
  if (want > 1 && K > 8 * kGK && !Cb && Cf && !bias && !relu) {
    slices = std::min(want, (K + 4 * kGK - 1) / (4 * kGK));
    if (slices > 1 && !accumulate) {
      if (ldcf == N)
        cudaMemsetAsync(Cf, 0, sizeof(float) * (size_t)M * N, st);
      else
        for (int r = 0; r < M; ++r) cudaMemsetAsync(Cf + (long)r * ldcf, 0, sizeof(float) * N, st);
    }
  }
  const int kslice = slices > 1 ? ((K + slices - 1) / slices + kGK - 1) / kGK * kGK : K;
  slices = (K + kslice - 1) / kslice;
  k_gemm_tc<TA, TB><<<dim3(gx, gy, slices), 128, kGSmem, st>>>(
      M, N, K, kslice, A, lda, B, ldb, bias, relu ? 1 : 0, accumulate ? 1 : 0, slices > 1 ? 1 : 0,
      Cf, ldcf, Cb, ldcb, err);
}

template void gemm_tc<false, false>(int, int, int, const bf16*, int, const bf16*, int, const float*,
                                    bool, bool, float*, int, bf16*, int, int*, cudaStream_t);
template void gemm_tc<true, false>(int, int, int, const bf16*, int, const bf16*, int, const float*,
                                   bool, bool, float*, int, bf16*, int, int*, cudaStream_t);
template void gemm_tc<false, true>(int, int, int, const bf16*, int, const bf16*, int, const float*,
                                   bool, bool, float*, int, bf16*, int, int*, cudaStream_t);

void mlp_tc_pack(const bf16* W, int K, int Kt, bf16* out, cudaStream_t st) {
  const long n = (long)K * kTcN;
  k_mlp_tc_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(W, K, Kt, out);
}

fn_status mlp_tc_forward(const ArmK& A, const float* s0, const float* s1, int E, const bf16* W1p,
                         const bf16* W23p, const float* b1, const float* b2, const float* b3,
                         const bf16* W4b, const float* b4, float* Y, int* err, cudaStream_t st,
                         const int* E_dev) {
  if (E <= 0) return FN_OK;
  static bool attr[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    if (cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem) !=
        cudaSuccess)
      return FN_ECUDA;
    attr[dev] = true;
  }
  const int ntiles = (E + kTcM - 1) / kTcM;
  const int grid = ntiles < num_sms() ? ntiles : num_sms();
  k_mlp_tc<<<grid, kTcThreads, kTcSmem, st>>>(A, s0, s1, E, W1p, W23p, b1, b2, b3, W4b, b4, Y,
                                               err, E_dev);
  return launch_status();
}

}  // namespace fn
