// Tensor memory (TMEM) as per-lane scratch for the paired torque evaluation.
//
// A CTA allocates columns of the SM's tensor memory (128 lanes x 512 columns
// of 32 bits); warp w may access only lane quarter w % 4 (lanes 32 (w % 4)
// .. 32 (w % 4) + 31), so thread t of the warp owns row 32 (w % 4) + t of
// every allocated column.  The paired torque evaluation keeps its per-link
// records there instead of in shared memory: 7 links x 10 float2 = 140
// columns per warp, link j's first 16 words at column 16 j and its last 4 at
// 112 + 4 j, so every access is aligned to its own width.
#pragma once

#include <stdint.h>

#include "fn_arm.cuh"

namespace fn {

#define FN_TM_COLS_PER_WARP 144   // 140 used, rounded to a multiple of 16

// alloc / dealloc are warp-collective: one warp of the CTA calls both
__device__ __forceinline__ void tmem_alloc(uint32_t* s_addr, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(s_addr)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols)
               : "memory");
}
// block-wide barrier that orders tensor-memory accesses around it
__device__ __forceinline__ void tmem_sync_block() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// The stash of torque_at_pair in tensor memory.  Every lane of the warp must
// make each call (the tcgen05 loads and stores are warp-collective).
struct TmemStash {
  uint32_t base;   // lane-quarter row and first column of this warp's block
  __device__ __forceinline__ void store(int j, const float2 (&r)[FN_REC2]) const {
    const uint32_t a = base + 16u * (uint32_t)j, b = base + 112u + 4u * (uint32_t)j;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(a),
        "f"(r[0].x), "f"(r[0].y), "f"(r[1].x), "f"(r[1].y), "f"(r[2].x), "f"(r[2].y),
        "f"(r[3].x), "f"(r[3].y), "f"(r[4].x), "f"(r[4].y), "f"(r[5].x), "f"(r[5].y),
        "f"(r[6].x), "f"(r[6].y), "f"(r[7].x), "f"(r[7].y)
        : "memory");
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};\n" ::"r"(b),
                 "f"(r[8].x), "f"(r[8].y), "f"(r[9].x), "f"(r[9].y)
                 : "memory");
  }
  // the outward pass's stores complete before the inward pass reads them
  __device__ __forceinline__ void stored() const {
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
  }
  __device__ __forceinline__ void load(int j, float2 (&r)[FN_REC2]) const {
    const uint32_t a = base + 16u * (uint32_t)j, b = base + 112u + 4u * (uint32_t)j;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=f"(r[0].x), "=f"(r[0].y), "=f"(r[1].x), "=f"(r[1].y), "=f"(r[2].x), "=f"(r[2].y),
          "=f"(r[3].x), "=f"(r[3].y), "=f"(r[4].x), "=f"(r[4].y), "=f"(r[5].x), "=f"(r[5].y),
          "=f"(r[6].x), "=f"(r[6].y), "=f"(r[7].x), "=f"(r[7].y)
        : "r"(a)
        : "memory");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
                 : "=f"(r[8].x), "=f"(r[8].y), "=f"(r[9].x), "=f"(r[9].y)
                 : "r"(b)
                 : "memory");
    // the registers are defined once the wait returns: pass them through an
    // empty asm that depends on it, so no use is scheduled above the wait
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int k = 0; k < FN_REC2; ++k) asm volatile("" : "+f"(r[k].x), "+f"(r[k].y));
  }
};

}  // namespace fn
