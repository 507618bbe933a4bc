// Block layout of the paired edge scan with its per-link records in tensor
// memory (PairCore<TmemStash>), shared by the standalone edge-timing kernels
// and the planner's warp-per-edge edge body.
//
// One CTA of TM_WARPS = 12 warps per SM holds all 512 tensor-memory columns;
// warp w uses lane quarter w % 4 and the 144-column block 144 (w / 4) (three
// warps per quarter).  A warp works on runs of up to TM_GROUP edges: it
// stages a run, computes the end-sample splits of the whole run in one pass
// (split_group) and then scans the edges one by one.  The coefficients,
// staged edges, splits, the paired link table and the duration grid sit in
// dynamic shared memory, sized above half of the SM's so that no second CTA
// (which would wait for the columns) is placed on the SM.
#pragma once

#include <stdint.h>

#include "edge_core.cuh"
#include "fn_tmem.cuh"

namespace fn {

#define TM_WARPS 12
#define TM_GROUP 10
constexpr int kTmCols = 512;
constexpr size_t kTmCoef = (size_t)TM_WARPS * FN_CUBIC_WORDS * 32 * sizeof(float2);
constexpr size_t kTmEdge = (size_t)TM_WARPS * TM_GROUP * 32 * sizeof(float);
constexpr size_t kTmSplit = (size_t)TM_WARPS * TM_GROUP * FN_SPLIT_WORDS * sizeof(float);
constexpr size_t kTmLink = 7 * FN_LINK2_F4 * sizeof(float4);
constexpr size_t kTmGrid = FN_MAX_GRID * sizeof(float);
constexpr size_t kTmUsed = kTmCoef + kTmEdge + kTmSplit + kTmLink + kTmGrid + 16;   // + 4 words
constexpr size_t kTmSmem = 140 * 1024;
static_assert(kTmUsed <= kTmSmem, "tensor-memory scan: shared-memory layout");
static_assert(2 * (kTmSmem + 1024) > 233472, "one CTA per SM");
static_assert(kTmCoef % 16 == 0 && kTmEdge % 16 == 0 && kTmSplit % 16 == 0, "16-byte carve");
static_assert(FN_SPLIT_WORDS * sizeof(float) % 16 == 0, "16-byte split slots");
static_assert(TM_GROUP <= 10, "split_group takes at most ten edges");
static_assert(3 * FN_TM_COLS_PER_WARP <= kTmCols, "three warps per lane quarter");

// The CTA's carve of its dynamic shared memory and the calling warp's slots.
struct TmBlock {
  float2* coef;     // [TM_WARPS][FN_CUBIC_WORDS][32] paired coefficients
  float* edge;      // [TM_WARPS][TM_GROUP][32] staged edges
  float* split;     // [TM_WARPS][TM_GROUP][FN_SPLIT_WORDS] end-sample splits
  float4* link;     // [7][FN_LINK2_F4] paired link table
  float* grid;      // [FN_MAX_GRID] durations
  uint32_t* tmem;   // the allocation's base address
  int* next;        // the CTA's run counter
  int* aux;         // two words free for the kernel
  __device__ explicit TmBlock(void* smem) {
    char* b = reinterpret_cast<char*>(smem);
    coef = reinterpret_cast<float2*>(b);
    edge = reinterpret_cast<float*>(b + kTmCoef);
    split = reinterpret_cast<float*>(b + kTmCoef + kTmEdge);
    link = reinterpret_cast<float4*>(b + kTmCoef + kTmEdge + kTmSplit);
    grid = reinterpret_cast<float*>(b + kTmCoef + kTmEdge + kTmSplit + kTmLink);
    tmem = reinterpret_cast<uint32_t*>(b + kTmCoef + kTmEdge + kTmSplit + kTmLink + kTmGrid);
    next = reinterpret_cast<int*>(tmem + 1);
    aux = reinterpret_cast<int*>(tmem + 2);
  }
  __device__ float* edges_of(int w) const { return edge + TM_GROUP * 32 * w; }
  __device__ float* splits_of(int w) const { return split + TM_GROUP * FN_SPLIT_WORDS * w; }
  // warp w's core: its coefficient column and its tensor-memory block
  __device__ PairCore<TmemStash> core(uint32_t taddr, int w, int lane) const {
    return PairCore<TmemStash>{
        LinkTab2{link}, CubicLane2{coef + w * FN_CUBIC_WORDS * 32 + lane},
        TmemStash{taddr + ((uint32_t)((w & 3) * 32) << 16) +
                  FN_TM_COLS_PER_WARP * (uint32_t)(w >> 2)}};
  }
};

// Claim of a run by a warp of the CTA whose range holds `len` items: about
// (range left) / (2 TM_WARPS) items, at least two and at most TM_GROUP, so
// that runs shrink towards the end of the range and the warps finish
// together.  Returns the run's first item (relative to the range) and its
// length n (0: the range is done), the same on every lane.
__device__ __forceinline__ int tm_claim(int* next, int len, int& n) {
  const int lane = threadIdx.x & 31;
  int first = 0;
  n = 0;
  if (lane == 0) {
    const int seen = atomicAdd(next, 0);
    const int want = min(TM_GROUP, max(2, (len - seen) / (2 * TM_WARPS)));
    first = atomicAdd(next, want);
    n = max(0, min(want, len - first));
  }
  first = __shfl_sync(0xffffffffu, first, 0);
  n = __shfl_sync(0xffffffffu, n, 0);
  return first;
}

}  // namespace fn
