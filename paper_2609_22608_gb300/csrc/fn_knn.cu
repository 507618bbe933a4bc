// Parents of Algorithm 1 (Sec. IV-E): brute-force parallel scan of the tree
// for each query's k nearest nodes under the velocity-weighted squared joint
// distance, ties broken by the lower node index.
//
// Layout: one thread per query, 128 queries per block; the block streams its
// slice of the tree through shared memory in tiles of 128 nodes (8 KB), so
// every node is read from L2 once per block and then broadcast from shared
// memory to all 128 queries.  Each thread keeps a sorted top-KM list
// (KM = 8 or 16) in registers.  The node range is split over `nsplit` blocks
// per query tile to fill the GPU; partial lists go to the caller's workspace
// and a second kernel merges them.
#include <cuda_runtime.h>

#include "fn_internal.h"
#include "knn_core.cuh"

namespace fn {

template <int KM>
__global__ void __launch_bounds__(128) k_knn_partial(const float4* __restrict__ tree, int N,
                                                     int first, const float4* __restrict__ queries,
                                                     int B, float w_vel, int nsplit, int k,
                                                     float* __restrict__ part_d,
                                                     int32_t* __restrict__ part_i,
                                                     float* __restrict__ out_d,
                                                     int32_t* __restrict__ out_i) {
  __shared__ float4 tile[KNN_TILE * 4];
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int split = blockIdx.y;
  const int span = N - first;
  const int per = (span + nsplit - 1) / nsplit;
  const int lo = first + split * per;
  const int hi = min(N, lo + per);
  TopK<KM> top;
  top.init();
  float qv[14];
  const bool active = b < B;
  if (active) load_query(queries + 4 * (long)b, qv);
  else
    for (int j = 0; j < 14; ++j) qv[j] = 0.f;
  knn_scan_range<KM>(tree, lo, hi, qv, w_vel, top, tile);
  if (!active) return;
  if (nsplit == 1) {
    top.store(out_d + (long)b * k, out_i + (long)b * k, k);
  } else {
    const long off = ((long)split * B + b) * KM;
    top.store(part_d + off, part_i + off, KM);
  }
}

// Merge of the split lists with one warp per query: lane l holds split l's
// sorted list; k rounds of a warp-wide (d, index) argmin over the list heads,
// the winning lane drops its head.
template <int KM>
__global__ void __launch_bounds__(256) k_knn_merge(int B, int nsplit, int k,
                                                   const float* __restrict__ part_d,
                                                   const int32_t* __restrict__ part_i,
                                                   float* __restrict__ out_d,
                                                   int32_t* __restrict__ out_i) {
  const int lane = threadIdx.x & 31;
  const long b = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= B) return;
  float d[KM];
  int id[KM];
#pragma unroll
  for (int j = 0; j < KM; ++j) {
    d[j] = INFINITY;
    id[j] = 0x7fffffff;
  }
  if (lane < nsplit) {
    const long off = ((long)lane * B + b) * KM;
#pragma unroll
    for (int j = 0; j < KM; ++j) {
      d[j] = part_d[off + j];
      id[j] = part_i[off + j];
    }
  }
  for (int r = 0; r < k; ++r) {
    float md = d[0];
    int mi = id[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float od = __shfl_xor_sync(0xffffffffu, md, o);
      const int oi = __shfl_xor_sync(0xffffffffu, mi, o);
      if (knn_less(od, oi, md, mi)) { md = od; mi = oi; }
    }
    if (lane == 0) {
      const bool empty = (mi == 0x7fffffff);
      out_d[b * k + r] = empty ? INFINITY : md;
      out_i[b * k + r] = empty ? -1 : mi;
    }
    if (id[0] == mi && mi != 0x7fffffff) {  // the winner drops its head
#pragma unroll
      for (int j = 0; j + 1 < KM; ++j) {
        d[j] = d[j + 1];
        id[j] = id[j + 1];
      }
      d[KM - 1] = INFINITY;
      id[KM - 1] = 0x7fffffff;
    }
  }
}

int knn_km(int k) { return k <= 8 ? 8 : 16; }

// split count: about two blocks per SM, each split at least 4 tiles of
// nodes, at most 32 (one merge lane per split)
int knn_nsplit(int B, int N) {
  const int qblocks = (B + 127) / 128;
  const int want = (2 * num_sms() + qblocks - 1) / std::max(qblocks, 1);
  const int chunks = std::max(1, N / (4 * KNN_TILE));
  return std::max(1, std::min(std::min(want, chunks), 32));
}

size_t knn_ws_bytes(int B, int N, int k) {
  if (B <= 0 || N <= 0 || k < 1 || k > FN_MAX_KNN) return 0;
  const int ns = knn_nsplit(B, N);
  if (ns <= 1) return 0;
  const size_t per = (size_t)ns * B * knn_km(k);
  const size_t a = (per * sizeof(float) + 255) & ~(size_t)255;
  return a + per * sizeof(int32_t);
}

fn_status knn_launch(const float* tree, int N, int first, const float* queries, int B, int k,
                     float w_vel, int32_t* idx, float* d2, int nsplit, float* part_d,
                     int32_t* part_i, cudaStream_t st) {
  dim3 grid((B + 127) / 128, nsplit);
  if (knn_km(k) == 8) {
    k_knn_partial<8><<<grid, 128, 0, st>>>((const float4*)tree, N, first, (const float4*)queries,
                                           B, w_vel, nsplit, k, part_d, part_i, d2, idx);
    if (nsplit > 1)
      k_knn_merge<8><<<(B + 7) / 8, 256, 0, st>>>(B, nsplit, k, part_d, part_i, d2, idx);
  } else {
    k_knn_partial<16><<<grid, 128, 0, st>>>((const float4*)tree, N, first, (const float4*)queries,
                                            B, w_vel, nsplit, k, part_d, part_i, d2, idx);
    if (nsplit > 1)
      k_knn_merge<16><<<(B + 7) / 8, 256, 0, st>>>(B, nsplit, k, part_d, part_i, d2, idx);
  }
  return launch_status();
}

}  // namespace fn

using namespace fn;

extern "C" size_t fn_knn_workspace_bytes(int B, int N, int k) { return knn_ws_bytes(B, N, k); }

extern "C" fn_status fn_knn_tree(const float* tree, int N, int first, const float* queries, int B,
                                 int k, float w_vel, int32_t* idx, float* d2, void* workspace,
                                 size_t workspace_bytes, void* stream) {
  if (N < 0 || first < 0 || first > N || B < 0 || k < 1 || k > FN_MAX_KNN) return FN_EINVAL;
  if (!(w_vel >= 0.f) || !std::isfinite(w_vel)) return FN_EINVAL;
  if (B == 0) return FN_OK;
  if (!queries || !idx || !d2 || !aligned16(queries)) return FN_EINVAL;
  if (N > first && (!tree || !aligned16(tree))) return FN_EINVAL;
  int nsplit = 1;
  float* part_d = nullptr;
  int32_t* part_i = nullptr;
  const size_t need = knn_ws_bytes(B, N, k);
  if (workspace && need > 0) {
    if (workspace_bytes < need || !aligned256(workspace)) return FN_EINVAL;
    nsplit = knn_nsplit(B, N);
    const size_t per = (size_t)nsplit * B * knn_km(k);
    part_d = (float*)workspace;
    part_i = (int32_t*)((char*)workspace + ((per * sizeof(float) + 255) & ~(size_t)255));
  }
  return knn_launch(tree, N, first, queries, B, k, w_vel, idx, d2, nsplit, part_d, part_i,
                    (cudaStream_t)stream);
}
