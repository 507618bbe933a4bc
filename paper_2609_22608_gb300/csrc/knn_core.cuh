// Register top-k list and the shared-memory tile scan of the nearest-parent
// search (Sec. IV-E "Parents": brute-force parallel scan).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define KNN_TILE 128

namespace fn {

// (d, i) < (d', i') lexicographically: nearer first, then lower node index
__device__ __forceinline__ bool knn_less(float d, int i, float d2, int i2) {
  return d < d2 || (d == d2 && i < i2);
}

template <int KM>
struct TopK {
  float d[KM];
  int i[KM];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int j = 0; j < KM; ++j) {
      d[j] = INFINITY;
      i[j] = 0x7fffffff;
    }
  }
  // insert keeping (d, i) ascending; the candidate bubbles through the list
  __device__ __forceinline__ void push(float cd, int ci) {
    if (!knn_less(cd, ci, d[KM - 1], i[KM - 1])) return;
#pragma unroll
    for (int j = 0; j < KM; ++j) {
      const bool sw = knn_less(cd, ci, d[j], i[j]);
      const float td = d[j];
      const int ti = i[j];
      d[j] = sw ? cd : td;
      i[j] = sw ? ci : ti;
      cd = sw ? td : cd;
      ci = sw ? ti : ci;
    }
  }
  __device__ __forceinline__ void store(float* od, int32_t* oi, int k) const {
#pragma unroll
    for (int j = 0; j < KM; ++j) {
      if (j < k) {
        const bool empty = (i[j] == 0x7fffffff);
        od[j] = empty ? INFINITY : d[j];
        oi[j] = empty ? -1 : i[j];
      }
    }
  }
};

__device__ __forceinline__ void load_query(const float4* __restrict__ p, float* qv) {
  const float4 a = __ldg(p + 0), b = __ldg(p + 1), c = __ldg(p + 2), e = __ldg(p + 3);
  qv[0] = a.x; qv[1] = a.y; qv[2] = a.z; qv[3] = a.w; qv[4] = b.x; qv[5] = b.y; qv[6] = b.z;
  qv[7] = c.x; qv[8] = c.y; qv[9] = c.z; qv[10] = c.w; qv[11] = e.x; qv[12] = e.y; qv[13] = e.z;
}

// squared distance d = sum (q - q')^2 + w sum (qd - qd')^2 against a node in shared memory
__device__ __forceinline__ float knn_dist(const float* qv, const float4* nd, float w) {
  const float4 a = nd[0], b = nd[1], c = nd[2], e = nd[3];
  float t, dq = 0.f, dv = 0.f;
  t = qv[0] - a.x; dq = fmaf(t, t, dq);
  t = qv[1] - a.y; dq = fmaf(t, t, dq);
  t = qv[2] - a.z; dq = fmaf(t, t, dq);
  t = qv[3] - a.w; dq = fmaf(t, t, dq);
  t = qv[4] - b.x; dq = fmaf(t, t, dq);
  t = qv[5] - b.y; dq = fmaf(t, t, dq);
  t = qv[6] - b.z; dq = fmaf(t, t, dq);
  t = qv[7] - c.x; dv = fmaf(t, t, dv);
  t = qv[8] - c.y; dv = fmaf(t, t, dv);
  t = qv[9] - c.z; dv = fmaf(t, t, dv);
  t = qv[10] - c.w; dv = fmaf(t, t, dv);
  t = qv[11] - e.x; dv = fmaf(t, t, dv);
  t = qv[12] - e.y; dv = fmaf(t, t, dv);
  t = qv[13] - e.z; dv = fmaf(t, t, dv);
  return fmaf(w, dv, dq);
}

// Scan nodes [lo, hi) of `tree` ([N][16] f32 as float4 x 4) for one query
// per thread.  Every thread of the block must call this (it synchronises).
template <int KM>
__device__ __forceinline__ void knn_scan_range(const float4* __restrict__ tree, int lo, int hi,
                                               const float* qv, float w, TopK<KM>& top,
                                               float4* tile) {
  for (int base = lo; base < hi; base += KNN_TILE) {
    const int cnt = min(KNN_TILE, hi - base);
    __syncthreads();
    for (int x = threadIdx.x; x < cnt * 4; x += blockDim.x) tile[x] = __ldg(tree + 4L * base + x);
    __syncthreads();
    int n = 0;
    for (; n + 4 <= cnt; n += 4) {   // four independent distance chains
      const float d0 = knn_dist(qv, tile + 4 * n, w);
      const float d1 = knn_dist(qv, tile + 4 * (n + 1), w);
      const float d2 = knn_dist(qv, tile + 4 * (n + 2), w);
      const float d3 = knn_dist(qv, tile + 4 * (n + 3), w);
      top.push(d0, base + n);
      top.push(d1, base + n + 1);
      top.push(d2, base + n + 2);
      top.push(d3, base + n + 3);
    }
    for (; n < cnt; ++n) top.push(knn_dist(qv, tile + 4 * n, w), base + n);
  }
}

}  // namespace fn
