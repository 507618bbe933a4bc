// Edge materialisation of Algorithm 1's inner loop: each candidate is joined
// to its parent set P = {root} + (k-1) nearest tree nodes (Sec. IV-E), and
// each (candidate, parent) pair becomes one edge with its duration bound:
//   goal candidate:  T_p = T_req - t(p)          (fixed duration, checked once)
//   free candidate:  T_p <= t_best - t(p)        (cap of the duration scan)
// Both differences are taken in FP32 (the kernels' precision decides them).
#include <cuda_runtime.h>

#include "fn_internal.h"

namespace fn {

// one thread per (candidate, parent slot, float4 chunk)
__global__ void k_make_edges(const float4* __restrict__ tree, const float* __restrict__ t_node,
                             const float4* __restrict__ cand, int B, int n_goal,
                             const int32_t* __restrict__ nn_idx, int k_nn,
                             const float* __restrict__ T_req, float t_best,
                             float4* __restrict__ s0, float4* __restrict__ s1,
                             float* __restrict__ T_param, int32_t* __restrict__ parent) {
  const int k = k_nn + 1;
  const long n = (long)B * k * 4;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const long e = i >> 2;
    const int part = (int)(i & 3);
    const long b = e / k;
    const int j = (int)(e - b * k);
    const int p = j == 0 ? 0 : __ldg(nn_idx + b * k_nn + (j - 1));
    float4 v;
    if (p >= 0) {
      v = __ldg(tree + 4L * p + part);
    } else {
      v = make_float4(NAN, NAN, NAN, NAN);  // missing neighbour: invalid edge
    }
    s0[4 * e + part] = v;
    s1[4 * e + part] = __ldg(cand + 4 * b + part);
    if (part == 0) {
      const float tp = p >= 0 ? __ldg(t_node + p) : 0.f;
      T_param[e] = b < n_goal ? __fsub_rn(__ldg(T_req + b), tp) : __fsub_rn(t_best, tp);
      if (parent) parent[e] = p;
    }
  }
}

}  // namespace fn

using namespace fn;

extern "C" fn_status fn_make_edges(const float* tree, const float* t_node, const float* cand,
                                   int B, int n_goal, const int32_t* nn_idx, int k_nn,
                                   const float* T_req, float t_best, float* s0, float* s1,
                                   float* T_param, int32_t* parent, void* stream) {
  if (B < 0 || n_goal < 0 || n_goal > B || k_nn < 0 || k_nn > FN_MAX_KNN) return FN_EINVAL;
  if (B == 0) return FN_OK;
  if (!tree || !t_node || !cand || !s0 || !s1 || !T_param) return FN_EINVAL;
  if ((k_nn > 0 && !nn_idx) || (n_goal > 0 && !T_req)) return FN_EINVAL;
  if (!aligned16(tree) || !aligned16(cand) || !aligned16(s0) || !aligned16(s1)) return FN_EINVAL;
  const long n = (long)B * (k_nn + 1) * 4;
  const long blocks = std::min<long>((n + 255) / 256, 1L << 20);
  k_make_edges<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
      (const float4*)tree, t_node, (const float4*)cand, B, n_goal, nn_idx, k_nn, T_req, t_best,
      (float4*)s0, (float4*)s1, T_param, parent);
  return launch_status();
}
