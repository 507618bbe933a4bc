// Rounds of the N-ary search for the minimum feasible time (Sec. IV-D, the
// search after Def. "Minimum feasible time"), shared by the standalone
// refinement (fn_nary.cu) and the planner's refine stage: the bracket
// (a, b], with b feasible, is split into N = 32 equal slots; the 31
// interior slot boundaries are checked in ascending order with the edge
// scan of edge_core.cuh, and the slot where the check first passes becomes
// the next bracket.  The points are formed in single precision,
// t_j = fmaf(j, (b - a) / 32, a).
#pragma once

#include "edge_core.cuh"

namespace fn {

#define NARY_N 32

// the round's interior points t_1..t_31 in the warp's slot sub[0..30]
__device__ __forceinline__ void nary_points(float* sub, float a, float b) {
  const int lane = threadIdx.x & 31;
  const float wd = (b - a) * (1.f / NARY_N);
  __syncwarp();
  if (lane < NARY_N - 1) sub[lane] = fmaf(__int2float_rn(lane + 1), wd, a);
  __syncwarp();
}

// The bracket after a round whose scan returned idx (the first passing
// point sub[idx], or -1 when only the known-feasible b passes), with w_out
// the sample that proved the point just below it infeasible; rt, rp follow
// the feasible end.
__device__ __forceinline__ void nary_bracket(const float* sub, int idx, int w_out, float t_rt,
                                             float t_rp, float& a, float& b, int& wit, float& rt,
                                             float& rp) {
  if (idx >= 0) {
    if (idx > 0) {
      a = sub[idx - 1];
      wit = w_out;
    }
    b = sub[idx];
    rt = t_rt;
    rp = t_rp;
  } else {
    a = sub[NARY_N - 2];
    wit = w_out;
  }
}

// Rounds on the staged edge es while b - a > eps, at most max_rounds (wit:
// the sample that proved a infeasible, -1 if unknown).  Returns the rounds
// run, or FN_SCAN_ABORT if a round's scan hit its pass bound.  One edge_scan
// call site.
template <class Core>
__device__ __forceinline__ int nary_rounds(const ArmK& A, const Core& core, float* es,
                                           float* split, float* sub, int S, float eps,
                                           int max_rounds, float& a, float& b, int wit, float& rt,
                                           float& rp, unsigned& nsamp) {
  int r = 0;
  while (r < max_rounds && b - a > eps) {
    nary_points(sub, a, b);
    float t_rt = NAN, t_rp = NAN;
    int w_out = -1;
    const int idx = edge_scan(A, core, es, split, sub, NARY_N - 1, S, false, 0.f, false, t_rt, t_rp,
                              nsamp, 0, 2, wit, &w_out);
    if (idx == FN_SCAN_ABORT) return FN_SCAN_ABORT;   // the scan's pass bound
    nary_bracket(sub, idx, w_out, t_rt, t_rp, a, b, wit, rt, rp);
    ++r;
  }
  return r;
}

}  // namespace fn
