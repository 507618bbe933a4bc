// Minimum feasible time refined by the N-ary search (Sec. IV-D, the search
// after Def. "Minimum feasible time"): the grid scan finds the first
// feasible grid index k*, then the bracket (T_{k*-1}, T_{k*}] (T_{-1} = 0)
// is split into N = 32 equal slots per round; the 31 interior slot
// boundaries are checked and the slot where the check first passes is
// kept, until the bracket is no wider than eps.  rho_v is checked once, at
// the refined duration.
//
// One warp per edge.  A round is the grid scan's own probe/verify machinery
// (edge_core.cuh) run over a 31-entry duration list in the warp's shared
// slot, so the kernel keeps a single torque-evaluation call site: the grid
// pass and every round go through the same edge_scan call in one loop.  The
// rounds use witness probing: the 31 points are so close together that the
// points below T* usually violate at the sample that proved the bracket's
// lower end infeasible, so a round starts by probing that sample at every
// point, and a failed verify passes its violating sample on the same way.
#include <cuda_runtime.h>

#include "fn_internal.h"
#include "nary_core.cuh"
#include "fn_tune.h"

namespace fn {

struct NaryGrid {
  float T[FN_MAX_GRID];
};

#define NARY_WARPS 3   // as the grid scan: static shared memory within 48 KB
#define NARY_MAX_ROUNDS 16

// Persistent: warp w takes edges w, w + W, ...  MINB sets the register
// budget, as for the grid scan's kernel, whose tuned variant it follows.
template <int MINB>
__global__ void __launch_bounds__(32 * NARY_WARPS, MINB)
    k_time_edges_nary(ArmK A, NaryGrid G, int K, int S, const float* __restrict__ s0,
                      const float* __restrict__ s1, int E, const float* __restrict__ T_cap,
                      float eps, int max_rounds, int32_t* __restrict__ k_star,
                      float* __restrict__ T_star, float* __restrict__ T_lo,
                      float* __restrict__ rho3, uint8_t* __restrict__ ok,
                      int32_t* __restrict__ rounds, unsigned long long* __restrict__ counter) {
  __shared__ float sT[FN_MAX_GRID];
  __shared__ float sSub[NARY_WARPS][32];
  __shared__ float sEdge[NARY_WARPS][32];
  __shared__ float sCoef[NARY_WARPS][FN_CUBIC_WORDS * 32];
  __shared__ float sWr[NARY_WARPS][FN_LINK_WORDS * 32];
  __shared__ __align__(16) float sSplit[NARY_WARPS][FN_SPLIT_WORDS];
  __shared__ float4 sLink[7 * FN_LINK_F4];
  fill_links(A, sLink);
  for (int i = threadIdx.x; i < K; i += blockDim.x) sT[i] = G.T[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* es = sEdge[w];
  float* sub = sSub[w];
  const CubicLane cb{&sCoef[w][lane]};
  const LaneLink wr{&sWr[w][lane]};
  const LinkTab L{sLink};
  const long W = (long)gridDim.x * NARY_WARPS;
  unsigned nsamp = 0;
  for (long e = (long)blockIdx.x * NARY_WARPS + w; e < E; e += W) {
    const bool finite = stage_rows(s0 + 16 * e, s1 + 16 * e, es);
    const float Tp = T_cap ? __ldg(T_cap + e) : INFINITY;
    int k = -2, r = 0;
    float a = NAN, b = NAN, rt = NAN, rp = NAN, rv = NAN;
    if (finite) {
      const float* dur = sT;                 // the grid, then each round's points
      int n = grid_prefix(sT, K, Tp);
      int wit = -1;                          // sample that proved a infeasible
      for (;;) {
        float t_rt = NAN, t_rp = NAN;
        int w_out = -1;
        const bool grid = dur == sT;
        const int idx = edge_scan(A, ScalarCore{L, cb, wr}, es, sSplit[w], dur, n, S, false, 0.f, false, t_rt, t_rp, nsamp,
                                  0, grid ? 1 : 2, wit, &w_out);
        if (idx == FN_SCAN_ABORT) {          // the scan's pass bound (never expected)
          k = FN_SCAN_ABORT;
          break;
        }
        if (grid) {
          k = idx;
          if (idx < 0) break;
          a = idx > 0 ? sT[idx - 1] : 0.f;
          b = sT[idx];
          wit = idx > 0 ? w_out : -1;
          rt = t_rt;
          rp = t_rp;
        } else {
          nary_bracket(sub, idx, w_out, t_rt, t_rp, a, b, wit, rt, rp);
          ++r;
        }
        if (r >= max_rounds || !(b - a > eps)) break;
        nary_points(sub, a, b);
        dur = sub;
        n = NARY_N - 1;
      }
      if (k >= 0) rv = warp_rho_v(A, es, b);
    }
    if (lane == 0) {
      k_star[e] = k;
      T_star[e] = k >= 0 ? b : (k == -1 ? INFINITY : NAN);   // -2 invalid, -3 aborted
      if (T_lo) T_lo[e] = k >= 0 ? a : NAN;
      rho3[3 * e + 0] = k >= 0 ? rt : NAN;
      rho3[3 * e + 1] = k >= 0 ? rp : NAN;
      rho3[3 * e + 2] = rv;
      ok[e] = (k >= 0 && rv <= 1.f) ? 1 : 0;
      if (rounds) rounds[e] = r;
    }
  }
  if (counter && lane == 0 && nsamp) atomicAdd(counter, (unsigned long long)nsamp);
}

}  // namespace fn

using namespace fn;

extern "C" fn_status fn_time_edges_nary(const fn_arm_t* arm, const float* s0, const float* s1,
                                        int E, const float* T_grid, int K, int S,
                                        const float* T_cap, float eps, int max_rounds,
                                        int32_t* k_star, float* T_star, float* T_lo, float* rho3,
                                        uint8_t* ok, int32_t* rounds,
                                        unsigned long long* sample_count, void* stream) {
  ArmK A;
  if (!make_armk(arm, &A)) return FN_EINVAL;
  if (E < 0 || S < 2 || S > FN_MAX_S) return FN_EINVAL;
  if (!(eps > 0.f) || !std::isfinite(eps)) return FN_EINVAL;
  if (max_rounds < 0 || max_rounds > NARY_MAX_ROUNDS) return FN_EINVAL;
  if (!T_grid || K < 1 || K > FN_MAX_GRID) return FN_EINVAL;
  NaryGrid G;
  for (int k = 0; k < K; ++k) {
    if (!(T_grid[k] > 0.f) || !std::isfinite(T_grid[k])) return FN_EINVAL;
    if (k > 0 && !(T_grid[k] > T_grid[k - 1])) return FN_EINVAL;
    G.T[k] = T_grid[k];
  }
  if (E == 0) return FN_OK;
  if (!s0 || !s1 || !k_star || !T_star || !rho3 || !ok) return FN_EINVAL;
  if (!aligned16(s0) || !aligned16(s1)) return FN_EINVAL;
  typedef void (*Kern)(ArmK, NaryGrid, int, int, const float*, const float*, int, const float*,
                       float, int, int32_t*, float*, float*, float*, uint8_t*, int32_t*,
                       unsigned long long*);
  const int vt = tuned_variant(TUNE_EDGES_FULL, E, K, S);   // its register budget
  const int v = vt < kEdgeVariants ? vt : kDefaultEdgeVariant;
  Kern kern = v == 0 ? k_time_edges_nary<2> : (v == 1 ? k_time_edges_nary<3> : k_time_edges_nary<4>);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * NARY_WARPS, 0) !=
          cudaSuccess || per_sm < 1)
    per_sm = 1;
  const long want = ((long)E + NARY_WARPS - 1) / NARY_WARPS;
  const int blocks = (int)std::max<long>(1, std::min<long>(want, (long)per_sm * num_sms()));
  kern<<<blocks, 32 * NARY_WARPS, 0, (cudaStream_t)stream>>>(A, G, K, S, s0, s1, E, T_cap, eps,
                                                             max_rounds, k_star, T_star, T_lo,
                                                             rho3, ok, rounds, sample_count);
  return launch_status();
}
