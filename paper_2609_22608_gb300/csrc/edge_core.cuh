// Device core of the edge check shared by the standalone edge-timing kernels
// and the planner's persistent edge kernel (Sec. IV-D).
//
// One warp times one edge.  The edge's two states sit in the warp's shared
// slot `es` (32 floats); every lane owns a column of the warp's coefficient
// buffer `cb` ([FN_CUBIC_WORDS][32] floats).
//   probe : lanes take 32 consecutive grid durations and evaluate the end
//           samples u = 0 and u = 1 (plain FP32 coefficients); a violation
//           at an end proves the duration infeasible;
//   verify: surviving durations in ascending order, all S samples with lanes
//           = samples (compensated coefficients), warp-ballot exit at the first
//           violating batch; the first duration that passes is k*, every lower
//           index having been shown infeasible by a violating sample;
//   rho_v : lane j < 7 takes joint j's exact velocity extremum at T_{k*}.
#pragma once

#include "fn_arm.cuh"

namespace fn {

struct EdgeResult {
  int k;          // grid index (FULL) / 0 (FIXED) / -1 none / -2 invalid
  float T;        // duration at k (FULL), the fixed duration (FIXED)
  float rt, rp, rv;
  bool ok;        // k >= 0 && rv <= 1
};

__device__ __forceinline__ float sample_u(int s, int S) {
  // u_s = s / (S-1): t_s = u_s T, exact at both ends (u = 0, u = 1)
  return __int2float_rn(s) / __int2float_rn(S - 1);
}

// Stage edge (row0, row1) in the warp's shared slot; returns whether all 28
// state values are finite.  `pad` lanes (index 7 of each half-row) are ignored.
__device__ __forceinline__ bool stage_rows(const float* row0, const float* row1, float* es) {
  const int lane = threadIdx.x & 31;
  const float v = lane < 16 ? __ldg(row0 + lane) : __ldg(row1 + (lane - 16));
  __syncwarp();
  es[lane] = v;
  __syncwarp();
  const bool pad = (lane & 7) == 7;
  return __all_sync(0xffffffffu, pad || isfinite(v));
}

// All S samples of duration T with lanes = samples.  exit_early stops at the
// first violating batch.  Returns true iff every sample passes; rt/rp are the
// warp maxima over the evaluated samples.
__device__ __forceinline__ bool verify_duration(const ArmK& A, const float* es, CubicLane cb,
                                                float T, int S, bool exit_early, float& rt,
                                                float& rp, unsigned& nsamp) {
  const int lane = threadIdx.x & 31;
  {
    Cubic c;
    cubic_coef_sh<true>(es, T, c);
    cb.store(c);
  }
  float mt = 0.f, mp = 0.f;
  bool bad = false;
  for (int s0 = 0; s0 < S; s0 += 32) {
    const int s = s0 + lane;
    bool viol = false;
    if (s < S) {
      float a, b;
      sample_ratios(A, cb, sample_u(s, S), a, b);
      mt = fmaxf(mt, a);
      mp = fmaxf(mp, b);
      viol = !(a <= 1.f && b <= 1.f);
    }
    nsamp += min(32, S - s0);
    if (__any_sync(0xffffffffu, viol)) {
      bad = true;
      if (exit_early) break;
    }
  }
  rt = warp_max(mt);
  rp = warp_max(mp);
  return !bad;
}

__device__ __forceinline__ float warp_rho_v(const ArmK& A, const float* es, float T) {
  const int lane = threadIdx.x & 31;
  float r = 0.f;
  if (lane < 7) {
    Cubic c;
    cubic_coef_sh<true>(es, T, c);
#pragma unroll
    for (int j = 0; j < 7; ++j)
      if (lane == j) r = rho_v_joint(A, c, j);
  }
  return warp_max(r);
}

// first feasible grid index in [0, Kadm)
__device__ __forceinline__ int first_feasible(const ArmK& A, const float* es, CubicLane cb,
                                              const float* sT, int Kadm, int S, float& rt,
                                              float& rp, unsigned& nsamp) {
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < Kadm; base += 32) {
    const int k = base + lane;
    bool first_end = false, pass = false;
    if (k < Kadm) {
      {
        Cubic c;
        cubic_coef_sh<false>(es, sT[k], c);
        cb.store(c);
      }
      float a, b;
      sample_ratios(A, cb, 0.f, a, b);
      first_end = (a <= 1.f && b <= 1.f);
      if (first_end) {
        sample_ratios(A, cb, 1.f, a, b);
        pass = (a <= 1.f && b <= 1.f);
      }
    }
    nsamp += min(32, Kadm - base) + __popc(__ballot_sync(0xffffffffu, first_end));
    unsigned mask = __ballot_sync(0xffffffffu, pass);
    while (mask) {
      const int kk = base + __ffs(mask) - 1;
      if (verify_duration(A, es, cb, sT[kk], S, true, rt, rp, nsamp)) return kk;
      mask &= mask - 1;
    }
  }
  return -1;
}

// admissible prefix of the ascending grid: #{k : T_k <= cap}
__device__ __forceinline__ int grid_prefix(const float* sT, int K, float cap) {
  const int lane = threadIdx.x & 31;
  int cnt = 0;
  for (int b = 0; b < K; b += 32) {
    const int k = b + lane;
    cnt += __popc(__ballot_sync(0xffffffffu, k < K && sT[k] <= cap));
  }
  return cnt;
}

// Time one staged edge.  fixed: single duration Tp (goal branch of
// Algorithm 1); otherwise the first feasible grid duration with T_k <= Tp
// (Tp = +inf for no cap).
// exact = false lets a fixed-duration check stop at the first violating batch
// (its ratios are then lower bounds; ok is exact either way).
__device__ __forceinline__ EdgeResult time_edge(const ArmK& A, const float* es, CubicLane cb,
                                                bool finite, bool fixed, float Tp,
                                                const float* sT, int K, int S, bool exact,
                                                unsigned& nsamp) {
  EdgeResult r;
  r.rt = r.rp = r.rv = NAN;
  r.ok = false;
  if (fixed) {
    if (!finite || !(isfinite(Tp) && Tp > 0.f)) {
      r.k = -2;
      r.T = NAN;
      return r;
    }
    const bool pass = verify_duration(A, es, cb, Tp, S, !exact, r.rt, r.rp, nsamp);
    if (exact || pass) r.rv = warp_rho_v(A, es, Tp);
    r.k = pass ? 0 : -1;
    r.T = Tp;
    r.ok = pass && r.rv <= 1.f;
    return r;
  }
  if (!finite) {
    r.k = -2;
    r.T = NAN;
    return r;
  }
  const int Kadm = grid_prefix(sT, K, Tp);
  r.k = first_feasible(A, es, cb, sT, Kadm, S, r.rt, r.rp, nsamp);
  if (r.k >= 0) {
    r.T = sT[r.k];
    r.rv = warp_rho_v(A, es, r.T);
    r.ok = r.rv <= 1.f;
  } else {
    r.T = INFINITY;
    r.rt = r.rp = NAN;
  }
  return r;
}

}  // namespace fn
