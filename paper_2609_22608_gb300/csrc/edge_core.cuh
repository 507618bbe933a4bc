// Device core of the edge check shared by the standalone edge-timing kernels
// and the planner's persistent edge kernel (Sec. IV-D).
//
// One warp times one edge.  The edge's two states sit in the warp's shared
// slot `es` (32 floats); every lane owns a column of the warp's coefficient
// buffer `cb` ([FN_CUBIC_WORDS][32] floats).
//   probe : lanes take 32 consecutive grid durations and evaluate the end
//           samples u = 0 and u = 1, then four interior samples (plain FP32
//           coefficients); a violation at any probed sample proves the
//           duration infeasible;
//   verify: surviving durations in ascending order, all S samples with lanes
//           = samples (compensated coefficients), warp-ballot exit at the first
//           violating batch; the first duration that passes is k*, every lower
//           index having been shown infeasible by a violating sample;
//   witness: (optional) the sample that proved a duration infeasible is
//           probed at the other candidates before any verify of them; on
//           closely spaced durations (the N-ary rounds) neighbours tend to
//           violate at the same sample, on the log grid they do not often
//           enough to pay;
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

// Interior probe samples: indices round(j (S-1) / 5), j = 1..4, of the S
// collocation points (points of the check itself, so a violation there
// proves the duration infeasible).  Measured on random edges, durations
// whose two ends pass but which fail the full check violate at one of these
// four points in ~93 % of cases.
#define FN_MID_PROBES 4
__device__ __forceinline__ int mid_probe_index(int j, int S) {
  return (int)((2 * (j + 1) * (S - 1) + 5) / 10);  // round((j+1)(S-1)/5)
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

// Edge scan with a single torque-evaluation call site (the RNEA body is
// ~1.2k instructions; inlining it at several call sites overflowed the
// instruction cache).  Each pass evaluates at most one sample per lane:
//   PROBE_LO : lanes = grid durations base+lane, sample u = 0
//   PROBE_HI : the lanes whose u = 0 passed, sample u = 1
//   PROBE_MID: the lanes still passing, interior samples mid_probe_index(j)
//   VERIFY   : lanes = samples (s0 + lane) of one duration, compensated
//              coefficients, until a violating batch or all S samples pass
//   PROBE_W  : (wmode 2) one sample, the witness, at the remaining survivors
//              (plain coefficients): after a failed verify, that duration's
//              first violating sample; at the start, the caller's w_in
// Grid mode (fixed = false): returns the first feasible index in
// [k_begin, Kadm) (k_begin = 0 unless a caller scans a sub-range).
// Fixed mode: one duration Tfix is verified (all S samples when exact,
// else up to the first violating batch); returns 0 if it passes, else -1.
// Witness modes (grid mode only; callers other than the N-ary refinement
// pass 0 and the code folds away):
//   wmode 1: record, per duration, the sample that proved it infeasible, and
//            return in *w_out that of the duration just below the result
//            (of the last admissible duration if none passes; -1 if it was
//            not in the result's chunk of 32);
//   wmode 2: as 1, plus the witness probes (PROBE_W), starting with w_in
//            (if >= 0) at every duration in place of the end probes.
__device__ __forceinline__ int edge_scan(const ArmK& A, const float* es, CubicLane cb,
                                         LaneWrench wr, const float* sT, int Kadm, int S,
                                         bool fixed, float Tfix, bool exact, float& rt, float& rp,
                                         unsigned& nsamp, int k_begin = 0, int wmode = 0,
                                         int w_in = -1, int* w_out = nullptr) {
  enum { PROBE_LO = 0, PROBE_HI = 1, VERIFY = 2, PROBE_MID = 3, PROBE_W = 4 };
  const int lane = threadIdx.x & 31;
  int mode = PROBE_LO, base = k_begin, kk = 0, s0 = 0, mj = 0, sw = 0;
  int kill = -1;        // wmode > 0: sample that proved duration base + lane infeasible
  unsigned cand = 0u;   // PROBE_HI: lanes to evaluate; VERIFY: durations left in the chunk
  float mt = 0.f, mp = 0.f;
  bool bad = false;
  if (w_out) *w_out = -1;
  if (fixed) {
    mode = VERIFY;
    Cubic c;
    cubic_coef_sh<true>(es, Tfix, c);
    cb.store(c);
  } else {
    if (Kadm <= k_begin) return -1;
    Cubic c;
    if (base + lane < Kadm) cubic_coef_sh<false>(es, sT[base + lane], c);
    cb.store(c);
    if (wmode == 2 && w_in >= 0) {
      mode = PROBE_W;
      sw = w_in;
      cand = __ballot_sync(0xffffffffu, base + lane < Kadm);
    }
  }
  for (;;) {
    bool active;
    int si;               // sample index of this pass (probes)
    if (mode == VERIFY) {
      active = s0 + lane < S;
      si = s0 + lane;
    } else if (mode == PROBE_MID || mode == PROBE_W) {
      active = (cand >> lane) & 1u;
      si = mode == PROBE_MID ? mid_probe_index(mj, S) : sw;
    } else {
      active = mode == PROBE_LO ? (base + lane < Kadm) : ((cand >> lane) & 1u);
      si = mode == PROBE_LO ? 0 : S - 1;
    }
    const float u = sample_u(si, S);
    float a = 0.f, b = 0.f;
    if (active) sample_ratios(A, cb, u, a, b, wr);   // the single call site
    const bool pass = active && a <= 1.f && b <= 1.f;
    const unsigned act = __ballot_sync(0xffffffffu, active);
    const unsigned ok = __ballot_sync(0xffffffffu, pass);
    nsamp += __popc(act);
    if (wmode > 0 && mode != VERIFY && active && !pass) kill = si;
    int next_dur = -1;  // duration to verify next, if any
    if (mode == PROBE_LO) {
      if (ok) {
        cand = ok;
        mode = PROBE_HI;
        continue;
      }
    } else if (mode == PROBE_HI || mode == PROBE_MID || mode == PROBE_W) {
      cand = ok;                       // durations whose probes so far pass
      if (cand && mode == PROBE_HI && S > 2) {
        mode = PROBE_MID;
        mj = 0;
        continue;
      }
      if (cand && mode == PROBE_MID && ++mj < FN_MID_PROBES) continue;
      if (cand) next_dur = base + __ffs(cand) - 1;
    } else {
      if (active) { mt = fmaxf(mt, a); mp = fmaxf(mp, b); }
      const bool viol = (act & ~ok) != 0u;
      if (fixed) {
        bad = bad || viol;
        if ((!viol || exact) && s0 + 32 < S) {
          s0 += 32;
          continue;
        }
        rt = warp_max(mt);
        rp = warp_max(mp);
        return bad ? -1 : 0;
      }
      if (viol) {                      // kk is infeasible
        if (wmode > 0) {
          sw = s0 + __ffs(act & ~ok) - 1;
          if (lane == kk - base) kill = sw;
        }
        cand &= cand - 1;
        if (cand && wmode == 2) {      // probe its witness sample at the rest
          mode = PROBE_W;
          Cubic c;
          if (base + lane < Kadm) cubic_coef_sh<false>(es, sT[base + lane], c);
          cb.store(c);
          continue;
        }
        if (cand) next_dur = base + __ffs(cand) - 1;
      } else if (s0 + 32 < S) {
        s0 += 32;
        continue;
      } else {
        rt = warp_max(mt);
        rp = warp_max(mp);
        if (w_out) {
          const int below = kk - 1 - base;
          const int w = __shfl_sync(0xffffffffu, kill, below >= 0 ? below : 0);
          *w_out = below >= 0 ? w : -1;
        }
        return kk;
      }
    }
    if (next_dur >= 0) {               // (re)start VERIFY on the next survivor
      kk = next_dur;
      s0 = 0;
      mt = mp = 0.f;
      mode = VERIFY;
      Cubic c;
      cubic_coef_sh<true>(es, sT[kk], c);
      cb.store(c);
      continue;
    }
    // nothing left in this chunk of 32 durations: probe the next one
    if (w_out) {
      const int last = Kadm - 1 - base;
      const int w = __shfl_sync(0xffffffffu, kill, last < 32 ? last : 0);
      *w_out = last < 32 ? w : -1;
    }
    base += 32;
    if (base >= Kadm) return -1;
    kill = -1;
    mode = PROBE_LO;
    cand = 0u;
    Cubic c;
    if (base + lane < Kadm) cubic_coef_sh<false>(es, sT[base + lane], c);
    cb.store(c);
  }
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
                                                LaneWrench wr, bool finite, bool fixed, float Tp,
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
    const bool pass = edge_scan(A, es, cb, wr, sT, 0, S, true, Tp, exact, r.rt, r.rp, nsamp) == 0;
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
  r.k = edge_scan(A, es, cb, wr, sT, Kadm, S, false, 0.f, false, r.rt, r.rp, nsamp);
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
