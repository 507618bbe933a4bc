// Device core of the edge check shared by the standalone edge-timing kernels
// and the planner's persistent edge kernel (Sec. IV-D).
//
// One warp times one edge.  The edge's two states sit in the warp's shared
// slot `es` (32 floats); every lane owns a column of the warp's coefficient
// buffer `cb` ([FN_CUBIC_WORDS][32] floats); `split` is the warp's slot of
// FN_SPLIT_WORDS floats for the end-sample torque split.
//   split : once per edge, lanes 0..5 = (end, part) evaluate Eq. (torque) at
//           the edge's two end states: tau(T) = alpha / T^2 + beta / T + gamma
//           at u = 0 and u = 1 (end_torque_part's decomposition), because the
//           end states do not depend on T and the acceleration enters
//           Eq. (torque) affinely;
//   probe : lanes take 32 consecutive grid durations and check both end
//           samples from the split (no torque evaluation), then four
//           interior samples (plain FP32 coefficients); a violation at any
//           probed sample proves the duration infeasible;
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
// the same spacing for n interior points: round((j+1)(S-1)/(n+1)), j < n
__device__ __forceinline__ int mid_probe_index(int j, int S, int n) {
  return (int)((2 * (j + 1) * (S - 1) + n + 1) / (2 * (n + 1)));
}

// The warp's end-sample split: per end (u = 0, u = 1) 28 floats, alpha[7],
// beta[7], gamma[7] and the end velocity qd[7] (16-byte aligned slot).
#define FN_SPLIT_WORDS 56

// es[7] (a pad slot of the first state) marks whether `split` holds the
// staged edge's split: stage_rows clears it, the scan sets it.
#define FN_SPLIT_MARK 7

// Stage edge (row0, row1) in the warp's shared slot; returns whether all 28
// state values are finite.  `pad` lanes (index 7 of each half-row) are
// ignored; slot 7 is cleared (no split computed for this edge yet).
__device__ __forceinline__ bool stage_rows(const float* row0, const float* row1, float* es) {
  const int lane = threadIdx.x & 31;
  const float v = lane < 16 ? __ldg(row0 + lane) : __ldg(row1 + (lane - 16));
  __syncwarp();
  es[lane] = lane == FN_SPLIT_MARK ? 0.f : v;
  __syncwarp();
  const bool pad = (lane & 7) == 7;
  return __all_sync(0xffffffffu, pad || isfinite(v));
}

// joint j's entry of a per-joint table of the robot, for a lane-dependent j
// (a select chain over the seven constants: the table stays an immediate
// operand instead of an indexed load from the parameter space)
__device__ __forceinline__ float joint_pick(const float (&t)[7], int j) {
  float v = t[0];
#pragma unroll
  for (int i = 1; i < 7; ++i) v = j == i ? t[i] : v;
  return v;
}

// rho_v at duration T: lane j < 7 takes joint j's exact velocity extremum
// (rho_v_joint's arithmetic with the joint's coefficients built from the
// staged edge), one code path for every lane; the warp maximum is returned
// to all lanes.
__device__ __forceinline__ float warp_rho_v(const ArmK& A, const float* es, float T) {
  const int lane = threadIdx.x & 31;
  float best = 0.f;
  if (lane < 7) {
    const int j = lane;
    float b1, b2, b3;
    joint_coef<true>(es[j], es[8 + j], es[16 + j], es[24 + j], T, b1, b2, b3);
    const float q0 = es[j], iT = 1.0f / T;
    const float lo = joint_pick(A.q_lo, j), hi = joint_pick(A.q_hi, j);
    const float vmax = joint_pick(A.qd_max, j), t2a = joint_pick(A.taper2a, j);
    float cand[3] = {0.f, 1.f, -1.f};
    if (b3 != 0.f) {
      const float us = -b2 / (3.0f * b3);
      if (us > 0.f && us < 1.f) cand[2] = us;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float u = cand[i];
      if (u < 0.f) continue;
      const float pos = fmaf(fmaf(fmaf(b3, u, b2), u, b1), u, q0);
      const float vel = fmaf(fmaf(3.0f * b3, u, 2.0f * b2), u, b1) * iT;
      const float m = fmaxf(fminf(pos - lo, hi - pos), 0.f);
      const float bound = fminf(vmax, sqrtf(t2a * m));
      float r;
      if (bound > 0.f) r = fabsf(vel) / bound;
      else r = (vel != 0.f) ? INFINITY : 0.f;
      best = fmaxf(best, r);
    }
  }
  return warp_max(best);
}

// Both end samples of duration T from the split: tau = alpha / T^2 +
// beta / T + gamma per joint, rho_tau and rho_P at the end velocity.
// Returns whether both pass; fail0: the u = 0 end failed.
__device__ __forceinline__ bool end_probe_pass(const ArmK& A, const float* split, float T,
                                               bool& fail0) {
  const float iT = 1.0f / T, iT2 = iT * iT;
  bool pass = true;
#pragma unroll
  for (int end = 0; end < 2; ++end) {
    const float4* c4 = reinterpret_cast<const float4*>(split + 28 * end);
    float f[28];
#pragma unroll
    for (int v = 0; v < 7; ++v) {
      const float4 t = c4[v];
      f[4 * v] = t.x; f[4 * v + 1] = t.y; f[4 * v + 2] = t.z; f[4 * v + 3] = t.w;
    }
    float r = 0.f, pw = 0.f;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      const float tau = fmaf(f[j], iT2, fmaf(f[7 + j], iT, f[14 + j]));
      r = fmaxf(r, fabsf(tau) * A.inv_tau[j]);
      pw = fmaf(tau, f[21 + j], pw);
    }
    const bool pe = r <= 1.f && fabsf(pw) * A.inv_w <= 1.f;
    if (end == 0) fail0 = !pe;
    pass = pass && pe;
  }
  return pass;
}

// position of the i-th lowest set bit of x (i = 0: the lowest); -1 if x has
// at most i set bits
__device__ __forceinline__ int nth_bit(unsigned x, int i) {
  for (int t = 0; t < i && x; ++t) x &= x - 1u;
  return __ffs(x) - 1;
}

// Upper bound on the passes of one edge_scan call over n admissible
// durations: per chunk of 32, one end probe plus, for each of its 32
// durations at most, one witness pass, four interior-probe passes and
// ceil(S/32) verification passes; plus the split and the final chunk step.
// Reaching it means the state machine failed to progress: the scan returns
// FN_SCAN_ABORT instead of looping on.
#define FN_SCAN_ABORT (-3)
__host__ __device__ __forceinline__ int scan_pass_cap(int n, int S) {
  return ((n + 31) / 32 + 1) * (2 + 32 * (5 + (S + 31) / 32)) + 2;
}

// the lowest (up to) n set bits of x
__device__ __forceinline__ unsigned lowest_bits(unsigned x, int n) {
  unsigned r = 0u;
  for (int t = 0; t < n && x; ++t) {
    const unsigned bit = x & (0u - x);
    r |= bit;
    x ^= bit;
  }
  return r;
}

// The torque evaluation of the scan ("core"): NS samples per lane per pass.
//   ScalarCore: one sample (torque_at_rolled; records in a LaneLink column)
//   PairCore  : two samples of the same cubic (torque_at_pair, paired FP32;
//               records in the Stash: a LaneLink2 column or tensor memory)
// eval() is called by every lane of the warp (tensor-memory records are
// warp-collective); sink(j, tau, qd, 1 / tau_max_j) gets pairs, whose .y
// half is meaningful only for NS = 2; gs, fs scale gravity and friction per
// half.  store2 gives the halves different cubics (the scalar core keeps x).
struct ScalarCore {
  static constexpr int NS = 1;
  LinkTab L;
  CubicLane cb;
  LaneLink wr;
  __device__ __forceinline__ void store(const Cubic& c) const { cb.store(c); }
  __device__ __forceinline__ void store2(const Cubic& cx, const Cubic&) const { cb.store(cx); }
  template <class Sink>
  __device__ __forceinline__ void eval(const ArmK& A, float2 u, float2 gs, float2 fs,
                                       Sink&& sink) const {
    torque_at_rolled(
        A, L, cb, u.x,
        [&](int j, float tau, float v, float inv_tau) {
          sink(j, make_float2(tau, 0.f), make_float2(v, 0.f), inv_tau);
        },
        wr, gs.x, fs.x);
  }
};

template <class Stash>
struct PairCore {
  static constexpr int NS = 2;
  LinkTab2 L;
  CubicLane2 cb;
  Stash st;
  __device__ __forceinline__ void store(const Cubic& c) const { cb.store(c); }
  __device__ __forceinline__ void store2(const Cubic& cx, const Cubic& cy) const {
    cb.store2(cx, cy);
  }
  template <class Sink>
  __device__ __forceinline__ void eval(const ArmK& A, float2 u, float2 gs, float2 fs,
                                       Sink&& sink) const {
    torque_at_pair(A, L, cb, u, sink, st, gs, fs);
  }
};

// The end-sample split cubic of item (end, part) of a staged edge: its
// u = 0 sample is (q, qd, qdd) exactly (iT = iT2 = 1, b1 = qd, b2 = qdd / 2):
// part 0 the end state with zero acceleration, parts 1 and 2 the two
// acceleration vectors of end_torque_part at zero velocity.
__device__ __forceinline__ void split_cubic(const float* es, int end, int part, Cubic& c) {
  c.iT = 1.f;
  c.iT2 = 1.f;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    const float d = es[16 + j] - es[j];
    const float qa = end ? -6.0f * d : 6.0f * d;
    const float qb = end ? fmaf(4.0f, es[24 + j], 2.0f * es[8 + j])
                         : -fmaf(4.0f, es[8 + j], 2.0f * es[24 + j]);
    c.q0[j] = es[16 * end + j];
    c.b1[j] = part == 0 ? es[16 * end + 8 + j] : 0.f;
    c.b2[j] = 0.5f * (part == 0 ? 0.f : (part == 1 ? qa : qb));
    c.b3[j] = 0.f;
  }
}

// The splits of n <= 5 NS staged edges in one pass: item i = 6 e + 3 end +
// part, items 0..29 on the x halves of lanes 0..29, items 30..59 on the y
// halves (NS = 2).  Edge e's states are es_g[32 e ..] and its split goes to
// split_g[FN_SPLIT_WORDS e ..]; each edge's split mark is set.  Edges whose
// states are not finite get a meaningless split they never use.
template <class Core>
__device__ __forceinline__ void split_group(const ArmK& A, const Core& core, float* es_g,
                                            float* split_g, int n, unsigned& nsamp) {
  const int lane = threadIdx.x & 31;
  const int ex = lane / 6, ey = 5 + lane / 6, ix = lane % 6;
  const int end = ix >= 3 ? 1 : 0, part = ix - 3 * end;
  const bool ax = lane < 30 && ex < n;
  const bool ay = Core::NS == 2 && lane < 30 && ey < n;
  Cubic cx, cy;
  split_cubic(es_g + 32 * (ax ? ex : 0), end, part, cx);
  split_cubic(es_g + 32 * (ay ? ey : 0), end, part, cy);
  core.store2(cx, cy);
  const float on = part == 0 ? 1.f : 0.f;   // parts 1, 2: M + I_m only
  const int so = 28 * end + (part == 0 ? 14 : 7 * (part - 1));
  float* sx = split_g + FN_SPLIT_WORDS * (ax ? ex : 0) + so;
  float* sy = split_g + FN_SPLIT_WORDS * (ay ? ey : 0) + so;
  core.eval(A, make_float2(0.f, 0.f), make_float2(on, on), make_float2(on, on),
            [&](int j, float2 tau, float2, float) {
              if (ax) sx[j] = tau.x;
              if (ay) sy[j] = tau.y;
            });
  nsamp += __popc(__ballot_sync(0xffffffffu, ax)) + __popc(__ballot_sync(0xffffffffu, ay));
  __syncwarp();
  for (int e = 0; e < n; ++e) {   // end velocities; the split is ready
    float* s = split_g + FN_SPLIT_WORDS * e;
    const float* es = es_g + 32 * e;
    if (lane < 7) {
      s[21 + lane] = es[8 + lane];
      s[49 + lane] = es[24 + lane];
    }
  }
  __syncwarp();
  if (lane < n) es_g[32 * lane + FN_SPLIT_MARK] = 1.f;
  __syncwarp();
}

// Edge scan with a single torque-evaluation call site (the RNEA body is
// ~1k instructions; inlining it at several call sites overflowed the
// instruction cache) and a single coefficient-build site.  Each pass
// evaluates NS = Core::NS samples per lane (x, and y for the paired core).
// Passes:
//   SPLIT    : (once per staged edge) lanes 0..5 = (end, part) evaluate the
//              end-sample split into `split`; part 0 is Eq. (torque) at the
//              end state with zero acceleration (gamma), parts 1 and 2 the
//              mass matrix plus armature times the two acceleration vectors
//              (alpha, beta: gravity, velocity and friction off)
//   PROBE_END: lanes = grid durations base+lane, both end samples from the
//              split (no torque evaluation)
//   PROBE_MID: interior samples mid_probe_index(j, S, 4 NS), j < 4 NS, of the
//              lowest survivors not yet probed there: packed (wmode 0), the
//              lowest eight survivors x 4 NS samples in one pass, lane = 4 i +
//              j (x: sample j, y: sample j + 4); otherwise lanes = durations,
//              NS samples per pass
//   PROBE_W  : (wmode 2) one sample, the witness, at the remaining survivors
//              (plain coefficients): after a failed verify, that duration's
//              first violating sample; on the first chunk, the caller's w_in
//   VERIFY   : lanes = samples of the lowest survivor once it passed its
//              interior probes (x: s0 + lane, y: s0 + 32 + lane), compensated
//              coefficients, until a violating batch or all S samples pass
// A survivor is verified only after its interior probes, and the lowest
// survivor first, so the first duration that passes is k*: every lower
// index was shown infeasible by a violating sample.
// Grid mode (fixed = false): returns the first feasible index in
// [k_begin, Kadm) (k_begin = 0 unless a caller scans a sub-range); `split`
// is the warp's FN_SPLIT_WORDS slot (16-byte aligned), reused across calls
// on the same staged edge.
// Fixed mode: one duration Tfix is verified (all S samples when exact,
// else up to the first violating batch); returns 0 if it passes, else -1;
// `split` may be null.
// Witness modes (grid mode only; callers other than the N-ary refinement
// pass 0 and the code folds away):
//   wmode 1: record, per duration, the sample that proved it infeasible, and
//            return in *w_out that of the duration just below the result
//            (of the last admissible duration if none passes; -1 if it was
//            not in the result's chunk of 32);
//   wmode 2: as 1, plus the witness probes (PROBE_W), starting with w_in
//            (if it is an interior sample) after the first chunk's end probes.
template <class Core>
__device__ __forceinline__ int edge_scan(const ArmK& A, const Core& core, float* es, float* split,
                                         const float* sT, int Kadm, int S, bool fixed, float Tfix,
                                         bool exact, float& rt, float& rp, unsigned& nsamp,
                                         int k_begin = 0, int wmode = 0, int w_in = -1,
                                         int* w_out = nullptr) {
  enum { SPLIT = 0, PROBE_END = 1, PROBE_W = 2, PROBE_MID = 3, VERIFY = 4 };
  enum { COEF_NONE = 0, COEF_PLAIN = 1, COEF_EXACT = 2, COEF_SPLIT = 3 };
  constexpr int NS = Core::NS;
  constexpr int NMID = FN_MID_PROBES * NS;   // interior probe samples per survivor
  constexpr int BATCH = 32 * NS;             // verification samples per pass
  const int lane = threadIdx.x & 31;
  const bool packed = wmode == 0;       // interior probes of 8 survivors x NMID samples per pass
  int mode = PROBE_END, base = k_begin, kk = 0, s0 = 0, mj = 0, sw = 0, coef = COEF_NONE;
  int cdur = -1;        // COEF_PLAIN: this lane's grid index (-1: none)
  int kill = -1;        // wmode > 0: sample that proved duration base + lane infeasible
  unsigned cand = 0u;   // durations (bits relative to base) still in the running
  unsigned mpr = 0u;    // of those, the ones whose interior probes passed
  unsigned sel = 0u;    // PROBE_MID: the durations being probed
  float mt = 0.f, mp = 0.f;
  bool bad = false;
  bool w_pending = wmode == 2 && w_in > 0 && w_in < S - 1;   // interior witness of the caller
  const int cap = scan_pass_cap(fixed ? 1 : max(Kadm - k_begin, 1), S);
  int passes = 0;
  if (w_out) *w_out = -1;
  if (fixed) {
    mode = VERIFY;
    coef = COEF_EXACT;
  } else {
    if (Kadm <= k_begin) return -1;
    if (es[FN_SPLIT_MARK] == 0.f) {
      mode = SPLIT;
      coef = COEF_SPLIT;
    }
  }
  for (;;) {
    if (++passes > cap) return FN_SCAN_ABORT;   // warp-uniform
    if (coef != COEF_NONE) {           // the single coefficient-build site
      Cubic c;
      if (coef == COEF_SPLIT) {
        // lane l < 6: end l / 3, part l % 3
        const int end = lane >= 3 ? 1 : 0;
        split_cubic(es, end, lane - 3 * end, c);
      } else if (coef == COEF_PLAIN) {
        if (cdur >= 0) {
          cubic_coef_sh<false>(es, sT[cdur], c);
        } else {                       // an idle lane: any finite cubic
          c.iT = c.iT2 = 1.f;
#pragma unroll
          for (int j = 0; j < 7; ++j) c.q0[j] = c.b1[j] = c.b2[j] = c.b3[j] = 0.f;
        }
      } else {
        cubic_coef_sh<true>(es, fixed ? Tfix : sT[kk], c);
      }
      core.store(c);
      coef = COEF_NONE;
    }
    bool decide = false;  // choose the next step from (cand, mpr)
    if (mode == PROBE_END) {
      const int k = base + lane;
      const bool active = k < Kadm;
      bool f0 = false;
      const bool pass = active && end_probe_pass(A, split, sT[active ? k : base], f0);
      if (wmode > 0 && active && !pass) kill = f0 ? 0 : S - 1;
      cand = __ballot_sync(0xffffffffu, pass);
      mpr = S > 2 ? 0u : 0xffffffffu;   // S <= 2: no interior samples
      if (cand && w_pending) {
        w_pending = false;
        mode = PROBE_W;
        sw = w_in;
        cdur = ((cand >> lane) & 1u) ? base + lane : -1;
        coef = COEF_PLAIN;
        continue;
      }
      decide = true;
    } else {
      bool ax, ay = false;  // the pass's active samples on this lane
      int sx, sy = 0;       // their sample indices
      if (mode == VERIFY) {
        sx = s0 + lane;
        sy = s0 + 32 + lane;
        ax = sx < S;
        ay = NS == 2 && sy < S;
      } else if (mode == SPLIT) {
        ax = lane < 6;
        sx = 0;
      } else if (mode == PROBE_MID && packed) {
        ax = cdur >= 0;
        ay = NS == 2 && ax;
        sx = mid_probe_index(lane & 3, S, NMID);
        sy = mid_probe_index((lane & 3) + 4, S, NMID);
      } else if (mode == PROBE_MID) {   // lanes = durations, NS samples per pass
        ax = ((sel & cand) >> lane) & 1u;
        ay = NS == 2 && ax;
        sx = mid_probe_index(mj, S, NMID);
        sy = mid_probe_index(mj + 1, S, NMID);
      } else {              // PROBE_W
        ax = (cand >> lane) & 1u;
        sx = sw;
      }
      const float2 u = make_float2(sample_u(sx, S), sample_u(ay ? sy : sx, S));
      const bool sp = mode == SPLIT;
      const float on = (sp && lane != 0 && lane != 3) ? 0.f : 1.f;   // parts 1, 2: M + I_m only
      const int so = lane >= 3 ? 28 : 0;
      const int sj = (lane == 0 || lane == 3) ? 14 : (lane == 1 || lane == 4 ? 0 : 7);
      float rx = 0.f, px = 0.f, ry = 0.f, py = 0.f;
      // the single torque-evaluation call site (every lane; idle halves are
      // ignored below)
      core.eval(A, u, dup2(on), dup2(on), [&](int j, float2 tau, float2 v, float inv_tau) {
        if (sp && ax) split[so + sj + j] = tau.x;
        rx = fmaxf(rx, fabsf(tau.x) * inv_tau);
        px = fmaf(tau.x, v.x, px);
        if (NS == 2) {
          ry = fmaxf(ry, fabsf(tau.y) * inv_tau);
          py = fmaf(tau.y, v.y, py);
        }
      });
      const float bx = fabsf(px) * A.inv_w, by = fabsf(py) * A.inv_w;
      const bool pass_x = ax && rx <= 1.f && bx <= 1.f;
      const bool pass_y = ay && ry <= 1.f && by <= 1.f;
      const unsigned act_x = __ballot_sync(0xffffffffu, ax);
      const unsigned ok_x = __ballot_sync(0xffffffffu, pass_x);
      const unsigned act_y = NS == 2 ? __ballot_sync(0xffffffffu, ay) : 0u;
      const unsigned ok_y = NS == 2 ? __ballot_sync(0xffffffffu, pass_y) : 0u;
      const unsigned fail_x = act_x & ~ok_x, fail_y = act_y & ~ok_y;
      nsamp += __popc(act_x) + __popc(act_y);
      if (sp) {                        // end velocities; the split is ready
        if (lane < 7) {
          split[21 + lane] = es[8 + lane];
          split[49 + lane] = es[24 + lane];
        }
        __syncwarp();
        if (lane == 0) es[FN_SPLIT_MARK] = 1.f;
        __syncwarp();
        mode = PROBE_END;
        continue;
      }
      if (mode == PROBE_W) {
        if (wmode > 0 && ax && !pass_x) kill = sx;
        cand &= ok_x;
        decide = true;
      } else if (mode == PROBE_MID && packed) {
        // survivor i (the i-th set bit of sel) passes iff its 4 lanes pass
        const unsigned okb = NS == 2 ? (ok_x & ok_y) : ok_x;
        const int ns = __popc(sel);
        unsigned failed = 0u;
        for (int i = 0; i < ns; ++i)
          if (((okb >> (4 * i)) & 0xFu) != 0xFu) failed |= 1u << nth_bit(sel, i);
        cand &= ~failed;
        mpr |= sel;
        decide = true;
      } else if (mode == PROBE_MID) {
        if (wmode > 0 && ax && !pass_x) kill = sx;
        else if (wmode > 0 && ay && !pass_y) kill = sy;
        cand &= ~(fail_x | fail_y);
        mj += NS;
        if (mj < NMID && (sel & cand)) continue;
        mpr |= sel;
        decide = true;
      } else {                         // VERIFY
        if (ax) { mt = fmaxf(mt, rx); mp = fmaxf(mp, bx); }
        if (ay) { mt = fmaxf(mt, ry); mp = fmaxf(mp, by); }
        const bool viol = (fail_x | fail_y) != 0u;
        if (fixed) {
          bad = bad || viol;
          if ((!viol || exact) && s0 + BATCH < S) {
            s0 += BATCH;
            continue;
          }
          rt = warp_max(mt);
          rp = warp_max(mp);
          return bad ? -1 : 0;
        }
        if (viol) {                    // kk is infeasible
          if (wmode > 0) {
            // the first violating sample: the x halves hold s0 .. s0 + 31
            sw = fail_x ? s0 + __ffs(fail_x) - 1 : s0 + 32 + __ffs(fail_y) - 1;
            if (lane == kk - base) kill = sw;
          }
          cand &= ~(1u << (kk - base));
          if (cand && wmode == 2) {    // probe its witness sample at the rest
            mode = PROBE_W;
            cdur = ((cand >> lane) & 1u) ? base + lane : -1;
            coef = COEF_PLAIN;
            continue;
          }
          decide = true;
        } else if (s0 + BATCH < S) {
          s0 += BATCH;
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
    }
    if (decide && cand) {
      const int low = __ffs(cand) - 1;
      if ((mpr >> low) & 1u) {         // verify the lowest survivor
        kk = base + low;
        s0 = 0;
        mt = mp = 0.f;
        mode = VERIFY;
        coef = COEF_EXACT;
        continue;
      }
      // interior probes of the lowest survivors not yet probed
      mode = PROBE_MID;
      mj = 0;
      if (packed) {
        sel = lowest_bits(cand & ~mpr, 8);
        const int i = lane >> 2;
        cdur = i < __popc(sel) ? base + nth_bit(sel, i) : -1;
      } else {
        sel = cand & ~mpr;
        cdur = ((sel >> lane) & 1u) ? base + lane : -1;
      }
      coef = COEF_PLAIN;
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
    mode = PROBE_END;
    cand = 0u;
  }
}

// Duration-surrogate window rules shared by the window scans.  The window's
// centre is the grid index nearest exp(y0) on the log-spaced grid (logT0 =
// log T_0, dlog the log step), or the top index when the feasibility logit
// y1 says infeasible, clamped into [0, Kc).  The window's scan starts
// FN_WINDOW_BELOW grid steps below the centre (not below the window's own
// certificate index): the prediction's error on the synthetic workloads is
// within four steps for ~93 % of feasible edges.
#ifndef FN_WINDOW_BELOW
#define FN_WINDOW_BELOW 4
#endif
__device__ __forceinline__ int window_centre(float y0, float y1, float logT0, float dlog, int Kc) {
  int c;
  if (y1 < 0.f || !isfinite(y0)) c = Kc - 1;
  else c = __float2int_rn((y0 - logT0) / dlog);
  return min(max(c, 0), Kc - 1);
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
template <class Core>
__device__ __forceinline__ EdgeResult time_edge(const ArmK& A, const Core& core, float* es,
                                                float* split, bool finite, bool fixed, float Tp,
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
    const int res = edge_scan(A, core, es, split, sT, 0, S, true, Tp, exact, r.rt, r.rp, nsamp);
    if (res == FN_SCAN_ABORT) {
      r.k = FN_SCAN_ABORT;
      r.T = NAN;
      return r;
    }
    const bool pass = res == 0;
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
  r.k = edge_scan(A, core, es, split, sT, Kadm, S, false, 0.f, false, r.rt, r.rp, nsamp);
  if (r.k == FN_SCAN_ABORT) {
    r.T = NAN;
    r.rt = r.rp = NAN;
  } else if (r.k >= 0) {
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
