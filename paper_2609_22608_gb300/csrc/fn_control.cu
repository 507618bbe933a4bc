// Control-side entry points of Sec. IV-F and Sec. IV-E:
//   fn_controller_torque  the tracking controller of Eq. (controller): the
//                         cubic refitted from the measured state to the
//                         rendezvous, its initial acceleration clipped to the
//                         taper box, Eq. (torque), then the torque, power and
//                         slew clips; one thread per controller instance;
//   fn_check_edges_full   the full-resolution recheck of a plan's edges at
//                         their own durations: all three ratios of Def.
//                         "Feasibility Check" over S samples and the
//                         clearance over S_clear points; one warp per edge.
#include <cuda_runtime.h>

#include "edge_core.cuh"
#include "fn_internal.h"
#include "fn_kin.cuh"

namespace fn {

// the limits the controller clips to, exactly as given (ArmK keeps only
// their reciprocals)
struct CtrlK {
  float tau_max[7];
  float w_max;
  float dslew[7];   // rate_j * dt
  float dt;
};

#define CTRL_ACC 1
#define CTRL_TORQUE 2
#define CTRL_POWER 4
#define CTRL_SLEW 8
#define CTRL_INVALID 0x80

__global__ void __launch_bounds__(128) k_controller(ArmK A, CtrlK L, int B,
                                                    const float* __restrict__ state,
                                                    const float* __restrict__ goal,
                                                    const float* __restrict__ Th,
                                                    const float* __restrict__ tau_prev,
                                                    float* __restrict__ tau,
                                                    float* __restrict__ qdd_out,
                                                    uint8_t* __restrict__ flags) {
  for (long b = (long)blockIdx.x * blockDim.x + threadIdx.x; b < B;
       b += (long)gridDim.x * blockDim.x) {
    EdgeStates es;
    bool fin = true;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      es.q0[j] = state[16 * b + j];
      es.qd0[j] = state[16 * b + 8 + j];
      es.q1[j] = goal[16 * b + j];
      es.qd1[j] = goal[16 * b + 8 + j];
      fin = fin && isfinite(es.q0[j]) && isfinite(es.qd0[j]) && isfinite(es.q1[j]) &&
            isfinite(es.qd1[j]);
    }
    const float T = Th[b];
    if (!fin || !(isfinite(T) && T > 0.f)) {
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        tau[7 * b + j] = NAN;
        if (qdd_out) qdd_out[7 * b + j] = NAN;
      }
      if (flags) flags[b] = CTRL_INVALID;
      continue;
    }
    unsigned f = 0;
    // Eq. (controller): the refitted cubic's acceleration at t = 0,
    // 2 b2 / T^2 = 6 (q_g - q) / T^2 - (4 qd + 2 qd_g) / T, from the
    // compensated coefficients (the two terms cancel on short horizons)
    Cubic cu;
    cubic_coef<true>(es, T, cu);
    PointCoef pc;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      float q, v, a;
      cubic_eval(cu, j, 0.f, q, v, a);
      // the box keeping the velocity after one period inside the taper
      const float bound = taper(A, j, es.q0[j]);
      const float lo = (-bound - es.qd0[j]) / L.dt, hi = (bound - es.qd0[j]) / L.dt;
      const float c = fminf(fmaxf(a, lo), hi);
      if (c != a) f |= CTRL_ACC;
      pc.q[j] = es.q0[j];
      pc.qd[j] = es.qd0[j];
      pc.qdd[j] = c;
      if (qdd_out) qdd_out[7 * b + j] = c;
    }
    float t7[7];
    torque_at(A, pc, 0.f, [&](int j, float tq, float) { t7[j] = tq; });
    float pw = 0.f;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      const float m = L.tau_max[j];
      const float c = fminf(fmaxf(t7[j], -m), m);
      if (c != t7[j]) f |= CTRL_TORQUE;
      t7[j] = c;
      pw = fmaf(c, es.qd0[j], pw);
    }
    if (fabsf(pw) > L.w_max) {
      const float sc = L.w_max / fabsf(pw);
#pragma unroll
      for (int j = 0; j < 7; ++j) t7[j] *= sc;
      f |= CTRL_POWER;
    }
    if (tau_prev) {
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        const float p = tau_prev[7 * b + j];
        const float c = fminf(fmaxf(t7[j], p - L.dslew[j]), p + L.dslew[j]);
        if (c != t7[j]) f |= CTRL_SLEW;
        t7[j] = c;
      }
    }
#pragma unroll
    for (int j = 0; j < 7; ++j) tau[7 * b + j] = t7[j];
    if (flags) flags[b] = (uint8_t)f;
  }
}

#define CHECK_WARPS 3  // as the grid scan: static shared memory within 48 KB

// one warp per edge: the exact fixed-duration check (all S samples), rho_v,
// then the clearance (lane = point)
__global__ void __launch_bounds__(32 * CHECK_WARPS, 3)
    k_check_edges(ArmK A, fn_problem_t P, int E, const int* __restrict__ E_dev, int S,
                  int S_clear, float margin, const float* __restrict__ s0,
                  const float* __restrict__ s1, const float* __restrict__ Tv,
                  float* __restrict__ rho3, float* __restrict__ clearance,
                  uint8_t* __restrict__ ok) {
  __shared__ float sEdge[CHECK_WARPS][32];
  __shared__ float sCoef[CHECK_WARPS][FN_CUBIC_WORDS * 32];
  __shared__ float sWr[CHECK_WARPS][FN_LINK_WORDS * 32];
  __shared__ float4 sLink[7 * FN_LINK_F4];
  fill_links(A, sLink);
  __syncthreads();
  if (E_dev) E = min(E, max(*E_dev, 0));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* es = sEdge[w];
  const CubicLane cb{&sCoef[w][lane]};
  const LaneLink wr{&sWr[w][lane]};
  const LinkTab L{sLink};
  unsigned nsamp = 0;
  for (long e = (long)blockIdx.x * CHECK_WARPS + w; e < E; e += (long)gridDim.x * CHECK_WARPS) {
    const bool finite = stage_rows(s0 + 16 * e, s1 + 16 * e, es);
    const float T = Tv[e];
    if (!finite || !(isfinite(T) && T > 0.f)) {
      if (lane == 0) {
        rho3[3 * e] = rho3[3 * e + 1] = rho3[3 * e + 2] = NAN;
        clearance[e] = NAN;
        ok[e] = 0;
      }
      continue;
    }
    float rt = NAN, rp = NAN;
    if (edge_scan(A, ScalarCore{L, cb, wr}, es, nullptr, nullptr, 0, S, true, T, true, rt, rp, nsamp) ==
        FN_SCAN_ABORT)
      rt = rp = NAN;   // the scan's pass bound (never expected): not ok
    const float rv = warp_rho_v(A, es, T);
    float cl = INFINITY;
    if (P.n_obs > 0) {
      Cubic c;
      cubic_coef_sh<true>(es, T, c);
      float mc = INFINITY;
#pragma unroll 1
      for (int s = lane; s < S_clear; s += 32) {
        const float u = sample_u(s, S_clear);
        float q[7];
#pragma unroll
        for (int j = 0; j < 7; ++j) {
          float v, a;
          cubic_eval(c, j, u, q[j], v, a);
        }
        mc = fminf(mc, config_clearance(A, q, P));
      }
      cl = -warp_max(-mc);
    }
    if (lane == 0) {
      rho3[3 * e] = rt;
      rho3[3 * e + 1] = rp;
      rho3[3 * e + 2] = rv;
      clearance[e] = cl;
      ok[e] = (rt <= 1.f && rp <= 1.f && rv <= 1.f && (P.n_obs == 0 || cl >= margin)) ? 1 : 0;
    }
  }
}

}  // namespace fn

using namespace fn;

extern "C" fn_status fn_controller_torque(const fn_arm_t* arm, int B, const float* state,
                                          const float* goal, const float* T,
                                          const float* tau_prev, float dt,
                                          const float* tau_rate_max, float* tau, float* qdd_des,
                                          uint8_t* flags, void* stream) {
  ArmK A;
  if (!make_armk(arm, &A)) return FN_EINVAL;
  if (B < 0 || !(dt > 0.f) || !std::isfinite(dt)) return FN_EINVAL;
  if (tau_prev && !tau_rate_max) return FN_EINVAL;
  CtrlK L;
  for (int j = 0; j < 7; ++j) {
    L.tau_max[j] = arm->tau_max[j];
    L.dslew[j] = 0.f;
    if (tau_prev) {
      if (!(tau_rate_max[j] >= 0.f) || !std::isfinite(tau_rate_max[j])) return FN_EINVAL;
      L.dslew[j] = tau_rate_max[j] * dt;
    }
  }
  L.w_max = arm->w_max;
  L.dt = dt;
  if (B == 0) return FN_OK;
  if (!state || !goal || !T || !tau) return FN_EINVAL;
  const int blocks = (int)std::min<long>(((long)B + 127) / 128, 8L * num_sms());
  k_controller<<<blocks, 128, 0, (cudaStream_t)stream>>>(A, L, B, state, goal, T, tau_prev, tau,
                                                         qdd_des, flags);
  return launch_status();
}

extern "C" fn_status fn_check_edges_full(const fn_arm_t* arm, const float* s0, const float* s1,
                                         const float* T, int E, const int* E_dev, int S,
                                         int S_clear, int n_obs, const float* obs, float margin,
                                         float* rho3, float* clearance, uint8_t* ok,
                                         void* stream) {
  ArmK A;
  if (!make_armk(arm, &A)) return FN_EINVAL;
  if (E < 0 || S < 2 || S > FN_MAX_S) return FN_EINVAL;
  if (n_obs < 0 || n_obs > FN_MAX_OBS || (n_obs > 0 && (!obs || S_clear < 2))) return FN_EINVAL;
  if (!std::isfinite(margin)) return FN_EINVAL;
  fn_problem_t P;
  memset(&P, 0, sizeof(P));
  P.n_obs = n_obs;
  for (int b = 0; b < n_obs; ++b)
    for (int c = 0; c < 4; ++c) P.obs[b][c] = obs[4 * b + c];
  if (E == 0) return FN_OK;
  if (!s0 || !s1 || !T || !rho3 || !clearance || !ok) return FN_EINVAL;
  if (!aligned16(s0) || !aligned16(s1)) return FN_EINVAL;
  const long want = ((long)E + CHECK_WARPS - 1) / CHECK_WARPS;
  const int blocks = (int)std::max<long>(1, std::min<long>(want, 3L * num_sms()));
  k_check_edges<<<blocks, 32 * CHECK_WARPS, 0, (cudaStream_t)stream>>>(
      A, P, E, E_dev, S, S_clear, margin, s0, s1, T, rho3, clearance, ok);
  return launch_status();
}
