// Edge timing: minimum feasible duration of cubic edges on a duration grid
// (Sec. IV-D, Def. "Minimum feasible time"), the fixed-duration check of
// goal candidates (Algorithm 1), and the torque dump used for parity.
//
// Work decomposition (one warp per edge):
//   1. probe: the 32 lanes take 32 consecutive grid durations and evaluate
//      the two end samples (t = 0 and t = T).  A violation at either end
//      proves that duration infeasible.  The ends carry the largest
//      accelerations of a cubic, so most short durations fail here after two
//      torque evaluations instead of S.
//   2. verify: the surviving durations are taken in ascending order; for each
//      the lanes evaluate all S samples (S/32 per lane) with a warp-ballot
//      exit at the first violating batch.  The first duration that passes
//      every sample is k*: each lower index was shown infeasible by a
//      violating sample, so no monotonicity in T is assumed.
//   3. rho_v at T_{k*}: lane j < 7 takes joint j's exact velocity extremum.
#include <cuda_runtime.h>

#include "fn_arm.cuh"
#include "fn_internal.h"

namespace fn {

struct GridK {
  float T[FN_MAX_GRID];
};

__device__ __forceinline__ float sample_time(float T, int s, int S) {
  // t_s = T * (s / (S-1)): exact at both ends (t_0 = 0, t_{S-1} = T)
  return T * (__int2float_rn(s) / __int2float_rn(S - 1));
}

// full S-sample check of one duration with lanes = samples.
// exit_early: stop at the first batch with a violation (result then only
// says "infeasible").  Returns true if every sample passes; rt/rp are the
// warp maxima over the evaluated samples.
__device__ __forceinline__ bool verify_duration(const ArmK& A, const float* es, float T, int S,
                                                bool exit_early, float& rt, float& rp,
                                                unsigned& nsamp) {
  const int lane = threadIdx.x & 31;
  Cubic c;
  cubic_coef_sh(es, T, c);
  float mt = 0.f, mp = 0.f;
  bool bad = false;
  for (int s0 = 0; s0 < S; s0 += 32) {
    const int s = s0 + lane;
    bool viol = false;
    if (s < S) {
      float a, b;
      sample_ratios(A, c, sample_time(T, s, S), a, b);
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
  Cubic c;
  cubic_coef_sh(es, T, c);
  float r = 0.f;
#pragma unroll
  for (int j = 0; j < 7; ++j)
    if (lane == j) r = rho_v_joint(A, c, j, T);
  return warp_max(r);
}

__device__ __forceinline__ void load_edge(const float4* s0, const float4* s1, long e,
                                          EdgeStates& es) {
  load_state(s0 + 4 * e, es.q0, es.qd0);
  load_state(s1 + 4 * e, es.q1, es.qd1);
}

// Stage edge e in the warp's shared slot (32 floats: s0 row then s1 row) and
// report whether all 28 state values are finite.
__device__ __forceinline__ bool stage_edge(const float* s0, const float* s1, long e, float* sh) {
  const int lane = threadIdx.x & 31;
  const float v = lane < 16 ? __ldg(s0 + 16 * e + lane) : __ldg(s1 + 16 * e + (lane - 16));
  __syncwarp();
  sh[lane] = v;
  __syncwarp();
  const bool pad = (lane & 7) == 7;
  return __all_sync(0xffffffffu, pad || isfinite(v));
}

// k* search of one edge over grid indices [0, Kadm) (all lanes participate).
// nsamp counts the torque evaluations of the warp (probe ends + verify samples).
__device__ __forceinline__ int first_feasible(const ArmK& A, const float* es,
                                              const float* sT, int Kadm, int S, float& rt,
                                              float& rp, unsigned& nsamp) {
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < Kadm; base += 32) {
    const int k = base + lane;
    bool first_end = false, pass = false;
    if (k < Kadm) {
      const float T = sT[k];
      Cubic c;
      cubic_coef_sh(es, T, c);
      float a, b;
      sample_ratios(A, c, 0.f, a, b);
      first_end = (a <= 1.f && b <= 1.f);
      if (first_end) {
        sample_ratios(A, c, T, a, b);
        pass = (a <= 1.f && b <= 1.f);
      }
    }
    nsamp += min(32, Kadm - base) + __popc(__ballot_sync(0xffffffffu, first_end));
    unsigned mask = __ballot_sync(0xffffffffu, pass);
    while (mask) {
      const int kk = base + __ffs(mask) - 1;
      if (verify_duration(A, es, sT[kk], S, true, rt, rp, nsamp)) return kk;
      mask &= mask - 1;
    }
  }
  return -1;
}

__global__ void __launch_bounds__(128) k_time_full(ArmK A, GridK G, int K, int S,
                                                   const float4* __restrict__ s0,
                                                   const float4* __restrict__ s1, int E,
                                                   const float* __restrict__ T_cap,
                                                   int32_t* __restrict__ k_star,
                                                   float* __restrict__ T_star,
                                                   float* __restrict__ rho3,
                                                   uint8_t* __restrict__ ok,
                                                   unsigned long long* __restrict__ counter) {
  __shared__ float sT[FN_MAX_GRID];
  __shared__ float sEdge[4][32];
  for (int i = threadIdx.x; i < K; i += blockDim.x) sT[i] = G.T[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  float* es = sEdge[threadIdx.x >> 5];
  const long warps = (long)gridDim.x * (blockDim.x >> 5);
  for (long e = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < E; e += warps) {
    const bool finite = stage_edge((const float*)s0, (const float*)s1, e, es);
    int kres;
    float rt = NAN, rp = NAN, rv = NAN, Ts;
    if (!finite) {
      kres = -2;
      Ts = NAN;
    } else {
      int Kadm = K;
      if (T_cap) {
        const float cap = __ldg(T_cap + e);
        // admissible prefix of the ascending grid: T_k <= cap
        int cnt = 0;
        for (int b = 0; b < K; b += 32) {
          const int k = b + lane;
          cnt += __popc(__ballot_sync(0xffffffffu, k < K && sT[k] <= cap));
        }
        Kadm = cnt;
      }
      unsigned nsamp = 0;
      kres = first_feasible(A, es, sT, Kadm, S, rt, rp, nsamp);
      if (counter && lane == 0) atomicAdd(counter, (unsigned long long)nsamp);
      if (kres >= 0) {
        Ts = sT[kres];
        rv = warp_rho_v(A, es, Ts);
      } else {
        Ts = INFINITY;
        rt = rp = NAN;
      }
    }
    if (lane == 0) {
      k_star[e] = kres;
      T_star[e] = Ts;
      rho3[3 * e + 0] = rt;
      rho3[3 * e + 1] = rp;
      rho3[3 * e + 2] = rv;
      ok[e] = (kres >= 0 && rv <= 1.f) ? 1 : 0;
    }
  }
}

__global__ void __launch_bounds__(128) k_time_fixed(ArmK A, int S, const float4* __restrict__ s0,
                                                    const float4* __restrict__ s1, int E,
                                                    const float* __restrict__ T_fixed,
                                                    int32_t* __restrict__ k_star,
                                                    float* __restrict__ T_star,
                                                    float* __restrict__ rho3,
                                                    uint8_t* __restrict__ ok,
                                                    unsigned long long* __restrict__ counter) {
  __shared__ float sEdge[4][32];
  const int lane = threadIdx.x & 31;
  float* es = sEdge[threadIdx.x >> 5];
  const long warps = (long)gridDim.x * (blockDim.x >> 5);
  for (long e = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < E; e += warps) {
    const bool finite = stage_edge((const float*)s0, (const float*)s1, e, es);
    const float T = __ldg(T_fixed + e);
    int kres;
    float rt = NAN, rp = NAN, rv = NAN, Ts = T;
    if (!finite || !(isfinite(T) && T > 0.f)) {
      kres = -2;
      Ts = NAN;
    } else {
      unsigned nsamp = 0;
      const bool pass = verify_duration(A, es, T, S, false, rt, rp, nsamp);
      if (counter && lane == 0) atomicAdd(counter, (unsigned long long)nsamp);
      rv = warp_rho_v(A, es, T);
      kres = pass ? 0 : -1;
    }
    if (lane == 0) {
      k_star[e] = kres;
      T_star[e] = Ts;
      rho3[3 * e + 0] = rt;
      rho3[3 * e + 1] = rp;
      rho3[3 * e + 2] = rv;
      ok[e] = (kres == 0 && rv <= 1.f) ? 1 : 0;
    }
  }
}

// tau[e][s][j]: one thread per (edge, sample)
__global__ void __launch_bounds__(128) k_rnea_dump(ArmK A, const float4* __restrict__ s0,
                                                   const float4* __restrict__ s1,
                                                   const float* __restrict__ Tv, int E, int S,
                                                   float* __restrict__ tau) {
  const long n = (long)E * S;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const long e = i / S;
    const int s = (int)(i - e * S);
    EdgeStates es;
    load_edge(s0, s1, e, es);
    const float T = __ldg(Tv + e);
    Cubic c;
    cubic_coef(es, T, c);
    float* out = tau + i * 7;
    torque_at(A, c, sample_time(T, s, S), [&](int j, float tq, float) { out[j] = tq; });
  }
}

}  // namespace fn

using namespace fn;

extern "C" fn_status fn_time_edges_counted(const fn_arm_t* arm, const float* s0, const float* s1,
                                           int E, const float* T_grid, int K, int S, int mode,
                                           const float* T_fixed, const float* T_cap,
                                           int32_t* k_star, float* T_star, float* rho3,
                                           uint8_t* ok, unsigned long long* sample_count,
                                           void* stream) {
  ArmK A;
  if (!make_armk(arm, &A)) return FN_EINVAL;
  if (E < 0 || S < 2 || S > FN_MAX_S) return FN_EINVAL;
  if (mode != FN_MODE_FULL && mode != FN_MODE_FIXED) return FN_EINVAL;
  if (E == 0) return FN_OK;
  if (!s0 || !s1 || !k_star || !T_star || !rho3 || !ok) return FN_EINVAL;
  if (!aligned16(s0) || !aligned16(s1)) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int threads = 128;
  const int wpb = threads / 32;
  if (mode == FN_MODE_FULL) {
    if (!T_grid || K < 1 || K > FN_MAX_GRID) return FN_EINVAL;
    GridK G;
    for (int k = 0; k < K; ++k) {
      if (!(T_grid[k] > 0.f) || !isfinite(T_grid[k])) return FN_EINVAL;
      if (k > 0 && !(T_grid[k] > T_grid[k - 1])) return FN_EINVAL;
      G.T[k] = T_grid[k];
    }
    const long blocks = std::min<long>(((long)E + wpb - 1) / wpb, 1L << 20);
    k_time_full<<<(unsigned)blocks, threads, 0, st>>>(A, G, K, S, (const float4*)s0,
                                                     (const float4*)s1, E, T_cap, k_star, T_star,
                                                     rho3, ok, sample_count);
  } else {
    if (!T_fixed) return FN_EINVAL;
    const long blocks = std::min<long>(((long)E + wpb - 1) / wpb, 1L << 20);
    k_time_fixed<<<(unsigned)blocks, threads, 0, st>>>(A, S, (const float4*)s0, (const float4*)s1,
                                                      E, T_fixed, k_star, T_star, rho3, ok,
                                                      sample_count);
  }
  return launch_status();
}

extern "C" fn_status fn_time_edges(const fn_arm_t* arm, const float* s0, const float* s1, int E,
                                   const float* T_grid, int K, int S, int mode,
                                   const float* T_fixed, const float* T_cap, int32_t* k_star,
                                   float* T_star, float* rho3, uint8_t* ok, void* stream) {
  return fn_time_edges_counted(arm, s0, s1, E, T_grid, K, S, mode, T_fixed, T_cap, k_star, T_star,
                               rho3, ok, nullptr, stream);
}

extern "C" fn_status fn_rnea_dump(const fn_arm_t* arm, const float* s0, const float* s1,
                                  const float* T, int E, int S, float* tau, void* stream) {
  ArmK A;
  if (!make_armk(arm, &A)) return FN_EINVAL;
  if (E < 0 || S < 2 || S > FN_MAX_S) return FN_EINVAL;
  if (E == 0) return FN_OK;
  if (!s0 || !s1 || !T || !tau || !aligned16(s0) || !aligned16(s1)) return FN_EINVAL;
  const long n = (long)E * S;
  const long blocks = std::min<long>((n + 127) / 128, 1L << 20);
  k_rnea_dump<<<(unsigned)blocks, 128, 0, (cudaStream_t)stream>>>(A, (const float4*)s0,
                                                                  (const float4*)s1, T, E, S, tau);
  return launch_status();
}
