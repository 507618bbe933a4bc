// Edge timing entry points: minimum feasible duration of cubic edges on a
// duration grid (Sec. IV-D, Def. "Minimum feasible time"), the same search
// guided by the duration surrogate's window, the fixed-duration check of
// goal candidates (Algorithm 1), and the torque dump used for parity.  The per-edge work is edge_core.cuh; this file holds the
// persistent kernels, their occupancy variants and the host entry points.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <unordered_map>

#include "edge_core.cuh"
#include "tm_scan.cuh"
#include "fn_internal.h"
#include "fn_tune.h"

namespace fn {

struct GridK {
  float T[FN_MAX_GRID];
};

// three warps per block keep the per-warp coefficient and link buffers
// (~12.6 KB) within a block's 48 KB of static shared memory
#define EDGE_WARPS 3

// Persistent: the grid is sized to the resident capacity and warp w takes
// edges w, w + W, w + 2W, ...  MINB sets the register budget (and so the
// occupancy) through __launch_bounds__; the tuner picks the variant.
template <int MINB>
__global__ void __launch_bounds__(32 * EDGE_WARPS, MINB)
    k_time_edges(ArmK A, GridK G, int K, int S, int mode, const float* __restrict__ s0,
                 const float* __restrict__ s1, int E, const float* __restrict__ Tparam,
                 int32_t* __restrict__ k_star, float* __restrict__ T_star,
                 float* __restrict__ rho3, uint8_t* __restrict__ ok,
                 unsigned long long* __restrict__ counter) {
  __shared__ float sT[FN_MAX_GRID];
  __shared__ float sEdge[EDGE_WARPS][32];
  __shared__ float sCoef[EDGE_WARPS][FN_CUBIC_WORDS * 32];
  __shared__ float sWr[EDGE_WARPS][FN_LINK_WORDS * 32];
  __shared__ __align__(16) float sSplit[EDGE_WARPS][FN_SPLIT_WORDS];
  __shared__ float4 sLink[7 * FN_LINK_F4];
  fill_links(A, sLink);
  if (mode == FN_MODE_FULL)
    for (int i = threadIdx.x; i < K; i += blockDim.x) sT[i] = G.T[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* es = sEdge[w];
  const CubicLane cb{&sCoef[w][lane]};
  const LaneLink wr{&sWr[w][lane]};
  const LinkTab L{sLink};
  const long W = (long)gridDim.x * EDGE_WARPS;
  unsigned nsamp = 0;
  for (long e = (long)blockIdx.x * EDGE_WARPS + w; e < E; e += W) {
    const bool finite = stage_rows(s0 + 16 * e, s1 + 16 * e, es);
    const bool fixed = mode == FN_MODE_FIXED;
    const float Tp = Tparam ? __ldg(Tparam + e) : INFINITY;
    const EdgeResult r =
        time_edge(A, ScalarCore{L, cb, wr}, es, sSplit[w], finite, fixed, Tp, sT, K, S, true, nsamp);
    if (lane == 0) {
      k_star[e] = r.k;
      T_star[e] = r.T;
      rho3[3 * e + 0] = r.rt;
      rho3[3 * e + 1] = r.rp;
      rho3[3 * e + 2] = r.rv;
      ok[e] = r.ok ? 1 : 0;
    }
  }
  if (counter && lane == 0 && nsamp) atomicAdd(counter, (unsigned long long)nsamp);
}

// The paired scan (two samples per lane, PairCore) with the per-link records
// of the torque evaluation in tensor memory, on tm_scan.cuh's block layout
// (one CTA of TM_WARPS warps per SM).  CTA b owns a contiguous range of the
// edges, which its warps claim in runs that shrink towards the end of the
// range (tm_claim): an edge's cost varies with the passes it needs, and
// shrinking runs keep the warps busy until the range is done.  A warp
// stages its run, computes the end-sample splits in one pass (split_group:
// up to sixty (edge, end, part) items on the lanes' two halves), then scans
// the edges one by one.
__global__ void __launch_bounds__(32 * TM_WARPS, 1)
    k_time_edges_tm(ArmK A, GridK G, int K, int S, int mode, const float* __restrict__ s0,
                    const float* __restrict__ s1, int E, const float* __restrict__ Tparam,
                    int32_t* __restrict__ k_star, float* __restrict__ T_star,
                    float* __restrict__ rho3, uint8_t* __restrict__ ok,
                    unsigned long long* __restrict__ counter) {
  extern __shared__ float4 tm_smem[];
  const TmBlock blk(tm_smem);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* sT = blk.grid;
  fill_links2(A, blk.link);
  const long per = ((long)E + gridDim.x - 1) / gridDim.x;
  const long r_lo = std::min<long>((long)blockIdx.x * per, E), r_hi = std::min<long>(r_lo + per, E);
  if (threadIdx.x == 0) *blk.next = 0;
  if (mode == FN_MODE_FULL)
    for (int i = threadIdx.x; i < K; i += blockDim.x) sT[i] = G.T[i];
  if (w == 0) tmem_alloc(blk.tmem, kTmCols);
  tmem_sync_block();
  const uint32_t tmem = *blk.tmem;
  const PairCore<TmemStash> core = blk.core(tmem, w, lane);
  float* es_g = blk.edges_of(w);
  float* split_g = blk.splits_of(w);
  const bool fixed = mode == FN_MODE_FIXED;
  const int len = (int)(r_hi - r_lo);
  unsigned nsamp = 0;
  for (;;) {
    int n;
    const int first = tm_claim(blk.next, len, n);
    if (n == 0) break;                               // warp-uniform
    const long e0 = r_lo + first;
    unsigned fin = 0u;
    for (int i = 0; i < n; ++i)
      if (stage_rows(s0 + 16 * (e0 + i), s1 + 16 * (e0 + i), es_g + 32 * i)) fin |= 1u << i;
    if (!fixed) split_group(A, core, es_g, split_g, n, nsamp);
    for (int i = 0; i < n; ++i) {
      const long e = e0 + i;
      const float Tp = Tparam ? __ldg(Tparam + e) : INFINITY;
      const EdgeResult r = time_edge(A, core, es_g + 32 * i, split_g + FN_SPLIT_WORDS * i,
                                     ((fin >> i) & 1u) != 0u, fixed, Tp, sT, K, S, true, nsamp);
      if (lane == 0) {
        k_star[e] = r.k;
        T_star[e] = r.T;
        rho3[3 * e + 0] = r.rt;
        rho3[3 * e + 1] = r.rp;
        rho3[3 * e + 2] = r.rv;
        ok[e] = r.ok ? 1 : 0;
      }
    }
  }
  if (counter && lane == 0 && nsamp) atomicAdd(counter, (unsigned long long)nsamp);
  tmem_sync_block();   // every warp's tensor-memory accesses precede the release
  if (w == 0) tmem_dealloc(tmem, kTmCols);
}

// ---------------------------------------------------------------------------
// Surrogate window on the paired core: the minimum feasible duration of each
// edge (Def. "Minimum feasible time") where a learned prediction of log T*
// names a window of W grid durations, [lo, lo + W) around the predicted
// index c, and the index a = lo - 1 below it carries the certificate.
//
// The window's outcome is the first feasible duration in [a, hi) (hi =
// min(lo + W, K)); it is accepted when it is at least lo (or lo = 0), "none"
// is accepted when the window reaches the top of the grid or T_{K-1} is
// infeasible, and otherwise the exact scan of the rest of the grid decides
// (below the window first, then T_{K-1}, then above the window).  The
// window is scanned from s = max(c - FN_WINDOW_BELOW, a) up, not from a: the scan
// of [s, hi) shows every duration below its result infeasible, so a result
// k > s is the window's outcome under the paper's monotonicity of the limit
// ratios in T (nothing below an infeasible duration is feasible), as is
// "none"; a feasible s sends the scan on to [a, s).  Starting near the
// prediction skips the interior probes of the end-sample survivors between
// a and the prediction, which is most of what the window saves over the
// full scan.  The block layout and the run claiming are those of
// k_time_edges_tm.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * TM_WARPS, 1)
    k_time_window_tm(ArmK A, GridK G, int K, int S, const float* __restrict__ s0,
                     const float* __restrict__ s1, int E, const float* __restrict__ Y, int Wn,
                     float logT0, float dlog, int32_t* __restrict__ k_star,
                     float* __restrict__ T_star, float* __restrict__ rho3,
                     uint8_t* __restrict__ ok, uint8_t* __restrict__ path,
                     unsigned long long* __restrict__ counter) {
  extern __shared__ float4 tm_smem[];
  const TmBlock blk(tm_smem);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* sT = blk.grid;
  fill_links2(A, blk.link);
  const long per = ((long)E + gridDim.x - 1) / gridDim.x;
  const long r_lo = std::min<long>((long)blockIdx.x * per, E), r_hi = std::min<long>(r_lo + per, E);
  if (threadIdx.x == 0) *blk.next = 0;
  for (int i = threadIdx.x; i < K; i += blockDim.x) sT[i] = G.T[i];
  if (w == 0) tmem_alloc(blk.tmem, kTmCols);
  tmem_sync_block();
  const uint32_t tmem = *blk.tmem;
  const PairCore<TmemStash> core = blk.core(tmem, w, lane);
  float* es_g = blk.edges_of(w);
  float* split_g = blk.splits_of(w);
  const int len = (int)(r_hi - r_lo);
  unsigned nsamp = 0;
  for (;;) {
    int n;
    const int first = tm_claim(blk.next, len, n);
    if (n == 0) break;                               // warp-uniform
    const long e0 = r_lo + first;
    unsigned fin = 0u;
    for (int i = 0; i < n; ++i)
      if (stage_rows(s0 + 16 * (e0 + i), s1 + 16 * (e0 + i), es_g + 32 * i)) fin |= 1u << i;
    split_group(A, core, es_g, split_g, n, nsamp);
    for (int i = 0; i < n; ++i) {
      const long e = e0 + i;
      float* es = es_g + 32 * i;
      float* split = split_g + FN_SPLIT_WORDS * i;
      int kres = -2, route = 1;
      float rt = NAN, rp = NAN;
      if ((fin >> i) & 1u) {
        const int c = window_centre(__ldg(Y + 2 * e), __ldg(Y + 2 * e + 1), logT0, dlog, K);
        const int lo = min(max(c - Wn / 2, 0), max(K - Wn, 0));
        const int hi = min(K, lo + Wn), a = max(lo - 1, 0);
        const int sc = min(max(c - FN_WINDOW_BELOW, a), hi);
        // FROM_S: [sc, hi); BELOW_S: [a, sc) after a feasible sc; the rest as the
        // plain window scan, entered with the window's outcome
        enum { FROM_S, BELOW_S, WIN, LOW_AFTER_WIN, LAST, LOW_AFTER_LAST, HIGH, DONE };
        int step = FROM_S, b0 = sc, b1 = hi, kalt = -1;
        float rt_alt = NAN, rp_alt = NAN;
        while (step != DONE) {
          float t1 = NAN, t2 = NAN;
          int k = (b1 > b0) ? edge_scan(A, core, es, split, sT, b1, S, false, 0.f, false, t1, t2,
                                        nsamp, b0)
                            : -1;
          if (k == FN_SCAN_ABORT) {
            kres = FN_SCAN_ABORT;
            break;
          }
          if (step == FROM_S) {
            if (k == sc && sc > a) {                 // sc feasible: the window below it
              kalt = k; rt_alt = t1; rp_alt = t2;
              step = BELOW_S; b0 = a; b1 = sc;
              continue;
            }
            step = WIN;                              // k: the window's outcome
          } else if (step == BELOW_S) {
            if (k < 0) { k = kalt; t1 = rt_alt; t2 = rp_alt; }
            step = WIN;
          }
          if (step == WIN) {
            if (k >= 0 && (k >= lo || lo == 0)) {
              kres = k; rt = t1; rp = t2; route = 0; step = DONE;
            } else if (k >= 0) {                     // T_{lo-1} feasible: look below it
              kalt = k; rt_alt = t1; rp_alt = t2;
              step = LOW_AFTER_WIN; b0 = 0; b1 = a;
            } else if (hi == K) {                    // window reaches the top: certified none
              kres = -1; route = 0; step = DONE;
            } else {
              step = LAST; b0 = K - 1; b1 = K;
            }
          } else if (step == LOW_AFTER_WIN) {
            if (k >= 0) { kres = k; rt = t1; rp = t2; }
            else { kres = kalt; rt = rt_alt; rp = rp_alt; }
            step = DONE;
          } else if (step == LAST) {
            if (k < 0) {                             // T_{K-1} infeasible: certified none
              kres = -1; route = 0; step = DONE;
            } else {
              kalt = k; rt_alt = t1; rp_alt = t2;
              step = LOW_AFTER_LAST; b0 = 0; b1 = a;
            }
          } else if (step == LOW_AFTER_LAST) {
            if (k >= 0) { kres = k; rt = t1; rp = t2; step = DONE; }
            else { step = HIGH; b0 = hi; b1 = K - 1; }
          } else {                                   // HIGH
            if (k >= 0) { kres = k; rt = t1; rp = t2; }
            else { kres = kalt; rt = rt_alt; rp = rp_alt; }
            step = DONE;
          }
        }
      }
      float rv = NAN, Ts = kres <= -2 ? NAN : INFINITY;
      if (kres >= 0) {
        Ts = sT[kres];
        rv = warp_rho_v(A, es, Ts);
      } else {
        rt = rp = NAN;
      }
      if (lane == 0) {
        k_star[e] = kres;
        T_star[e] = Ts;
        rho3[3 * e] = rt;
        rho3[3 * e + 1] = rp;
        rho3[3 * e + 2] = rv;
        ok[e] = (kres >= 0 && rv <= 1.f) ? 1 : 0;
        if (path) path[e] = (uint8_t)route;
      }
    }
  }
  if (counter && lane == 0 && nsamp) atomicAdd(counter, (unsigned long long)nsamp);
  tmem_sync_block();
  if (w == 0) tmem_dealloc(tmem, kTmCols);
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
    load_state(s0 + 4 * e, es.q0, es.qd0);
    load_state(s1 + 4 * e, es.q1, es.qd1);
    const float T = __ldg(Tv + e);
    Cubic c;
    cubic_coef<true>(es, T, c);
    float* out = tau + i * 7;
    torque_at(A, c, sample_u(s, S), [&](int j, float tq, float) { out[j] = tq; });
  }
}

typedef void (*EdgeKernel)(ArmK, GridK, int, int, int, const float*, const float*, int,
                           const float*, int32_t*, float*, float*, uint8_t*,
                           unsigned long long*);

static EdgeKernel edge_variant(int v) {
  switch (v) {
    case 0: return k_time_edges<2>;
    case 1: return k_time_edges<3>;
    default: return k_time_edges<4>;
  }
}

static int resident_blocks(EdgeKernel k) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * EDGE_WARPS, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * num_sms();
}

static fn_status launch_time_edges_tm(const ArmK& A, const GridK* G, int K, int S, int mode,
                                      const float* s0, const float* s1, int E,
                                      const float* Tparam, int32_t* k_star, float* T_star,
                                      float* rho3, uint8_t* ok, unsigned long long* counter,
                                      cudaStream_t st) {
  static std::once_flag once[64];
  static bool attr_ok[64];
  int dev = 0;
  cudaGetDevice(&dev);
  std::call_once(once[dev & 63], [&] {
    attr_ok[dev & 63] = cudaFuncSetAttribute(k_time_edges_tm,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kTmSmem) == cudaSuccess;
  });
  if (!attr_ok[dev & 63]) return FN_ECUDA;
  const long want = ((long)E + TM_WARPS - 1) / TM_WARPS;
  const int blocks = (int)std::max<long>(1, std::min<long>(want, num_sms()));
  static GridK empty;
  k_time_edges_tm<<<blocks, 32 * TM_WARPS, kTmSmem, st>>>(A, G ? *G : empty, K, S, mode, s0, s1, E,
                                                           Tparam, k_star, T_star, rho3, ok,
                                                           counter);
  return launch_status();
}

static fn_status launch_time_window_tm(const ArmK& A, const GridK& G, int K, int S,
                                       const float* s0, const float* s1, int E, const float* Y,
                                       int W, float logT0, float dlog, int32_t* k_star,
                                       float* T_star, float* rho3, uint8_t* ok, uint8_t* path,
                                       unsigned long long* counter, cudaStream_t st) {
  static std::once_flag once[64];
  static bool attr_ok[64];
  int dev = 0;
  cudaGetDevice(&dev);
  std::call_once(once[dev & 63], [&] {
    attr_ok[dev & 63] = cudaFuncSetAttribute(k_time_window_tm,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kTmSmem) == cudaSuccess;
  });
  if (!attr_ok[dev & 63]) return FN_ECUDA;
  const long want = ((long)E + TM_WARPS - 1) / TM_WARPS;
  const int blocks = (int)std::max<long>(1, std::min<long>(want, num_sms()));
  k_time_window_tm<<<blocks, 32 * TM_WARPS, kTmSmem, st>>>(A, G, K, S, s0, s1, E, Y, W, logT0,
                                                            dlog, k_star, T_star, rho3, ok, path,
                                                            counter);
  return launch_status();
}

fn_status launch_time_edges(const ArmK& A, const GridK* G, int K, int S, int mode,
                            const float* s0, const float* s1, int E, const float* Tparam,
                            int32_t* k_star, float* T_star, float* rho3, uint8_t* ok,
                            unsigned long long* counter, cudaStream_t st, int variant) {
  if (variant == kPairEdgeVariant)
    return launch_time_edges_tm(A, G, K, S, mode, s0, s1, E, Tparam, k_star, T_star, rho3, ok,
                                counter, st);
  EdgeKernel k = edge_variant(variant);
  const long want = ((long)E + EDGE_WARPS - 1) / EDGE_WARPS;
  const int blocks = (int)std::max<long>(1, std::min<long>(want, resident_blocks(k)));
  static GridK empty;
  k<<<blocks, 32 * EDGE_WARPS, 0, st>>>(A, G ? *G : empty, K, S, mode, s0, s1, E, Tparam, k_star,
                                         T_star, rho3, ok, counter);
  return launch_status();
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
  if (mode == FN_MODE_FULL) {
    if (!T_grid || K < 1 || K > FN_MAX_GRID) return FN_EINVAL;
    GridK G;
    for (int k = 0; k < K; ++k) {
      if (!(T_grid[k] > 0.f) || !std::isfinite(T_grid[k])) return FN_EINVAL;
      if (k > 0 && !(T_grid[k] > T_grid[k - 1])) return FN_EINVAL;
      G.T[k] = T_grid[k];
    }
    const int v = tuned_variant(TUNE_EDGES_FULL, E, K, S);
    return launch_time_edges(A, &G, K, S, mode, s0, s1, E, T_cap, k_star, T_star, rho3, ok,
                             sample_count, st, v);
  }
  if (!T_fixed) return FN_EINVAL;
  const int v = tuned_variant(TUNE_EDGES_FIXED, E, 1, S);
  return launch_time_edges(A, nullptr, 0, S, mode, s0, s1, E, T_fixed, k_star, T_star, rho3, ok,
                           sample_count, st, v);
}

extern "C" fn_status fn_time_edges(const fn_arm_t* arm, const float* s0, const float* s1, int E,
                                   const float* T_grid, int K, int S, int mode,
                                   const float* T_fixed, const float* T_cap, int32_t* k_star,
                                   float* T_star, float* rho3, uint8_t* ok, void* stream) {
  return fn_time_edges_counted(arm, s0, s1, E, T_grid, K, S, mode, T_fixed, T_cap, k_star, T_star,
                               rho3, ok, nullptr, stream);
}

extern "C" fn_status fn_time_edges_window(const fn_arm_t* arm, const float* s0, const float* s1,
                                          int E, const float* T_grid, int K, int S,
                                          const float* Y, int W, int32_t* k_star, float* T_star,
                                          float* rho3, uint8_t* ok, uint8_t* path,
                                          unsigned long long* sample_count, void* stream) {
  ArmK A;
  if (!make_armk(arm, &A)) return FN_EINVAL;
  if (E < 0 || S < 2 || S > FN_MAX_S || K < 2 || K > FN_MAX_GRID || W < 1) return FN_EINVAL;
  if (E == 0) return FN_OK;
  if (!s0 || !s1 || !T_grid || !Y || !k_star || !T_star || !rho3 || !ok) return FN_EINVAL;
  if (!aligned16(s0) || !aligned16(s1)) return FN_EINVAL;
  GridK G;
  for (int k = 0; k < K; ++k) {
    if (!(T_grid[k] > 0.f) || !std::isfinite(T_grid[k])) return FN_EINVAL;
    if (k > 0 && !(T_grid[k] > T_grid[k - 1])) return FN_EINVAL;
    G.T[k] = T_grid[k];
  }
  const float logT0 = std::log(T_grid[0]);
  const float dlog = (std::log(T_grid[K - 1]) - logT0) / (float)(K - 1);
  return launch_time_window_tm(A, G, K, S, s0, s1, E, Y, std::min(W, K), logT0, dlog, k_star,
                               T_star, rho3, ok, path, sample_count, (cudaStream_t)stream);
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
