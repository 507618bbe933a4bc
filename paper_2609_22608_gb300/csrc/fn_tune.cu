// Autotuner: variant cache and the timing loop of fn_autotune_time_edges.
#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "fn_arm.cuh"
#include "fn_internal.h"
#include "fn_tune.h"

namespace fn {

static std::mutex g_mu;
static std::map<std::tuple<int, int, int, int, int>, int> g_cache;

static int bucket(long n) {
  int b = 0;
  while (n > 1 && b < 40) { n = (n + 1) / 2; ++b; }
  return b;
}

static int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

int tuned_variant(int kind, long n, int K, int S) {
  std::lock_guard<std::mutex> g(g_mu);
  auto it = g_cache.find(std::make_tuple(current_device(), kind, bucket(n), K, S));
  if (it != g_cache.end()) return it->second;
  if (kind == TUNE_KNN) return 0;
  return (kind == TUNE_EDGES_FULL || kind == TUNE_EDGES_FIXED) ? kPairEdgeVariant
                                                               : kDefaultEdgeVariant;
}

void set_tuned_variant(int kind, long n, int K, int S, int v) {
  std::lock_guard<std::mutex> g(g_mu);
  g_cache[std::make_tuple(current_device(), kind, bucket(n), K, S)] = v;
}

struct GridK;
fn_status launch_time_edges(const ArmK& A, const GridK* G, int K, int S, int mode,
                            const float* s0, const float* s1, int E, const float* Tparam,
                            int32_t* k_star, float* T_star, float* rho3, uint8_t* ok,
                            unsigned long long* counter, cudaStream_t st, int variant);

}  // namespace fn

using namespace fn;

extern "C" fn_status fn_time_edges_counted(const fn_arm_t* arm, const float* s0, const float* s1,
                                           int E, const float* T_grid, int K, int S, int mode,
                                           const float* T_fixed, const float* T_cap,
                                           int32_t* k_star, float* T_star, float* rho3,
                                           uint8_t* ok, unsigned long long* sample_count,
                                           void* stream);

extern "C" fn_status fn_time_edges_set_variant(int mode, int E, int K, int S, int variant) {
  if (mode != FN_MODE_FULL && mode != FN_MODE_FIXED) return FN_EINVAL;
  if (variant < 0 || variant >= kTimeEdgeVariants) return FN_EINVAL;
  if (E < 1 || S < 2 || S > FN_MAX_S) return FN_EINVAL;
  if (mode == FN_MODE_FULL && (K < 1 || K > FN_MAX_GRID)) return FN_EINVAL;
  const bool full = mode == FN_MODE_FULL;
  set_tuned_variant(full ? TUNE_EDGES_FULL : TUNE_EDGES_FIXED, E, full ? K : 1, S, variant);
  return FN_OK;
}

extern "C" fn_status fn_autotune_time_edges(const fn_arm_t* arm, const float* s0,
                                            const float* s1, int E, const float* T_grid, int K,
                                            int S, int mode, const float* T_fixed,
                                            const float* T_cap, int32_t* k_star, float* T_star,
                                            float* rho3, uint8_t* ok, int reps, int* chosen,
                                            float* variant_ms, void* stream) {
  if (reps < 1 || E <= 0) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int kind = mode == FN_MODE_FULL ? TUNE_EDGES_FULL : TUNE_EDGES_FIXED;
  const int Kb = mode == FN_MODE_FULL ? K : 1;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return FN_ECUDA;
  int best = kPairEdgeVariant;
  float best_ms = INFINITY;
  fn_status rc = FN_OK;
  for (int v = 0; v < kTimeEdgeVariants && rc == FN_OK; ++v) {
    set_tuned_variant(kind, E, Kb, S, v);
    // one untimed run, then `reps` timed runs
    rc = fn_time_edges_counted(arm, s0, s1, E, T_grid, K, S, mode, T_fixed, T_cap, k_star,
                               T_star, rho3, ok, nullptr, stream);
    cudaEventRecord(a, st);
    for (int r = 0; r < reps && rc == FN_OK; ++r)
      rc = fn_time_edges_counted(arm, s0, s1, E, T_grid, K, S, mode, T_fixed, T_cap, k_star,
                                 T_star, rho3, ok, nullptr, stream);
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess) rc = FN_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    ms /= reps;
    if (variant_ms) variant_ms[v] = ms;
    if (ms < best_ms) { best_ms = ms; best = v; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  set_tuned_variant(kind, E, Kb, S, best);
  if (chosen) *chosen = best;
  return rc;
}
