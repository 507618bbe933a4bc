// Schedule variants and the autotuner's cache.
//
// Each tunable launch has a small set of compiled variants (register budget /
// occupancy of the edge kernel, node-split of the parent search).  The cache
// maps (kind, shape bucket) -> variant; it is filled by fn_autotune_* calls,
// which time every variant on the caller's own workload, and read by every
// launch.  Untuned buckets use the default variant.
#pragma once

namespace fn {

enum TuneKind { TUNE_EDGES_FULL = 0, TUNE_EDGES_FIXED = 1, TUNE_PLAN_EDGES = 2, TUNE_KNN = 3 };

constexpr int kEdgeVariants = 3;  // __launch_bounds__ min blocks 2, 3, 4
constexpr int kDefaultEdgeVariant = 1;
// fn_time_edges has one more: the paired scan with its records in tensor
// memory (its default); kernels without it map that index to their default
constexpr int kPairEdgeVariant = 3;
constexpr int kTimeEdgeVariants = 4;
// the planner's edge body: the packed stages at the three register budgets,
// and (kPairEdgeVariant) one warp-per-edge launch on the paired core
constexpr int kPlanEdgeVariants = 4;

int tuned_variant(int kind, long n, int K, int S);
void set_tuned_variant(int kind, long n, int K, int S, int v);

}  // namespace fn
