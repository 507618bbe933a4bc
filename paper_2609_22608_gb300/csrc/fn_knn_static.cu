// Nearest-parent search for callers that cannot allocate device memory.
//
// fn_knn_tree needs a caller-supplied workspace for its split pass.  Some
// callers cannot provide one: a real-time planning thread that must not
// enter the driver's allocator mid-cycle (cudaMalloc can synchronise the
// device and take milliseconds, far beyond a 20 ms planning budget), or an
// embedded host whose device memory is fully budgeted at start-up.  This
// variant keeps its scratch in a fixed file-scope device array instead, so a
// call allocates nothing.
#include <cuda_runtime.h>

#include <mutex>

#include "fn_internal.h"

namespace fn {
fn_status knn_launch(const float* tree, int N, int first, const float* queries, int B, int k,
                     float w_vel, int32_t* idx, float* d2, int nsplit, float* part_d,
                     int32_t* part_i, cudaStream_t st);
int knn_km(int k);
int knn_nsplit(int B, int N);
}  // namespace fn

using namespace fn;

// Scratch of the split pass: per split, query and list slot one distance
// (f32) and one node index (i32).  Every device that loads the library holds
// this array until the process exits.
#define FN_KNN_STATIC_SCRATCH_BYTES ((size_t)16 << 20)
static __device__ __align__(256) unsigned char g_knn_scratch[FN_KNN_STATIC_SCRATCH_BYTES];

#define FN_KNN_STATIC_DEVICES 64
static std::mutex g_scratch_mu;
static void* g_scratch_ptr[FN_KNN_STATIC_DEVICES];

// Device address of the array on the current device (host code may not use
// the symbol itself: in host code it names a host-side stand-in).  Taken
// once per device, on that device's first call.
static fn_status static_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FN_ECUDA;
  if (dev < 0 || dev >= FN_KNN_STATIC_DEVICES) return FN_EINVAL;
  std::lock_guard<std::mutex> g(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_knn_scratch) != cudaSuccess || !p) return FN_ECUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return FN_OK;
}

extern "C" fn_status fn_knn_tree_static(const float* tree, int N, int first, const float* queries,
                                        int B, int k, float w_vel, int32_t* idx, float* d2,
                                        void* stream) {
  if (N < 0 || first < 0 || first > N || B < 0 || k < 1 || k > FN_MAX_KNN) return FN_EINVAL;
  if (B > FN_KNN_STATIC_MAX_QUERIES) return FN_EINVAL;
  if (!(w_vel >= 0.f) || !std::isfinite(w_vel)) return FN_EINVAL;
  if (B == 0) return FN_OK;
  if (!queries || !idx || !d2 || !aligned16(queries)) return FN_EINVAL;
  if (N > first && (!tree || !aligned16(tree))) return FN_EINVAL;
  void* scratch = nullptr;
  fn_status rc = static_scratch(&scratch);
  if (rc != FN_OK) return rc;
  const size_t km = (size_t)knn_km(k);
  // as many node splits as the array holds (at least two fit for any
  // B <= FN_KNN_STATIC_MAX_QUERIES), at most what the shape asks for
  const size_t per_split = (size_t)B * km;
  auto bytes_for = [&](size_t ns) {
    return ((ns * per_split * sizeof(float) + 255) & ~(size_t)255) + ns * per_split * sizeof(int32_t);
  };
  int nsplit = knn_nsplit(B, N);
  while (nsplit > 1 && bytes_for((size_t)nsplit) > FN_KNN_STATIC_SCRATCH_BYTES) --nsplit;
  float* part_d = nullptr;
  int32_t* part_i = nullptr;
  if (nsplit > 1) {
    part_d = (float*)scratch;
    part_i = (int32_t*)((char*)scratch +
                        (((size_t)nsplit * per_split * sizeof(float) + 255) & ~(size_t)255));
  }
  return knn_launch(tree, N, first, queries, B, k, w_vel, idx, d2, nsplit, part_d, part_i,
                    (cudaStream_t)stream);
}
