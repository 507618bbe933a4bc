// Tensor-core (tcgen05 / TMEM) inference of the duration surrogate.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fn_api.h"
#include "fn_arm.cuh"

namespace fn {

// Packed weight layout (the UMMA canonical K-major layout without swizzle):
// a chunk holds N = 256 output rows x Kt input columns; element (n, k) of a
// chunk sits at byte ((n / 8) * (Kt / 8) + k / 8) * 128 + (n % 8) * 16 +
// (k % 8) * 2, i.e. 8 x 8 "core matrices" of 128 contiguous bytes, adjacent
// along K 128 B apart and along N Kt * 16 B apart.
constexpr int kTcN = 256;              // hidden width (MMA N)
constexpr int kTcM = 128;              // edges per tile (MMA M, one TMEM lane each)
constexpr int kTcK1 = 32;              // layer-1 inputs (28 features + 4 zeros)
constexpr int kTcKc = 64;              // K columns per streamed weight chunk
constexpr int kTcChunkBytes = kTcN * kTcKc * 2;         // 32 KB
constexpr int kTcW1Bytes = kTcN * kTcK1 * 2;            // 16 KB
constexpr int kTcW23Bytes = 2 * 4 * kTcChunkBytes;      // layers 2 and 3: 8 chunks

// Pack bf16 weights W [K][256] (row-major over the outputs) into chunks of
// Kt columns (K a multiple of Kt).
void mlp_tc_pack(const __nv_bfloat16* W, int K, int Kt, __nv_bfloat16* out, cudaStream_t st);

// Y[e] = MLP(features(s0[e], s1[e])) for e < E with the packed layers 1-3,
// the bf16 layer-4 weights W4b [256][2] and the FP32 biases.  *err is set
// to 1 if a wait on the tensor core or a copy timed out.  Y: device [E][2].
// E_dev (device, may be NULL): the rows actually present, at most E.
fn_status mlp_tc_forward(const ArmK& A, const float* s0, const float* s1, int E,
                         const __nv_bfloat16* W1p, const __nv_bfloat16* W23p, const float* b1,
                         const float* b2, const float* b3, const __nv_bfloat16* W4b,
                         const float* b4, float* Y, int* err, cudaStream_t st,
                         const int* E_dev = nullptr);

// General BF16 GEMM on the tensor cores (FP32 accumulation):
// C = op(A) op(B) (+ bias, ReLU), op = transpose when TA / TB (see
// fn_mlp_tc.cu); C as FP32 (Cf, overwritten or, `accumulate`, added to) and
// / or BF16 (Cb).  A long K without bias, ReLU or BF16 output is split over
// CTAs whose FP32 partial sums are added atomically.  *err is set to 1 if a
// wait on the tensor core timed out.
template <bool TA, bool TB>
void gemm_tc(int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
             const float* bias, bool relu, bool accumulate, float* Cf, int ldcf,
             __nv_bfloat16* Cb, int ldcb, int* err, cudaStream_t st);

}  // namespace fn

struct fn_mlp;

namespace fn {

// The model's tensor-core forward over rows counted on the device (for a
// caller inside a captured sequence): refreshes the packed weights first if
// they changed.  Stream-ordered, no host synchronisation.
fn_status mlp_forward_rows(fn_mlp* m, const ArmK& A, const float* s0, const float* s1, int E_max,
                           const int* E_dev, float* Y, cudaStream_t st);

}  // namespace fn
