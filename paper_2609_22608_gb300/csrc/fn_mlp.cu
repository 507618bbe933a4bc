// Duration surrogate: an MLP 28 -> 256 -> 256 -> 256 -> 2 (ReLU) predicting
// (log T*, feasibility logit) of an edge from its boundary states, trained
// on labels produced by the exact duration scan (the windowed scan that uses
// it is fn_edges.cu's k_time_window_tm).  The paper has no learned
// component; this is the project's addition on top of Sec. IV-D's search.
//
// Precision (identical in the FP64 test oracle): inputs, weights and hidden
// activations are rounded to bf16 and contracted on the tensor cores with
// FP32 accumulation; biases, losses and gradients of the outputs are FP32;
// Adam keeps FP32 master weights and refreshes the bf16 copies after every
// step.
//
// The contractions use mma.sync.m16n8k16 (bf16 in, f32 accumulate) in a
// tiled 64x64x32 kernel with optional transposed operands, which serves the
// forward pass (h W), the input gradients (dz W^T) and the weight gradients
// (h^T dz).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "edge_core.cuh"
#include "fn_internal.h"
#include "fn_mlp_tc.h"

namespace fn {

typedef __nv_bfloat16 bf16;

static const int kDims[5] = {32, 256, 256, 256, 2};  // input padded from 28 to 32
#define MLP_LAYERS 4
#define MLP_H 256

// ---------------------------------------------------------------------------
// features: q scaled by the joint box to [-1, 1], qd by qd_max, both states
// ---------------------------------------------------------------------------
__global__ void k_mlp_features(ArmK A, const float* __restrict__ s0, const float* __restrict__ s1,
                               int E, bf16* __restrict__ X) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)E * 32) return;
  const long e = i >> 5;
  const int f = (int)(i & 31);
  float v = 0.f;
  if (f < 28) {
    const int j = f % 7, part = f / 7;
    const float* s = (part < 2 ? s0 : s1) + 16 * e;
    const float c = 0.5f * (A.q_lo[j] + A.q_hi[j]);
    const float h = 0.5f * (A.q_hi[j] - A.q_lo[j]);
    v = (part & 1) ? s[8 + j] / A.qd_max[j] : (s[j] - c) / h;
  }
  X[i] = __float2bfloat16_rn(v);
}

// ---------------------------------------------------------------------------
// C (M x N) = act(A (M x K) B (K x N) + bias), bf16 operands, f32 accumulate.
// A(m, k) = A[m lda + k] (TA: A[k lda + m]); B(k, n) = B[k ldb + n]
// (TB: B[n ldb + k]).  Outputs: Cf (f32, optionally accumulated) and/or Cb
// (bf16).  Tiles: 64 x 64 per block, 32 along K; 4 warps of 32 x 32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K,
                                                   const bf16* __restrict__ A, int lda,
                                                   const bf16* __restrict__ B, int ldb,
                                                   const float* __restrict__ bias, int relu,
                                                   int accumulate, float* __restrict__ Cf,
                                                   int ldcf, bf16* __restrict__ Cb, int ldcb) {
  __shared__ __align__(16) bf16 As[64][40];  // [m][k]
  __shared__ __align__(16) bf16 Bs[64][40];  // [n][k]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 1, wn = warp & 1;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const bf16 zero = __float2bfloat16_rn(0.f);
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int t = tid; t < 64 * 32; t += 128) {
      int r, c;  // (m, k) with the contiguous global index fastest
      if (TA) { r = t & 63; c = t >> 6; } else { r = t >> 5; c = t & 31; }
      const int gm = m0 + r, gk = k0 + c;
      bf16 v = zero;
      if (gm < M && gk < K) v = TA ? A[(long)gk * lda + gm] : A[(long)gm * lda + gk];
      As[r][c] = v;
    }
    for (int t = tid; t < 64 * 32; t += 128) {
      int r, c;  // (n, k)
      if (TB) { r = t >> 5; c = t & 31; } else { r = t & 63; c = t >> 6; }
      const int gn = n0 + r, gk = k0 + c;
      bf16 v = zero;
      if (gn < N && gk < K) v = TB ? B[(long)gn * ldb + gk] : B[(long)gk * ldb + gn];
      Bs[r][c] = v;
    }
    __syncthreads();
    const int g = lane >> 2, tg = lane & 3;
#pragma unroll
    for (int ks = 0; ks < 32; ks += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r0 = wm * 32 + mi * 16 + g, c0 = ks + 2 * tg;
        a[mi][0] = *reinterpret_cast<const uint32_t*>(&As[r0][c0]);
        a[mi][1] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][c0]);
        a[mi][2] = *reinterpret_cast<const uint32_t*>(&As[r0][c0 + 8]);
        a[mi][3] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][c0 + 8]);
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int n = wn * 32 + ni * 8 + g;
        b[ni][0] = *reinterpret_cast<const uint32_t*>(&Bs[n][ks + 2 * tg]);
        b[ni][1] = *reinterpret_cast<const uint32_t*>(&Bs[n][ks + 2 * tg + 8]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], a[mi], b[ni]);
    }
    __syncthreads();
  }
  const int g = lane >> 2, tg = lane & 3;
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int row = m0 + wm * 32 + mi * 16 + g + 8 * h;
          const int col = n0 + wn * 32 + ni * 8 + 2 * tg + cc;
          if (row >= M || col >= N) continue;
          float v = acc[mi][ni][2 * h + cc] + (bias ? bias[col] : 0.f);
          if (relu) v = fmaxf(v, 0.f);
          if (Cf) {
            float* o = Cf + (long)row * ldcf + col;
            *o = accumulate ? *o + v : v;
          }
          if (Cb) Cb[(long)row * ldcb + col] = __float2bfloat16_rn(v);
        }
}

// The training GEMMs with a 256-wide output (and 16-byte aligned rows) run
// on the tensor cores (tcgen05, gemm_tc); the two-column ones of layer 4 on
// mma.sync tiles.
template <bool TA, bool TB>
static void gemm(int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb,
                 const float* bias, bool relu, bool accumulate, float* Cf, int ldcf, bf16* Cb,
                 int ldcb, int* err, cudaStream_t st) {
  if (N >= 128 && lda % 8 == 0 && ldb % 8 == 0 && aligned16(A) && aligned16(B)) {
    gemm_tc<TA, TB>(M, N, K, A, lda, B, ldb, bias, relu, accumulate, Cf, ldcf, Cb, ldcb, err, st);
    return;
  }
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  k_gemm_bf16<TA, TB><<<grid, 128, 0, st>>>(M, N, K, A, lda, B, ldb, bias, relu ? 1 : 0,
                                            accumulate ? 1 : 0, Cf, ldcf, Cb, ldcb);
}

// loss L = (1/n) sum_i [ f_i (y_i0 - log T*_i)^2 + BCE(y_i1, f_i) ] and dL/dy
__global__ void k_mlp_loss(const float* __restrict__ Y, const int32_t* __restrict__ kstar,
                           const float* __restrict__ logT, int n, float* __restrict__ dY,
                           bf16* __restrict__ dYb, float* __restrict__ loss) {
  __shared__ float red[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float L = 0.f;
  if (i < n) {
    const int k = kstar[i];
    const float f = k >= 0 ? 1.f : 0.f;
    const float y0 = Y[2 * i], y1 = Y[2 * i + 1];
    const float d = k >= 0 ? y0 - logT[k] : 0.f;
    const float s = 1.f / (1.f + expf(-y1));
    L = f * d * d + fmaxf(y1, 0.f) - y1 * f + log1pf(expf(-fabsf(y1)));
    const float g0 = 2.f * f * d / (float)n, g1 = (s - f) / (float)n;
    dY[2 * i] = g0;
    dY[2 * i + 1] = g1;
    dYb[2 * i] = __float2bfloat16_rn(g0);
    dYb[2 * i + 1] = __float2bfloat16_rn(g1);
  }
  red[threadIdx.x] = L;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] / (float)n);
}

// dz = dh * 1[h > 0] -> bf16, and the column sums of dz (bias gradient)
__global__ void k_mlp_relu_back(const float* __restrict__ dH, const bf16* __restrict__ Hb, int n,
                                int width, bf16* __restrict__ dZb, float* __restrict__ gb) {
  const int c = threadIdx.x;  // blockDim.x = width
  const int rows = (n + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * rows, r1 = min(n, r0 + rows);
  float sum = 0.f;
  for (int r = r0; r < r1; ++r) {
    const long idx = (long)r * width + c;
    const float z = __bfloat162float(Hb[idx]) > 0.f ? dH[idx] : 0.f;
    dZb[idx] = __float2bfloat16_rn(z);
    sum += z;
  }
  atomicAdd(gb + c, sum);
}

// column sums of a [n][w] f32 matrix into gb (w <= 32)
__global__ void k_mlp_colsum(const float* __restrict__ D, int n, int w, float* __restrict__ gb) {
  float sum = 0.f;
  const int c = threadIdx.x % w;
  for (long r = (long)blockIdx.x * (blockDim.x / w) + threadIdx.x / w; r < n;
       r += (long)gridDim.x * (blockDim.x / w))
    sum += D[r * w + c];
  atomicAdd(gb + c, sum);
}

// Adam on FP32 master weights; bf16 copy refreshed
__global__ void k_mlp_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ g, bf16* __restrict__ pb, long n, float lr,
                           float b1, float b2, float eps, float c1, float c2) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = (mi / c1) / (sqrtf(vi / c2) + eps);
    const float pn = p[i] - lr * upd;
    p[i] = pn;
    if (pb) pb[i] = __float2bfloat16_rn(pn);
  }
}

__global__ void k_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

}  // namespace fn

using namespace fn;

struct fn_mlp {
  int max_batch;
  float* W[MLP_LAYERS];   // master [in][out]
  float* b[MLP_LAYERS];
  bf16* Wb[MLP_LAYERS];
  float* mW[MLP_LAYERS]; float* vW[MLP_LAYERS]; float* mb[MLP_LAYERS]; float* vb[MLP_LAYERS];
  float* gW[MLP_LAYERS]; float* gb[MLP_LAYERS];
  int step;
  // workspace for one batch
  bf16* X;        // [n][32]
  bf16* Hb[3];    // [n][256]
  float* Y;       // [n][2]
  float* dY;      // [n][2]
  bf16* dYb;      // [n][2]
  float* dH;      // [n][256]
  bf16* dZb;      // [n][256]
  float* loss;    // [1]
  float* logT;    // [FN_MAX_GRID]
  // tensor-core inference: layers 1-3 packed for tcgen05 (refreshed lazily
  // after any weight change) and the kernel's error flag
  bf16* W1p;      // [16 KB]
  bf16* W23p;     // [256 KB]
  int* tc_err;    // [1]
  bool packed;
  std::vector<void*> allocs;
};

static fn_status mlp_alloc(fn_mlp* m, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) return FN_ENOMEM;
  m->allocs.push_back(*p);
  return FN_OK;
}

extern "C" fn_status fn_mlp_destroy(fn_mlp_t* m) {
  if (!m) return FN_EINVAL;
  for (void* p : m->allocs) cudaFree(p);
  delete m;
  return FN_OK;
}

extern "C" fn_status fn_mlp_create(int max_batch, unsigned long long seed, fn_mlp_t** out) {
  if (!out || max_batch < 1 || max_batch > (1 << 22)) return FN_EINVAL;
  fn_mlp* m = new fn_mlp();
  m->max_batch = max_batch;
  m->step = 0;
  fn_status rc = FN_OK;
  auto A = [&](void** p, size_t bytes) {
    if (rc == FN_OK) rc = mlp_alloc(m, p, bytes);
  };
  for (int l = 0; l < MLP_LAYERS; ++l) {
    const size_t nw = (size_t)kDims[l] * kDims[l + 1], nb = kDims[l + 1];
    A((void**)&m->W[l], nw * 4); A((void**)&m->b[l], nb * 4); A((void**)&m->Wb[l], nw * 2);
    A((void**)&m->mW[l], nw * 4); A((void**)&m->vW[l], nw * 4);
    A((void**)&m->mb[l], nb * 4); A((void**)&m->vb[l], nb * 4);
    A((void**)&m->gW[l], nw * 4); A((void**)&m->gb[l], nb * 4);
  }
  const size_t n = max_batch;
  A((void**)&m->X, n * 32 * 2);
  for (int l = 0; l < 3; ++l) A((void**)&m->Hb[l], n * MLP_H * 2);
  A((void**)&m->Y, n * 2 * 4); A((void**)&m->dY, n * 2 * 4); A((void**)&m->dYb, n * 2 * 2);
  A((void**)&m->dH, n * MLP_H * 4); A((void**)&m->dZb, n * MLP_H * 2);
  A((void**)&m->loss, 4); A((void**)&m->logT, FN_MAX_GRID * 4);
  A((void**)&m->W1p, kTcW1Bytes); A((void**)&m->W23p, kTcW23Bytes); A((void**)&m->tc_err, 4);
  m->packed = false;
  if (rc != FN_OK) {
    fn_mlp_destroy(m);
    return rc;
  }
  cudaMemset(m->tc_err, 0, 4);
  // He-uniform initial weights (inputs 28 of 32 used), zero biases, zero moments
  std::mt19937_64 rng(seed);
  for (int l = 0; l < MLP_LAYERS; ++l) {
    const int fin = l == 0 ? 28 : kDims[l], nin = kDims[l], nout = kDims[l + 1];
    const double lim = std::sqrt(6.0 / fin);
    std::uniform_real_distribution<double> U(-lim, lim);
    std::vector<float> w((size_t)nin * nout);
    for (int i = 0; i < nin; ++i)
      for (int o = 0; o < nout; ++o) w[(size_t)i * nout + o] = (l == 0 && i >= 28) ? 0.f : (float)U(rng);
    if (cudaMemcpy(m->W[l], w.data(), w.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      rc = FN_ECUDA;
    const size_t nw = w.size();
    cudaMemset(m->b[l], 0, nout * 4);
    cudaMemset(m->mW[l], 0, nw * 4); cudaMemset(m->vW[l], 0, nw * 4);
    cudaMemset(m->mb[l], 0, nout * 4); cudaMemset(m->vb[l], 0, nout * 4);
    k_to_bf16<<<(unsigned)((nw + 255) / 256), 256>>>(m->W[l], m->Wb[l], (long)nw);
  }
  if (rc != FN_OK || cudaDeviceSynchronize() != cudaSuccess) {
    fn_mlp_destroy(m);
    return FN_ECUDA;
  }
  *out = m;
  return FN_OK;
}

// forward pass of n rows whose features are in m->X; Y = output
static void mlp_forward(fn_mlp* m, int n, cudaStream_t st) {
  gemm<false, false>(n, 256, 32, m->X, 32, m->Wb[0], 256, m->b[0], true, false, nullptr, 0,
                     m->Hb[0], 256, m->tc_err, st);
  gemm<false, false>(n, 256, 256, m->Hb[0], 256, m->Wb[1], 256, m->b[1], true, false, nullptr, 0,
                     m->Hb[1], 256, m->tc_err, st);
  gemm<false, false>(n, 256, 256, m->Hb[1], 256, m->Wb[2], 256, m->b[2], true, false, nullptr, 0,
                     m->Hb[2], 256, m->tc_err, st);
  gemm<false, false>(n, 2, 256, m->Hb[2], 256, m->Wb[3], 2, m->b[3], false, false, m->Y, 2,
                     nullptr, 0, m->tc_err, st);
}

static fn_status mlp_features(fn_mlp* m, const fn_arm_t* arm, const float* s0, const float* s1,
                              int n, cudaStream_t st) {
  ArmK A;
  if (!make_armk(arm, &A)) return FN_EINVAL;
  const long tot = (long)n * 32;
  k_mlp_features<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(A, s0, s1, n, m->X);
  return FN_OK;
}

// inference on the tcgen05 path (fused, no workspace, any E)
extern "C" fn_status fn_mlp_predict(fn_mlp_t* m, const fn_arm_t* arm, const float* s0,
                                    const float* s1, int E, float* Y, void* stream) {
  if (!m || E < 0 || !Y || (E > 0 && (!s0 || !s1))) return FN_EINVAL;
  if (E == 0) return FN_OK;
  if (!aligned16(s0) || !aligned16(s1)) return FN_EINVAL;
  ArmK A;
  if (!make_armk(arm, &A)) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (!m->packed) {
    mlp_tc_pack(m->Wb[0], 32, kTcK1, m->W1p, st);
    mlp_tc_pack(m->Wb[1], 256, kTcKc, m->W23p, st);
    mlp_tc_pack(m->Wb[2], 256, kTcKc, m->W23p + kTcW23Bytes / 4, st);
    m->packed = true;
  }
  return mlp_tc_forward(A, s0, s1, E, m->W1p, m->W23p, m->b[0], m->b[1], m->b[2], m->Wb[3],
                        m->b[3], Y, m->tc_err, st);
}

namespace fn {
fn_status mlp_forward_rows(fn_mlp* m, const ArmK& A, const float* s0, const float* s1, int E_max,
                           const int* E_dev, float* Y, cudaStream_t st) {
  if (!m || E_max < 0) return FN_EINVAL;
  if (E_max == 0) return FN_OK;
  if (!m->packed) {
    mlp_tc_pack(m->Wb[0], 32, kTcK1, m->W1p, st);
    mlp_tc_pack(m->Wb[1], 256, kTcKc, m->W23p, st);
    mlp_tc_pack(m->Wb[2], 256, kTcKc, m->W23p + kTcW23Bytes / 4, st);
    m->packed = true;
  }
  return mlp_tc_forward(A, s0, s1, E_max, m->W1p, m->W23p, m->b[0], m->b[1], m->b[2], m->Wb[3],
                        m->b[3], Y, m->tc_err, st, E_dev);
}
}  // namespace fn

// the same forward on the mma.sync path (the training kernels), E <= max_batch
// per internal batch
extern "C" fn_status fn_mlp_predict_ref(fn_mlp_t* m, const fn_arm_t* arm, const float* s0,
                                        const float* s1, int E, float* Y, void* stream) {
  if (!m || E < 0 || !Y || (E > 0 && (!s0 || !s1))) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  for (int e0 = 0; e0 < E; e0 += m->max_batch) {
    const int n = std::min(m->max_batch, E - e0);
    fn_status rc = mlp_features(m, arm, s0 + 16L * e0, s1 + 16L * e0, n, st);
    if (rc != FN_OK) return rc;
    mlp_forward(m, n, st);
    if (cudaMemcpyAsync(Y + 2L * e0, m->Y, (size_t)n * 8, cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
      return FN_ECUDA;
  }
  return launch_status();
}

extern "C" fn_status fn_mlp_error(fn_mlp_t* m, int* flag, int reset) {
  if (!m || !flag) return FN_EINVAL;
  if (cudaMemcpy(flag, m->tc_err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return FN_ECUDA;
  if (reset && cudaMemset(m->tc_err, 0, 4) != cudaSuccess) return FN_ECUDA;
  return FN_OK;
}

// forward + loss + backward into m->gW / m->gb (no update)
static fn_status mlp_backward(fn_mlp* m, int n, const int32_t* kstar, cudaStream_t st) {
  mlp_forward(m, n, st);
  cudaMemsetAsync(m->loss, 0, 4, st);
  k_mlp_loss<<<(n + 255) / 256, 256, 0, st>>>(m->Y, kstar, m->logT, n, m->dY, m->dYb, m->loss);
  for (int l = 0; l < MLP_LAYERS; ++l) {
    cudaMemsetAsync(m->gb[l], 0, kDims[l + 1] * 4, st);
  }
  // layer 4 (linear): dz4 = dy
  gemm<true, false>(256, 2, n, m->Hb[2], 256, m->dYb, 2, nullptr, false, false, m->gW[3], 2,
                    nullptr, 0, m->tc_err, st);
  k_mlp_colsum<<<64, 256, 0, st>>>(m->dY, n, 2, m->gb[3]);
  gemm<false, true>(n, 256, 2, m->dYb, 2, m->Wb[3], 2, nullptr, false, false, m->dH, 256, nullptr,
                    0, m->tc_err, st);
  const int rb = std::max(1, std::min(512, (n + 63) / 64));
  for (int l = 2; l >= 0; --l) {
    // dz_l = dh_l * 1[h_l > 0]; dW_l = h_{l-1}^T dz_l; dh_{l-1} = dz_l W_l^T
    k_mlp_relu_back<<<rb, 256, 0, st>>>(m->dH, m->Hb[l], n, 256, m->dZb, m->gb[l]);
    const bf16* hin = l == 0 ? m->X : m->Hb[l - 1];
    const int nin = kDims[l];
    gemm<true, false>(nin, 256, n, hin, nin, m->dZb, 256, nullptr, false, false, m->gW[l], 256,
                      nullptr, 0, m->tc_err, st);
    if (l > 0)
      gemm<false, true>(n, 256, 256, m->dZb, 256, m->Wb[l], 256, nullptr, false, false, m->dH, 256,
                        nullptr, 0, m->tc_err, st);
  }
  return launch_status();
}

static fn_status set_logT(fn_mlp* m, const float* T_grid, int K, cudaStream_t st) {
  if (!T_grid || K < 1 || K > FN_MAX_GRID) return FN_EINVAL;
  float lg[FN_MAX_GRID];
  for (int k = 0; k < K; ++k) {
    if (!(T_grid[k] > 0.f)) return FN_EINVAL;
    lg[k] = std::log(T_grid[k]);
  }
  if (cudaMemcpyAsync(m->logT, lg, K * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return FN_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? FN_OK : FN_ECUDA;
}

extern "C" fn_status fn_mlp_backward(fn_mlp_t* m, const fn_arm_t* arm, const float* s0,
                                     const float* s1, const int32_t* k_star, const float* T_grid,
                                     int K, int E, float* loss, void* stream) {
  if (!m || E < 1 || E > m->max_batch || !s0 || !s1 || !k_star) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  fn_status rc = set_logT(m, T_grid, K, st);
  if (rc != FN_OK) return rc;
  if ((rc = mlp_features(m, arm, s0, s1, E, st)) != FN_OK) return rc;
  if ((rc = mlp_backward(m, E, k_star, st)) != FN_OK) return rc;
  if (loss) {
    if (cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return FN_ECUDA;
  }
  return FN_OK;
}

extern "C" fn_status fn_mlp_adam_step(fn_mlp_t* m, float lr, void* stream) {
  if (!m || !(lr >= 0.f)) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  m->step += 1;
  m->packed = false;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = (float)(1.0 - std::pow(0.9, m->step));
  const float c2 = (float)(1.0 - std::pow(0.999, m->step));
  for (int l = 0; l < MLP_LAYERS; ++l) {
    const long nw = (long)kDims[l] * kDims[l + 1], nb = kDims[l + 1];
    k_mlp_adam<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(m->W[l], m->mW[l], m->vW[l], m->gW[l],
                                                            m->Wb[l], nw, lr, b1, b2, eps, c1, c2);
    k_mlp_adam<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(m->b[l], m->mb[l], m->vb[l], m->gb[l],
                                                            nullptr, nb, lr, b1, b2, eps, c1, c2);
  }
  return launch_status();
}

extern "C" fn_status fn_mlp_train_step(fn_mlp_t* m, const fn_arm_t* arm, const float* s0,
                                       const float* s1, const int32_t* k_star,
                                       const float* T_grid, int K, int E, float lr, float* loss,
                                       void* stream) {
  fn_status rc = fn_mlp_backward(m, arm, s0, s1, k_star, T_grid, K, E, nullptr, stream);
  if (rc != FN_OK) return rc;
  if ((rc = fn_mlp_adam_step(m, lr, stream)) != FN_OK) return rc;
  if (loss) {
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return FN_ECUDA;
  }
  return FN_OK;
}

// parameter / gradient / moment access (host arrays, layer l, W [in][out])
extern "C" fn_status fn_mlp_get_params(fn_mlp_t* m, int l, float* W, float* b) {
  if (!m || l < 0 || l >= MLP_LAYERS) return FN_EINVAL;
  const size_t nw = (size_t)kDims[l] * kDims[l + 1], nb = kDims[l + 1];
  if (cudaDeviceSynchronize() != cudaSuccess) return FN_ECUDA;
  if (W && cudaMemcpy(W, m->W[l], nw * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return FN_ECUDA;
  if (b && cudaMemcpy(b, m->b[l], nb * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return FN_ECUDA;
  return FN_OK;
}

extern "C" fn_status fn_mlp_set_params(fn_mlp_t* m, int l, const float* W, const float* b) {
  if (!m || l < 0 || l >= MLP_LAYERS) return FN_EINVAL;
  const size_t nw = (size_t)kDims[l] * kDims[l + 1], nb = kDims[l + 1];
  if (W && cudaMemcpy(m->W[l], W, nw * 4, cudaMemcpyHostToDevice) != cudaSuccess) return FN_ECUDA;
  if (b && cudaMemcpy(m->b[l], b, nb * 4, cudaMemcpyHostToDevice) != cudaSuccess) return FN_ECUDA;
  k_to_bf16<<<(unsigned)((nw + 255) / 256), 256>>>(m->W[l], m->Wb[l], (long)nw);
  m->packed = false;
  return cudaDeviceSynchronize() == cudaSuccess ? FN_OK : FN_ECUDA;
}

extern "C" fn_status fn_mlp_get_grads(fn_mlp_t* m, int l, float* gW, float* gb) {
  if (!m || l < 0 || l >= MLP_LAYERS) return FN_EINVAL;
  const size_t nw = (size_t)kDims[l] * kDims[l + 1], nb = kDims[l + 1];
  if (cudaDeviceSynchronize() != cudaSuccess) return FN_ECUDA;
  if (gW && cudaMemcpy(gW, m->gW[l], nw * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return FN_ECUDA;
  if (gb && cudaMemcpy(gb, m->gb[l], nb * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return FN_ECUDA;
  return FN_OK;
}

extern "C" fn_status fn_mlp_set_grads(fn_mlp_t* m, int l, const float* gW, const float* gb) {
  if (!m || l < 0 || l >= MLP_LAYERS) return FN_EINVAL;
  const size_t nw = (size_t)kDims[l] * kDims[l + 1], nb = kDims[l + 1];
  if (gW && cudaMemcpy(m->gW[l], gW, nw * 4, cudaMemcpyHostToDevice) != cudaSuccess) return FN_ECUDA;
  if (gb && cudaMemcpy(m->gb[l], gb, nb * 4, cudaMemcpyHostToDevice) != cudaSuccess) return FN_ECUDA;
  return FN_OK;
}

// binary file: "FNMLP1\0\0", step, then per layer W (f32 [in][out]) and b
extern "C" fn_status fn_mlp_save(fn_mlp_t* m, const char* path) {
  if (!m || !path) return FN_EINVAL;
  FILE* f = std::fopen(path, "wb");
  if (!f) return FN_EINVAL;
  const char magic[8] = {'F', 'N', 'M', 'L', 'P', '1', 0, 0};
  bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(&m->step, 4, 1, f) == 1;
  for (int l = 0; l < MLP_LAYERS && ok; ++l) {
    std::vector<float> W((size_t)kDims[l] * kDims[l + 1]), b(kDims[l + 1]);
    ok = fn_mlp_get_params(m, l, W.data(), b.data()) == FN_OK &&
         std::fwrite(W.data(), 4, W.size(), f) == W.size() &&
         std::fwrite(b.data(), 4, b.size(), f) == b.size();
  }
  std::fclose(f);
  return ok ? FN_OK : FN_ECUDA;
}

extern "C" fn_status fn_mlp_load(fn_mlp_t* m, const char* path) {
  if (!m || !path) return FN_EINVAL;
  FILE* f = std::fopen(path, "rb");
  if (!f) return FN_EINVAL;
  char magic[8];
  int step = 0;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "FNMLP1", 6) == 0 &&
            std::fread(&step, 4, 1, f) == 1;
  for (int l = 0; l < MLP_LAYERS && ok; ++l) {
    std::vector<float> W((size_t)kDims[l] * kDims[l + 1]), b(kDims[l + 1]);
    ok = std::fread(W.data(), 4, W.size(), f) == W.size() &&
         std::fread(b.data(), 4, b.size(), f) == b.size() &&
         fn_mlp_set_params(m, l, W.data(), b.data()) == FN_OK;
  }
  std::fclose(f);
  if (ok) m->step = step;
  return ok ? FN_OK : FN_EINVAL;
}

