// The planner: one round of Algorithm 1 ("FRUITNINJA: one planning cycle",
// Sec. IV-E) for P independent problems at once, entirely on the device.
//
// Memory (Sec. IV-E: "preallocated struct-of-arrays"): every buffer is sized
// once in fn_planner_create for P problems x n_cap nodes x b_max candidates;
// per-problem counts (tree size, incumbent, t_best) live in device memory,
// so an iteration never reads anything back before its end and can be
// captured as a CUDA graph.  One iteration is a fixed sequence of launches
// over all problems:
//   schedule  : per-problem work offsets, work-queue reset
//   sample    : goal chart / uniform candidates (Philox counters)
//   knn       : flattened (problem, query tile, node split) work items
//   knn_merge : warp-per-query merge of the node splits
//   edges     : ONE persistent launch; warps pull (problem, candidate,
//               parent) edges from a device work queue (free edges first),
//               time them (edge_core.cuh) and check clearance
//   attach    : block per problem: best parent, stable compaction, scoring,
//               incumbent
//   prune     : block per problem (optional): Eq. (reach)
//   output    : rendezvous per problem
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <vector>

#include "edge_core.cuh"
#include "fn_internal.h"
#include "fn_kin.cuh"
#include "fn_tune.h"
#include "knn_core.cuh"

#define PL_NSPLIT_MAX 8
#define PL_MAX_P 1024

namespace fn {

struct Incumbent {
  int id;
  float J;
  float t_best;
  int pad;
};

struct Sched {
  unsigned int queue_head;
  int n_free_edges;   // free edges of all problems (the queue's first part)
  int n_edges;        // all edges
  int knn_items;      // (problem, query tile, split) items
  int free_off[PL_MAX_P + 1];
  int goal_off[PL_MAX_P + 1];
  int knn_off[PL_MAX_P + 1];
  int nsplit[PL_MAX_P];
};

struct PlanDev {  // device pointers, passed by value to the kernels
  int P, NC, BM, KP, KN, KM, K, S, S_clear, G;
  float w_vel, vel_frac, margin;
  float* st;          // [P][NC][16]
  float* t;           // [P][NC]
  int32_t* par;       // [P][NC]
  float* J;           // [P][NC]
  float* nu;          // [P][NC]
  float* eT;          // [P][NC] edge duration into the node
  int32_t* n_nodes;   // [P]
  float* cand;        // [P][BM][16]
  float* treq;        // [P][BM]
  float* vrel;        // [P][BM]
  uint8_t* valid;     // [P][BM]
  int32_t* nn;        // [P][BM][KN]
  float* part_d;      // [P][NSPLIT][BM][KM]
  int32_t* part_i;
  float* e_T;         // [P][BM][KP]
  float* e_rv;
  uint8_t* e_ok;
  Incumbent* inc;     // [P]
  fn_problem_t* prob; // [P]
  Sched* sched;
  fn_rendezvous_t* out;  // [P]
  int* iter;
  int32_t* added;     // [P]
  int32_t* status;    // [P]
  // prune scratch
  int32_t* ptr;       // [P][NC]
  int32_t* newidx;    // [P][NC]
  uint8_t* alive;     // [P][NC]
  float* tmp_st;      // [P][NC][16]
  float* tmp_f;       // [P][NC][4]  (t, J, nu, eT)
  int32_t* tmp_par;   // [P][NC]
  unsigned long long* samples;  // work counter (torque evaluations)
};

struct GridKP {
  float T[FN_MAX_GRID];
};

// ---------------------------------------------------------------------------
// reset / load
// ---------------------------------------------------------------------------
__global__ void k_plan_reset(PlanDev D) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= D.P) return;
  const fn_problem_t& P = D.prob[p];
  float* s = D.st + (long)p * D.NC * 16;
#pragma unroll
  for (int j = 0; j < 16; ++j) s[j] = 0.f;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    s[j] = P.q0[j];
    s[8 + j] = P.qd0[j];
  }
  const long n0 = (long)p * D.NC;
  D.t[n0] = 0.f;
  D.par[n0] = -1;
  D.J[n0] = NAN;
  D.nu[n0] = 0.f;
  D.eT[n0] = 0.f;
  D.n_nodes[p] = 1;
  D.inc[p] = Incumbent{-1, -INFINITY, P.t_fall, 0};
  D.status[p] = 0;
}

__global__ void k_plan_loaded(PlanDev D, int p, int n) {
  // nodes given by fn_planner_load_tree carry no score and nu = 0
  const long base = (long)p * D.NC;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    D.J[base + i] = NAN;
    D.nu[base + i] = 0.f;
    D.eT[base + i] = i == 0 ? 0.f : NAN;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    D.n_nodes[p] = n;
    D.inc[p] = Incumbent{-1, -INFINITY, D.prob[p].t_fall, 0};
    D.status[p] = 0;
  }
}

// ---------------------------------------------------------------------------
// schedule: per-problem offsets of every flattened work list
// ---------------------------------------------------------------------------
__global__ void k_plan_schedule(PlanDev D) {
  if (threadIdx.x != 0) return;
  Sched* S = D.sched;
  int fo = 0, go = 0, ko = 0;
  for (int p = 0; p < D.P; ++p) {
    const fn_problem_t& P = D.prob[p];
    const int B = min(max(P.batch, 0), D.BM);
    const int G = min(max(P.n_goal, 0), B);
    S->free_off[p] = fo;
    S->goal_off[p] = go;
    S->knn_off[p] = ko;
    fo += (B - G) * D.KP;
    go += G * D.KP;
    const int span = D.n_nodes[p] - 1;  // non-root nodes
    int ns = 1;
    if (D.KN > 0 && span > 0) {
      ns = min(PL_NSPLIT_MAX, max(1, span / (4 * KNN_TILE)));
    }
    S->nsplit[p] = ns;
    ko += (D.KN > 0 && span > 0) ? ((B + 127) / 128) * ns : 0;
    D.added[p] = 0;
  }
  S->free_off[D.P] = fo;
  S->goal_off[D.P] = go;
  S->knn_off[D.P] = ko;
  S->n_free_edges = fo;
  S->n_edges = fo + go;
  S->knn_items = ko;
  S->queue_head = 0u;
}

// largest p with off[p] <= x (off ascending, off[0] = 0)
__device__ __forceinline__ int find_problem(const int* off, int P, int x) {
  int lo = 0, hi = P - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// samplers
// ---------------------------------------------------------------------------
// Free candidates: one thread each (uniform in the box, |qd| <= vel_frac qdbar).
__global__ void __launch_bounds__(128) k_plan_sample_free(PlanDev D, ArmK A) {
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = (int)(gid / D.BM);
  const int b = (int)(gid - (long)p * D.BM);
  if (p >= D.P) return;
  const fn_problem_t& P = D.prob[p];
  const int B = min(max(P.batch, 0), D.BM);
  const int G = min(max(P.n_goal, 0), B);
  if (b < G || b >= B) return;
  const int it = *D.iter;
  float u[16], q[7], qd[7];
#pragma unroll
  for (int s = 0; s < 4; ++s) philox_u4(P.seed, b, it, p, s, u + 4 * s);
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    q[j] = fmaf(u[j], A.q_hi[j] - A.q_lo[j], A.q_lo[j]);
    const float vb = D.vel_frac * taper(A, j, q[j]);
    qd[j] = fmaf(2.f, u[7 + j], -1.f) * vb;
  }
  const long ci = (long)p * D.BM + b;
  D.treq[ci] = NAN;
  D.vrel[ci] = NAN;
  D.valid[ci] = 1;
  float4* o4 = reinterpret_cast<float4*>(D.cand + ci * 16);
  o4[0] = make_float4(q[0], q[1], q[2], q[3]);
  o4[1] = make_float4(q[4], q[5], q[6], 0.f);
  o4[2] = make_float4(qd[0], qd[1], qd[2], qd[3]);
  o4[3] = make_float4(qd[4], qd[5], qd[6], 0.f);
}

// Goal candidates: a group of 4 lanes per candidate; lanes 0-2 run the three
// IK starts in parallel and the lowest start that converges wins (the same
// result as trying the starts in order).
__global__ void __launch_bounds__(128) k_plan_sample_goal(PlanDev D, ArmK A) {
  const long gid = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  const int sub = threadIdx.x & 3;
  const int p = (int)(gid / D.BM);
  const int b = (int)(gid - (long)p * D.BM);
  bool live = p < D.P;
  int G = 0;
  if (live) {
    const fn_problem_t& P0 = D.prob[p];
    const int B = min(max(P0.batch, 0), D.BM);
    G = min(max(P0.n_goal, 0), B);
    live = b < G;
  }
  const unsigned gmask = 0xfu << (threadIdx.x & 28);
  if (!__any_sync(0xffffffffu, live)) return;
  bool defined = false, found = false;
  ChartPose o;
  float q[7];
  const long ci = live ? (long)p * D.BM + b : 0;
  if (live) {
    const fn_problem_t& P = D.prob[p];
    const int it = *D.iter;
    float u[12], z[9];
#pragma unroll
    for (int s = 0; s < 3; ++s) philox_u4(P.seed, b, it, p, 8 + s, u + 4 * s);
#pragma unroll
    for (int i = 0; i < 9; ++i) z[i] = u[i];
    defined = chart_pose(A, P, z, o);
    if (defined && sub < FN_IK_STARTS) found = ik_solve(A, o.Rg, o.pg, o.q7, sub, q);
  }
  const unsigned won = __ballot_sync(0xffffffffu, found) & gmask;
  const int winner = won ? __ffs(won) - 1 : -1;
  const int lane = threadIdx.x & 31;
  if (!live) return;
  if (sub == 0 && winner < 0) {   // undefined: no IK start converged
    D.treq[ci] = o.T;
    D.vrel[ci] = o.vrel;
    D.valid[ci] = 0;
    float4* o4 = reinterpret_cast<float4*>(D.cand + ci * 16);
    o4[0] = o4[1] = o4[2] = o4[3] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (lane != winner) return;
  float qd[7];
  const bool ok = chart_velocity(A, o, q, qd);
  if (!ok)
#pragma unroll
    for (int j = 0; j < 7; ++j) q[j] = qd[j] = 0.f;
  D.treq[ci] = o.T;
  D.vrel[ci] = o.vrel;
  D.valid[ci] = ok ? 1 : 0;
  float4* o4 = reinterpret_cast<float4*>(D.cand + ci * 16);
  o4[0] = make_float4(q[0], q[1], q[2], q[3]);
  o4[1] = make_float4(q[4], q[5], q[6], 0.f);
  o4[2] = make_float4(qd[0], qd[1], qd[2], qd[3]);
  o4[3] = make_float4(qd[4], qd[5], qd[6], 0.f);
}

// ---------------------------------------------------------------------------
// parents: (problem, query tile, split) items over all problems
// ---------------------------------------------------------------------------
template <int KM>
__global__ void __launch_bounds__(128) k_plan_knn(PlanDev D) {
  __shared__ float4 tile[KNN_TILE * 4];
  const Sched* S = D.sched;
  const int items = S->knn_items;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int p = find_problem(S->knn_off, D.P, item);
    const int local = item - S->knn_off[p];
    const int ns = S->nsplit[p];
    const int qt = local / ns, split = local - qt * ns;
    const int B = min(max(D.prob[p].batch, 0), D.BM);
    const int N = D.n_nodes[p];
    const int span = N - 1;
    const int per = (span + ns - 1) / ns;
    const int lo = 1 + split * per, hi = min(N, lo + per);
    const int b = qt * 128 + threadIdx.x;
    const bool active = b < B;
    float qv[14];
    if (active) load_query(reinterpret_cast<const float4*>(D.cand) + 4 * ((long)p * D.BM + b), qv);
    else
      for (int j = 0; j < 14; ++j) qv[j] = 0.f;
    TopK<KM> top;
    top.init();
    knn_scan_range<KM>(reinterpret_cast<const float4*>(D.st) + 4L * p * D.NC, lo, hi, qv,
                       D.w_vel, top, tile);
    if (active) {
      if (ns == 1) {
        const long off = ((long)p * D.BM + b) * D.KN;
#pragma unroll
        for (int j = 0; j < KM; ++j)
          if (j < D.KN) D.nn[off + j] = top.i[j] == 0x7fffffff ? -1 : top.i[j];
      } else {
        const long off = (((long)p * PL_NSPLIT_MAX + split) * D.BM + b) * KM;
        top.store(D.part_d + off, D.part_i + off, KM);
      }
    }
    __syncthreads();
  }
}

template <int KM>
__global__ void __launch_bounds__(256) k_plan_knn_merge(PlanDev D) {
  const int lane = threadIdx.x & 31;
  const long w = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int p = (int)(w / D.BM);
  const int b = (int)(w - (long)p * D.BM);
  if (p >= D.P) return;
  const int B = min(max(D.prob[p].batch, 0), D.BM);
  const int ns = D.sched->nsplit[p];
  if (b >= B || ns <= 1 || D.n_nodes[p] <= 1) return;
  float d[KM];
  int id[KM];
#pragma unroll
  for (int j = 0; j < KM; ++j) { d[j] = INFINITY; id[j] = 0x7fffffff; }
  if (lane < ns) {
    const long off = (((long)p * PL_NSPLIT_MAX + lane) * D.BM + b) * KM;
#pragma unroll
    for (int j = 0; j < KM; ++j) { d[j] = D.part_d[off + j]; id[j] = D.part_i[off + j]; }
  }
  const long out = ((long)p * D.BM + b) * D.KN;
  for (int r = 0; r < D.KN; ++r) {
    float md = d[0];
    int mi = id[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float od = __shfl_xor_sync(0xffffffffu, md, o);
      const int oi = __shfl_xor_sync(0xffffffffu, mi, o);
      if (knn_less(od, oi, md, mi)) { md = od; mi = oi; }
    }
    if (lane == 0) D.nn[out + r] = mi == 0x7fffffff ? -1 : mi;
    if (id[0] == mi && mi != 0x7fffffff) {
#pragma unroll
      for (int j = 0; j + 1 < KM; ++j) { d[j] = d[j + 1]; id[j] = id[j + 1]; }
      d[KM - 1] = INFINITY;
      id[KM - 1] = 0x7fffffff;
    }
  }
}

// tree has a single node: no neighbours
__global__ void k_plan_nn_empty(PlanDev D) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long n = (long)D.P * D.BM * D.KN;
  if (i >= n) return;
  const int p = (int)(i / ((long)D.BM * D.KN));
  if (D.n_nodes[p] <= 1) D.nn[i] = -1;
}

// ---------------------------------------------------------------------------
// edges: one persistent launch, warps pull edges from the device queue
// ---------------------------------------------------------------------------
#define PL_EDGE_WARPS 4

template <int MINB>
__global__ void __launch_bounds__(32 * PL_EDGE_WARPS, MINB) k_plan_edges(PlanDev D, ArmK A,
                                                                         GridKP Gr) {
  __shared__ float sT[FN_MAX_GRID];
  __shared__ float sEdge[PL_EDGE_WARPS][32];
  __shared__ float sCoef[PL_EDGE_WARPS][FN_CUBIC_WORDS * 32];
  __shared__ float sWr[PL_EDGE_WARPS][FN_WRENCH_WORDS * 32];
  for (int i = threadIdx.x; i < D.K; i += blockDim.x) sT[i] = Gr.T[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* es = sEdge[w];
  const CubicLane cb{&sCoef[w][lane]};
  const LaneWrench wr{&sWr[w][lane]};
  Sched* S = D.sched;
  const int nfree = S->n_free_edges, ntot = S->n_edges;
  unsigned nsamp = 0;
  for (;;) {
    int e = 0;
    if (lane == 0) e = (int)atomicAdd(&S->queue_head, 1u);
    e = __shfl_sync(0xffffffffu, e, 0);
    if (e >= ntot) break;
    const bool goal = e >= nfree;
    const int x = goal ? e - nfree : e;
    const int* off = goal ? S->goal_off : S->free_off;
    const int p = find_problem(off, D.P, x);
    const int local = x - off[p];
    const fn_problem_t& P = D.prob[p];
    const int B = min(max(P.batch, 0), D.BM);
    const int G = min(max(P.n_goal, 0), B);
    // parent-slot-major order: every candidate's root edge (the longest
    // scans, t(p) = 0) is queued before any nearest-node edge
    const int nc = goal ? G : B - G;
    const int j = local / nc;
    const int slot = local - j * nc;
    const int b = goal ? slot : G + slot;
    const long ci = (long)p * D.BM + b;
    const long ei = ci * D.KP + j;
    const int pr = j == 0 ? 0 : D.nn[ci * D.KN + (j - 1)];
    if (pr < 0 || !D.valid[ci]) {
      if (lane == 0) { D.e_ok[ei] = 0; D.e_T[ei] = INFINITY; D.e_rv[ei] = NAN; }
      continue;
    }
    const long node = (long)p * D.NC + pr;
    const bool finite = stage_rows(D.st + node * 16, D.cand + ci * 16, es);
    const float tp = D.t[node];
    const float Tp = goal ? __fsub_rn(D.treq[ci], tp) : __fsub_rn(D.inc[p].t_best, tp);
    EdgeResult r = time_edge(A, es, cb, wr, finite, goal, Tp, sT, D.K, D.S, false, nsamp);
    bool ok = r.ok;
    if (ok && P.n_obs > 0) {
      // Clear: capsule clearance at S_clear points of the edge at T
      float mc = INFINITY;
      Cubic c;
      cubic_coef_sh<true>(es, r.T, c);
      for (int s0 = 0; s0 < D.S_clear; s0 += 32) {
        const int s = s0 + lane;
        if (s < D.S_clear) {
          const float u = sample_u(s, D.S_clear);
          float q[7];
#pragma unroll
          for (int jj = 0; jj < 7; ++jj) {
            float v, a;
            cubic_eval(c, jj, u, q[jj], v, a);
          }
          mc = fminf(mc, config_clearance(A, q, P));
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mc = fminf(mc, __shfl_xor_sync(0xffffffffu, mc, o));
      ok = mc >= D.margin;
    }
    if (lane == 0) {
      D.e_ok[ei] = ok ? 1 : 0;
      D.e_T[ei] = r.T;
      D.e_rv[ei] = r.rv;
    }
  }
  if (D.samples && lane == 0 && nsamp) atomicAdd(D.samples, (unsigned long long)nsamp);
}

// ---------------------------------------------------------------------------
// attach + score + incumbent: one block per problem
// ---------------------------------------------------------------------------
#define PL_ATTACH_THREADS 1024

__device__ __forceinline__ int block_scan_excl(int v, int* sh, int& total) {
  // exclusive scan of one int per thread (blockDim = PL_ATTACH_THREADS)
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int o = 1; o < blockDim.x; o <<= 1) {
    const int a = t >= o ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += a;
    __syncthreads();
  }
  total = sh[blockDim.x - 1];
  const int incl = sh[t];
  __syncthreads();
  return incl - v;
}

__global__ void __launch_bounds__(PL_ATTACH_THREADS) k_plan_attach(PlanDev D) {
  __shared__ int sh[PL_ATTACH_THREADS];
  __shared__ float sJ[PL_ATTACH_THREADS];
  __shared__ int sI[PL_ATTACH_THREADS];
  const int p = blockIdx.x;
  const fn_problem_t& P = D.prob[p];
  const int B = min(max(P.batch, 0), D.BM);
  const int G = min(max(P.n_goal, 0), B);
  const int N0 = D.n_nodes[p];
  const long nb = (long)p * D.NC;
  const int per = (B + blockDim.x - 1) / blockDim.x;
  const int c0 = threadIdx.x * per, c1 = min(B, c0 + per);
  // pass 1: count attachable candidates of this thread's contiguous chunk
  int cnt = 0;
  for (int b = c0; b < c1; ++b) {
    const long ci = (long)p * D.BM + b;
    for (int j = 0; j < D.KP; ++j)
      if (D.e_ok[ci * D.KP + j]) { ++cnt; break; }
  }
  int total;
  const int base = block_scan_excl(cnt, sh, total);
  // pass 2: attach in candidate order (Algorithm 1: argmin_p t(p) + T_p,
  // ties to the lower parent slot)
  float bestJ = -INFINITY;
  int bestI = 0x7fffffff;
  int r = base;
  for (int b = c0; b < c1; ++b) {
    const long ci = (long)p * D.BM + b;
    int bj = -1, bpar = -1;
    float bt = INFINITY;
    for (int j = 0; j < D.KP; ++j) {
      const long ei = ci * D.KP + j;
      if (!D.e_ok[ei]) continue;
      const int pr = j == 0 ? 0 : D.nn[ci * D.KN + (j - 1)];
      const float tt = __fadd_rn(D.t[nb + pr], D.e_T[ei]);
      if (tt < bt) { bt = tt; bj = j; bpar = pr; }
    }
    if (bj < 0) continue;
    const int node = N0 + r;
    ++r;
    if (node >= D.NC) {
      atomicOr(&D.status[p], 1);
      continue;
    }
    const long nd = nb + node;
    const float4* src = reinterpret_cast<const float4*>(D.cand + ci * 16);
    float4* dst = reinterpret_cast<float4*>(D.st + nd * 16);
    dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2]; dst[3] = src[3];
    D.t[nd] = bt;
    D.par[nd] = bpar;
    const float rv = D.e_rv[ci * D.KP + bj];
    const float nu = fmaxf(D.nu[nb + bpar], rv);
    D.nu[nd] = nu;
    D.eT[nd] = D.e_T[ci * D.KP + bj];
    float Jv = NAN;
    if (b < G) {
      Jv = objective(P, bt, D.vrel[ci], nu);
      if (Jv > bestJ || (Jv == bestJ && node < bestI)) { bestJ = Jv; bestI = node; }
    }
    D.J[nd] = Jv;
  }
  // incumbent: argmax J over the new rendezvous nodes (ties: lower id),
  // replacing the current one only if strictly better
  sJ[threadIdx.x] = bestJ;
  sI[threadIdx.x] = bestI;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const float oj = sJ[threadIdx.x + o];
      const int oi = sI[threadIdx.x + o];
      if (oj > sJ[threadIdx.x] || (oj == sJ[threadIdx.x] && oi < sI[threadIdx.x])) {
        sJ[threadIdx.x] = oj;
        sI[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int add = min(total, D.NC - N0);
    D.n_nodes[p] = N0 + add;
    D.added[p] = add;
    Incumbent in = D.inc[p];
    if (sI[0] != 0x7fffffff && sJ[0] > in.J) {
      in.id = sI[0];
      in.J = sJ[0];
      in.t_best = D.t[nb + sI[0]];
      D.inc[p] = in;
    }
  }
}

// ---------------------------------------------------------------------------
// prune (Eq. (reach)): one block per problem
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PL_ATTACH_THREADS) k_plan_prune(PlanDev D, ArmK A) {
  __shared__ int sh[PL_ATTACH_THREADS];
  __shared__ int s_flag;
  const int p = blockIdx.x;
  const fn_problem_t& P = D.prob[p];
  const int N = D.n_nodes[p];
  const long nb = (long)p * D.NC;
  const Incumbent in = D.inc[p];
  const float tb = in.t_best;
  // keep mask: root, the incumbent's path, and nodes that can reach the
  // object by t_best
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    bool keep = i == 0;
    if (!keep) {
      float q[7];
#pragma unroll
      for (int j = 0; j < 7; ++j) q[j] = D.st[(nb + i) * 16 + j];
      const int g = reach_index(A, P, q, D.t[nb + i], D.G);
      if (g >= 0) {
        const float Tg = fmaf((float)g, (P.t_fall - P.t_enter) / (float)(D.G - 1), P.t_enter);
        keep = Tg <= tb;
      }
    }
    D.alive[nb + i] = keep ? 1 : 0;
    D.ptr[nb + i] = D.par[nb + i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = in.id; c > 0; c = D.par[nb + c]) D.alive[nb + c] = 1;
  }
  __syncthreads();
  // descendants of pruned nodes are removed: alive_i &= alive_{ancestors},
  // by pointer jumping over the parent links
  for (int round = 0; round < 32; ++round) {
    if (threadIdx.x == 0) s_flag = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const int a = D.ptr[nb + i];
      if (a > 0) {
        const uint8_t al = D.alive[nb + i] & D.alive[nb + a];
        const int aa = D.ptr[nb + a];
        D.alive[nb + i] = al;
        D.ptr[nb + i] = aa;
        s_flag = 1;
      }
    }
    __syncthreads();
    if (!s_flag) break;
    __syncthreads();
  }
  // stable compaction with parent remap (through scratch copies)
  const int per = (N + blockDim.x - 1) / blockDim.x;
  const int c0 = threadIdx.x * per, c1 = min(N, c0 + per);
  int cnt = 0;
  for (int i = c0; i < c1; ++i) cnt += D.alive[nb + i];
  int total;
  int r = block_scan_excl(cnt, sh, total);
  for (int i = c0; i < c1; ++i) {
    D.newidx[nb + i] = D.alive[nb + i] ? r++ : -1;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int ni = D.newidx[nb + i];
    if (ni < 0) continue;
    const float4* src = reinterpret_cast<const float4*>(D.st + (nb + i) * 16);
    float4* dst = reinterpret_cast<float4*>(D.tmp_st + (nb + ni) * 16);
    dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2]; dst[3] = src[3];
    const int pa = D.par[nb + i];
    D.tmp_par[nb + ni] = pa >= 0 ? D.newidx[nb + pa] : -1;
    float* tf = D.tmp_f + (nb + ni) * 4;
    tf[0] = D.t[nb + i]; tf[1] = D.J[nb + i]; tf[2] = D.nu[nb + i]; tf[3] = D.eT[nb + i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const float4* src = reinterpret_cast<const float4*>(D.tmp_st + (nb + i) * 16);
    float4* dst = reinterpret_cast<float4*>(D.st + (nb + i) * 16);
    dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2]; dst[3] = src[3];
    D.par[nb + i] = D.tmp_par[nb + i];
    const float* tf = D.tmp_f + (nb + i) * 4;
    D.t[nb + i] = tf[0]; D.J[nb + i] = tf[1]; D.nu[nb + i] = tf[2]; D.eT[nb + i] = tf[3];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    D.n_nodes[p] = total;
    if (in.id >= 0) {
      Incumbent o = in;
      o.id = D.newidx[nb + in.id];
      D.inc[p] = o;
    }
  }
}

// ---------------------------------------------------------------------------
// output: the first segment of the incumbent plan (Algorithm 1's return)
// ---------------------------------------------------------------------------
__global__ void k_plan_output(PlanDev D) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= D.P) return;
  const long nb = (long)p * D.NC;
  const Incumbent in = D.inc[p];
  fn_rendezvous_t o;
  memset(&o, 0, sizeof(o));
  o.incumbent = in.id;
  o.J = in.J;
  o.t_best = in.t_best;
  o.n_nodes = D.n_nodes[p];
  o.n_added = D.added[p];
  o.status = D.status[p];
  if (in.id > 0) {
    int c = in.id;
    for (int guard = 0; guard < D.NC && D.par[nb + c] > 0; ++guard) c = D.par[nb + c];
    const float* s = D.st + (nb + c) * 16;
    for (int j = 0; j < 7; ++j) { o.q_g[j] = s[j]; o.qd_g[j] = s[8 + j]; }
    o.T = D.eT[nb + c];
  } else {
    o.T = NAN;
  }
  D.out[p] = o;
}

}  // namespace fn

using namespace fn;

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct fn_planner {
  fn_planner_cfg_t cfg;
  ArmK arm;
  GridKP grid;
  PlanDev D;
  int device;
  std::vector<void*> allocs;
  fn_problem_t* h_prob = nullptr;      // pinned staging
  fn_rendezvous_t* h_out = nullptr;    // pinned
  int* h_iter = nullptr;               // pinned
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  unsigned graph_flags = 0;
  int edge_variant = kDefaultEdgeVariant;
  int edge_blocks = 0;
  // per-phase events (schedule, sample, knn, edges, attach, prune, output)
  cudaEvent_t ev[8] = {};
  bool timing = false;
};

static fn_status pl_alloc(fn_planner* pl, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) return FN_ENOMEM;
  pl->allocs.push_back(*p);
  return FN_OK;
}

template <class T>
static fn_status pl_alloc_n(fn_planner* pl, T** p, size_t n) {
  return pl_alloc(pl, reinterpret_cast<void**>(p), n * sizeof(T));
}

typedef void (*PlanEdgeKernel)(PlanDev, ArmK, GridKP);
static PlanEdgeKernel plan_edge_variant(int v) {
  switch (v) {
    case 0: return k_plan_edges<2>;
    case 1: return k_plan_edges<3>;
    default: return k_plan_edges<4>;
  }
}

static int plan_edge_blocks(fn_planner* pl, int v) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plan_edge_variant(v),
                                                    32 * PL_EDGE_WARPS, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * num_sms();
}

extern "C" fn_status fn_planner_destroy(fn_planner_t* pl) {
  if (!pl) return FN_EINVAL;
  for (cudaEvent_t e : pl->ev)
    if (e) cudaEventDestroy(e);
  if (pl->graph_exec) cudaGraphExecDestroy(pl->graph_exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  for (void* p : pl->allocs) cudaFree(p);
  if (pl->h_prob) cudaFreeHost(pl->h_prob);
  if (pl->h_out) cudaFreeHost(pl->h_out);
  if (pl->h_iter) cudaFreeHost(pl->h_iter);
  delete pl;
  return FN_OK;
}

extern "C" fn_status fn_planner_create(const fn_planner_cfg_t* cfg, const fn_arm_t* arm,
                                       fn_planner_t** out) {
  if (!cfg || !arm || !out) return FN_EINVAL;
  const fn_planner_cfg_t c = *cfg;
  if (c.P < 1 || c.P > PL_MAX_P || c.n_cap < 2 || c.n_cap > (1 << 22) || c.b_max < 1 ||
      c.b_max > (1 << 16) || c.k < 1 || c.k > FN_MAX_KNN + 1 || c.K < 1 || c.K > FN_MAX_GRID ||
      c.S < 2 || c.S > FN_MAX_S || c.S_clear < 2 || c.S_clear > FN_MAX_S || c.reach_grid < 2 ||
      !(c.T_lo > 0.f) || !(c.T_hi >= c.T_lo) || !(c.w_vel >= 0.f) || !(c.vel_frac >= 0.f))
    return FN_EINVAL;
  fn_planner* pl = new fn_planner();
  pl->cfg = c;
  if (!make_armk(arm, &pl->arm)) {
    delete pl;
    return FN_EINVAL;
  }
  cudaGetDevice(&pl->device);
  for (int k = 0; k < c.K; ++k) {
    const double T = c.K == 1 ? c.T_lo
                              : (double)c.T_lo * std::pow((double)c.T_hi / c.T_lo, (double)k / (c.K - 1));
    pl->grid.T[k] = (float)T;
  }
  PlanDev& D = pl->D;
  memset(&D, 0, sizeof(D));
  D.P = c.P; D.NC = c.n_cap; D.BM = c.b_max; D.KP = c.k; D.KN = std::max(c.k - 1, 1);
  D.KM = (c.k - 1) <= 8 ? 8 : 16;
  D.K = c.K; D.S = c.S; D.S_clear = c.S_clear; D.G = c.reach_grid;
  D.w_vel = c.w_vel; D.vel_frac = c.vel_frac; D.margin = c.clear_margin;
  const size_t P = c.P, NC = c.n_cap, BM = c.b_max, KP = c.k, KN = D.KN, KM = D.KM;
  fn_status rc = FN_OK;
#define A_(ptr, n) if (rc == FN_OK) rc = pl_alloc_n(pl, &(ptr), (n))
  A_(D.st, P * NC * 16); A_(D.t, P * NC); A_(D.par, P * NC); A_(D.J, P * NC);
  A_(D.nu, P * NC); A_(D.eT, P * NC); A_(D.n_nodes, P);
  A_(D.cand, P * BM * 16); A_(D.treq, P * BM); A_(D.vrel, P * BM); A_(D.valid, P * BM);
  A_(D.nn, P * BM * KN);
  A_(D.part_d, P * PL_NSPLIT_MAX * BM * KM); A_(D.part_i, P * PL_NSPLIT_MAX * BM * KM);
  A_(D.e_T, P * BM * KP); A_(D.e_rv, P * BM * KP); A_(D.e_ok, P * BM * KP);
  A_(D.inc, P); A_(D.prob, P); A_(D.sched, 1); A_(D.out, P); A_(D.iter, 1);
  A_(D.added, P); A_(D.status, P);
  A_(D.ptr, P * NC); A_(D.newidx, P * NC); A_(D.alive, P * NC);
  A_(D.tmp_st, P * NC * 16); A_(D.tmp_f, P * NC * 4); A_(D.tmp_par, P * NC);
  A_(D.samples, 1);
#undef A_
  if (rc == FN_OK) {
    if (cudaMallocHost(&pl->h_prob, P * sizeof(fn_problem_t)) != cudaSuccess ||
        cudaMallocHost(&pl->h_out, P * sizeof(fn_rendezvous_t)) != cudaSuccess ||
        cudaMallocHost(&pl->h_iter, sizeof(int)) != cudaSuccess)
      rc = FN_ENOMEM;
  }
  if (rc == FN_OK && (cudaMemset(D.n_nodes, 0, P * sizeof(int)) != cudaSuccess ||
                      cudaMemset(D.samples, 0, sizeof(unsigned long long)) != cudaSuccess))
    rc = FN_ECUDA;
  if (rc != FN_OK) {
    fn_planner_destroy(pl);
    return rc;
  }
  for (int i = 0; i < 8; ++i)
    if (cudaEventCreate(&pl->ev[i]) != cudaSuccess) {
      fn_planner_destroy(pl);
      return FN_ECUDA;
    }
  pl->edge_variant = tuned_variant(TUNE_PLAN_EDGES, (long)c.P * c.b_max * c.k, c.K, c.S);
  pl->edge_blocks = c.edge_blocks > 0 ? c.edge_blocks : plan_edge_blocks(pl, pl->edge_variant);
  *out = pl;
  return FN_OK;
}

static fn_status stage_problems(fn_planner* pl, const fn_problem_t* probs, cudaStream_t st) {
  for (int p = 0; p < pl->cfg.P; ++p) {
    const fn_problem_t& q = probs[p];
    if (q.batch < 0 || q.batch > pl->cfg.b_max || q.n_goal < 0 || q.n_goal > q.batch ||
        q.n_obs < 0 || q.n_obs > FN_MAX_OBS || !(q.t_fall >= q.t_enter) || !(q.v_tip > 0.f))
      return FN_EINVAL;
  }
  memcpy(pl->h_prob, probs, sizeof(fn_problem_t) * pl->cfg.P);
  if (cudaMemcpyAsync(pl->D.prob, pl->h_prob, sizeof(fn_problem_t) * pl->cfg.P,
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return FN_ECUDA;
  return FN_OK;
}

extern "C" fn_status fn_planner_reset(fn_planner_t* pl, const fn_problem_t* probs, void* stream) {
  if (!pl || !probs) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  fn_status rc = stage_problems(pl, probs, st);
  if (rc != FN_OK) return rc;
  k_plan_reset<<<(pl->cfg.P + 127) / 128, 128, 0, st>>>(pl->D);
  rc = launch_status();
  if (rc == FN_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = FN_ECUDA;
  return rc;
}

extern "C" fn_status fn_planner_load_tree(fn_planner_t* pl, int p, const float* states,
                                          const float* t, const int32_t* parent, int n,
                                          void* stream) {
  if (!pl || p < 0 || p >= pl->cfg.P || n < 1 || n > pl->cfg.n_cap || !states || !t || !parent)
    return FN_EINVAL;
  if (parent[0] != -1) return FN_EINVAL;
  for (int i = 1; i < n; ++i)
    if (parent[i] < 0 || parent[i] >= i) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const long nb = (long)p * pl->cfg.n_cap;
  PlanDev& D = pl->D;
  if (cudaMemcpyAsync(D.st + nb * 16, states, sizeof(float) * 16 * n, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(D.t + nb, t, sizeof(float) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(D.par + nb, parent, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    return FN_ECUDA;
  k_plan_loaded<<<(n + 255) / 256, 256, 0, st>>>(D, p, n);
  fn_status rc = launch_status();
  if (rc == FN_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = FN_ECUDA;
  return rc;
}

extern "C" fn_status fn_planner_set_candidates(fn_planner_t* pl, int p, const float* states,
                                               int B, int n_goal, const float* T_req,
                                               const float* v_rel, void* stream) {
  if (!pl || p < 0 || p >= pl->cfg.P || B < 0 || B > pl->cfg.b_max || n_goal < 0 || n_goal > B)
    return FN_EINVAL;
  if (B > 0 && !states) return FN_EINVAL;
  if (n_goal > 0 && (!T_req || !v_rel)) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  PlanDev& D = pl->D;
  const long cb = (long)p * pl->cfg.b_max;
  std::vector<uint8_t> ones(B, 1);
  std::vector<float> nanv(B, NAN);
  if (B > 0) {
    if (cudaMemcpyAsync(D.cand + cb * 16, states, sizeof(float) * 16 * B, cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(D.valid + cb, ones.data(), B, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(D.treq + cb, nanv.data(), sizeof(float) * B, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(D.vrel + cb, nanv.data(), sizeof(float) * B, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
      return FN_ECUDA;
  }
  if (n_goal > 0) {
    if (cudaMemcpyAsync(D.treq + cb, T_req, sizeof(float) * n_goal, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(D.vrel + cb, v_rel, sizeof(float) * n_goal, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
      return FN_ECUDA;
  }
  // the host vectors must outlive the copies
  return cudaStreamSynchronize(st) == cudaSuccess ? FN_OK : FN_ECUDA;
}

// enqueue one iteration (problems and iteration counter already staged)
static fn_status enqueue_iteration(fn_planner* pl, unsigned flags, cudaStream_t st,
                                   bool timed) {
  PlanDev& D = pl->D;
  const int P = pl->cfg.P;
  auto mark = [&](int i) {
    if (timed) cudaEventRecord(pl->ev[i], st);
  };
  mark(0);
  k_plan_schedule<<<1, 32, 0, st>>>(D);
  mark(1);
  if (!(flags & FN_PLAN_EXTERNAL)) {
    const long n = (long)P * D.BM;
    k_plan_sample_goal<<<(unsigned)((4 * n + 127) / 128), 128, 0, st>>>(D, pl->arm);
    k_plan_sample_free<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(D, pl->arm);
  }
  mark(2);
  if (pl->cfg.k > 1) {
    const long nn = (long)P * D.BM * D.KN;
    k_plan_nn_empty<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(D);
    const int kb = 2 * num_sms();
    if (D.KM == 8) {
      k_plan_knn<8><<<kb, 128, 0, st>>>(D);
      k_plan_knn_merge<8><<<(unsigned)(((long)P * D.BM + 7) / 8), 256, 0, st>>>(D);
    } else {
      k_plan_knn<16><<<kb, 128, 0, st>>>(D);
      k_plan_knn_merge<16><<<(unsigned)(((long)P * D.BM + 7) / 8), 256, 0, st>>>(D);
    }
  }
  mark(3);
  plan_edge_variant(pl->edge_variant)<<<pl->edge_blocks, 32 * PL_EDGE_WARPS, 0, st>>>(
      D, pl->arm, pl->grid);
  mark(4);
  k_plan_attach<<<P, PL_ATTACH_THREADS, 0, st>>>(D);
  mark(5);
  if (flags & FN_PLAN_PRUNE) k_plan_prune<<<P, PL_ATTACH_THREADS, 0, st>>>(D, pl->arm);
  mark(6);
  k_plan_output<<<(P + 127) / 128, 128, 0, st>>>(D);
  mark(7);
  if (cudaMemcpyAsync(pl->h_out, D.out, sizeof(fn_rendezvous_t) * P, cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return FN_ECUDA;
  return launch_status();
}

extern "C" fn_status fn_plan_iteration(fn_planner_t* pl, const fn_problem_t* probs, int iter,
                                       unsigned flags, fn_rendezvous_t* out, void* stream) {
  if (!pl || !probs || !out) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  fn_status rc = stage_problems(pl, probs, st);
  if (rc != FN_OK) return rc;
  *pl->h_iter = iter;
  if (cudaMemcpyAsync(pl->D.iter, pl->h_iter, sizeof(int), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return FN_ECUDA;
  rc = enqueue_iteration(pl, flags, st, true);
  if (rc != FN_OK) return rc;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FN_ECUDA;
  memcpy(out, pl->h_out, sizeof(fn_rendezvous_t) * pl->cfg.P);
  pl->timing = true;
  return FN_OK;
}

// durations (ms) of the last fn_plan_iteration's phases, measured with CUDA
// events on its stream: schedule, sample, parents, edges, attach, prune, output
extern "C" fn_status fn_planner_phase_ms(fn_planner_t* pl, float* ms) {
  if (!pl || !ms) return FN_EINVAL;
  if (!pl->timing) return FN_EINVAL;
  for (int i = 0; i < 7; ++i)
    if (cudaEventElapsedTime(&ms[i], pl->ev[i], pl->ev[i + 1]) != cudaSuccess) return FN_ECUDA;
  return FN_OK;
}

extern "C" fn_status fn_planner_capture(fn_planner_t* pl, unsigned flags, void* stream) {
  if (!pl) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (!st) return FN_EINVAL;  // the legacy stream cannot be captured
  if (pl->graph_exec) { cudaGraphExecDestroy(pl->graph_exec); pl->graph_exec = nullptr; }
  if (pl->graph) { cudaGraphDestroy(pl->graph); pl->graph = nullptr; }
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return FN_ECUDA;
  // the staged problems and iteration counter are copied inside the graph
  cudaMemcpyAsync(pl->D.prob, pl->h_prob, sizeof(fn_problem_t) * pl->cfg.P, cudaMemcpyHostToDevice,
                  st);
  cudaMemcpyAsync(pl->D.iter, pl->h_iter, sizeof(int), cudaMemcpyHostToDevice, st);
  fn_status rc = enqueue_iteration(pl, flags, st, false);
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(st, &g) != cudaSuccess || rc != FN_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc != FN_OK ? rc : FN_ECUDA;
  }
  pl->graph = g;
  if (cudaGraphInstantiate(&pl->graph_exec, g, 0) != cudaSuccess) return FN_ECUDA;
  pl->graph_flags = flags;
  return FN_OK;
}

extern "C" fn_status fn_plan_replay(fn_planner_t* pl, const fn_problem_t* probs, int iter,
                                    fn_rendezvous_t* out, void* stream) {
  if (!pl || !probs || !out || !pl->graph_exec) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  for (int p = 0; p < pl->cfg.P; ++p) {
    const fn_problem_t& q = probs[p];
    if (q.batch < 0 || q.batch > pl->cfg.b_max || q.n_goal < 0 || q.n_goal > q.batch ||
        q.n_obs < 0 || q.n_obs > FN_MAX_OBS)
      return FN_EINVAL;
  }
  memcpy(pl->h_prob, probs, sizeof(fn_problem_t) * pl->cfg.P);
  *pl->h_iter = iter;
  if (cudaGraphLaunch(pl->graph_exec, st) != cudaSuccess) return FN_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FN_ECUDA;
  memcpy(out, pl->h_out, sizeof(fn_rendezvous_t) * pl->cfg.P);
  return FN_OK;
}

extern "C" fn_status fn_planner_get_tree(fn_planner_t* pl, int p, float* states, float* t,
                                         int32_t* parent, float* J, float* nu, int* n, int cap) {
  if (!pl || p < 0 || p >= pl->cfg.P || !n) return FN_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return FN_ECUDA;
  int cnt = 0;
  if (cudaMemcpy(&cnt, pl->D.n_nodes + p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return FN_ECUDA;
  *n = cnt;
  const int m = std::min(cnt, cap);
  const long nb = (long)p * pl->cfg.n_cap;
  bool ok = true;
  if (states) ok &= cudaMemcpy(states, pl->D.st + nb * 16, sizeof(float) * 16 * m, cudaMemcpyDeviceToHost) == cudaSuccess;
  if (t) ok &= cudaMemcpy(t, pl->D.t + nb, sizeof(float) * m, cudaMemcpyDeviceToHost) == cudaSuccess;
  if (parent) ok &= cudaMemcpy(parent, pl->D.par + nb, sizeof(int32_t) * m, cudaMemcpyDeviceToHost) == cudaSuccess;
  if (J) ok &= cudaMemcpy(J, pl->D.J + nb, sizeof(float) * m, cudaMemcpyDeviceToHost) == cudaSuccess;
  if (nu) ok &= cudaMemcpy(nu, pl->D.nu + nb, sizeof(float) * m, cudaMemcpyDeviceToHost) == cudaSuccess;
  return ok ? FN_OK : FN_ECUDA;
}

extern "C" fn_status fn_planner_get_candidates(fn_planner_t* pl, int p, float* states,
                                               float* T_req, float* v_rel, uint8_t* valid,
                                               int cap) {
  if (!pl || p < 0 || p >= pl->cfg.P || cap < 0) return FN_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return FN_ECUDA;
  const int m = std::min(cap, pl->cfg.b_max);
  const long cb = (long)p * pl->cfg.b_max;
  bool ok = true;
  if (states) ok &= cudaMemcpy(states, pl->D.cand + cb * 16, sizeof(float) * 16 * m, cudaMemcpyDeviceToHost) == cudaSuccess;
  if (T_req) ok &= cudaMemcpy(T_req, pl->D.treq + cb, sizeof(float) * m, cudaMemcpyDeviceToHost) == cudaSuccess;
  if (v_rel) ok &= cudaMemcpy(v_rel, pl->D.vrel + cb, sizeof(float) * m, cudaMemcpyDeviceToHost) == cudaSuccess;
  if (valid) ok &= cudaMemcpy(valid, pl->D.valid + cb, m, cudaMemcpyDeviceToHost) == cudaSuccess;
  return ok ? FN_OK : FN_ECUDA;
}

// work counter of the edge kernel (torque evaluations since the last reset)
extern "C" fn_status fn_planner_sample_count(fn_planner_t* pl, unsigned long long* count,
                                             int reset) {
  if (!pl || !count) return FN_EINVAL;
  if (cudaMemcpy(count, pl->D.samples, sizeof(unsigned long long), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return FN_ECUDA;
  if (reset && cudaMemset(pl->D.samples, 0, sizeof(unsigned long long)) != cudaSuccess)
    return FN_ECUDA;
  return FN_OK;
}

// Autotuner of the planner's edge kernel: runs the iteration's prefix
// (schedule, samplers unless FN_PLAN_EXTERNAL, parents) once, then times
// every register-budget variant of the persistent edge kernel on that edge
// batch (`reps` runs each, after one warm-up) and keeps the fastest for this
// planner and for planners created later with the same shape.  The tree is
// not modified.  chosen: host (may be NULL); variant_ms: host [3] (may be NULL).
extern "C" fn_status fn_planner_autotune(fn_planner_t* pl, const fn_problem_t* probs, int iter,
                                         unsigned flags, int reps, int* chosen,
                                         float* variant_ms, void* stream) {
  if (!pl || !probs || reps < 1) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  fn_status rc = stage_problems(pl, probs, st);
  if (rc != FN_OK) return rc;
  *pl->h_iter = iter;
  if (cudaMemcpyAsync(pl->D.iter, pl->h_iter, sizeof(int), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return FN_ECUDA;
  PlanDev& D = pl->D;
  const int P = pl->cfg.P;
  k_plan_schedule<<<1, 32, 0, st>>>(D);
  if (!(flags & FN_PLAN_EXTERNAL)) {
    const long n = (long)P * D.BM;
    k_plan_sample_goal<<<(unsigned)((4 * n + 127) / 128), 128, 0, st>>>(D, pl->arm);
    k_plan_sample_free<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(D, pl->arm);
  }
  if (pl->cfg.k > 1) {
    const long nn = (long)P * D.BM * D.KN;
    k_plan_nn_empty<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(D);
    const int kb = 2 * num_sms();
    if (D.KM == 8) {
      k_plan_knn<8><<<kb, 128, 0, st>>>(D);
      k_plan_knn_merge<8><<<(unsigned)(((long)P * D.BM + 7) / 8), 256, 0, st>>>(D);
    } else {
      k_plan_knn<16><<<kb, 128, 0, st>>>(D);
      k_plan_knn_merge<16><<<(unsigned)(((long)P * D.BM + 7) / 8), 256, 0, st>>>(D);
    }
  }
  if ((rc = launch_status()) != FN_OK) return rc;
  float best_ms = INFINITY;
  int best = pl->edge_variant;
  for (int v = 0; v < kEdgeVariants; ++v) {
    const int blocks = pl->cfg.edge_blocks > 0 ? pl->cfg.edge_blocks : plan_edge_blocks(pl, v);
    float tot = 0.f;
    for (int r = 0; r <= reps; ++r) {
      k_plan_schedule<<<1, 32, 0, st>>>(D);  // resets the work queue
      cudaEventRecord(pl->ev[0], st);
      plan_edge_variant(v)<<<blocks, 32 * PL_EDGE_WARPS, 0, st>>>(D, pl->arm, pl->grid);
      cudaEventRecord(pl->ev[1], st);
      if (cudaEventSynchronize(pl->ev[1]) != cudaSuccess) return FN_ECUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, pl->ev[0], pl->ev[1]);
      if (r > 0) tot += ms;
    }
    if ((rc = launch_status()) != FN_OK) return rc;
    const float ms = tot / reps;
    if (variant_ms) variant_ms[v] = ms;
    if (ms < best_ms) { best_ms = ms; best = v; }
  }
  pl->edge_variant = best;
  pl->edge_blocks = pl->cfg.edge_blocks > 0 ? pl->cfg.edge_blocks : plan_edge_blocks(pl, best);
  set_tuned_variant(TUNE_PLAN_EDGES, (long)pl->cfg.P * pl->cfg.b_max * pl->cfg.k, pl->cfg.K,
                    pl->cfg.S, best);
  if (chosen) *chosen = best;
  pl->timing = false;  // the phase events were reused
  return FN_OK;
}
