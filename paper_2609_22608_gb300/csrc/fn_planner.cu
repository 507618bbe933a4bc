// The planner: one round of Algorithm 1 ("FRUITNINJA: one planning cycle",
// Sec. IV-E) for P independent problems at once, entirely on the device.
//
// Memory (Sec. IV-E: "preallocated struct-of-arrays"): every buffer is sized
// once in fn_planner_create for P problems x n_cap nodes x b_max candidates;
// per-problem counts (tree size, incumbent, t_best) live in device memory,
// so an iteration never reads anything back before its end and can be
// captured as a CUDA graph.  One iteration is a fixed sequence of launches
// over all problems (each launched with programmatic dependent launch):
//   schedule : per-problem work offsets, work-queue resets
//   sample   : goal chart (warp per candidate, lane-parallel IK) and
//              uniform candidates (Philox counters); parent-search prep
//              (tree mirror) in the same launch
//   knn      : warps claim (problem, query, node split) items; the warp
//              finishing a query's last split merges the split lists
//   edges    : prep + item scan (eprep, escan, expand), probe of both end
//              samples of every (edge, admissible duration), probe of four
//              interior samples of the survivors (mprobe), verification
//              (vinit, two packed stages + selections, leftover stage),
//              rho_v and clearance at the accepted duration
//   attach   : block per problem: best parent, stable compaction, scoring,
//              incumbent
//   prune    : block per problem (optional): Eq. (reach)
//   output   : rendezvous per problem
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "edge_core.cuh"
#include "fn_internal.h"
#include "tm_scan.cuh"
#include "fn_kin.cuh"
#include "nary_core.cuh"
#include "fn_mlp_tc.h"
#include "fn_tune.h"
#include "knn_core.cuh"

#define PL_NSPLIT_MAX 32
#define PL_KNN_WARPS 4
#ifndef PL_KNN_QW
#define PL_KNN_QW 1                           // queries per warp
#endif
#define PL_KNN_SPAN 4096                      // nodes per split (at least)
#ifndef PL_KNN_SPAN_GOAL
#define PL_KNN_SPAN_GOAL 512                  // the same for goal queries (few, and late)
#endif
#ifndef PL_KNN_SPAN_MIN
#define PL_KNN_SPAN_MIN 1024                  // smallest split of a free query's search
#endif
#ifndef PL_KNN_TW
#define PL_KNN_TW 8                           // tiled search: free queries (one per warp) per CTA
#endif
#ifndef PL_KNN_TRING
#define PL_KNN_TRING 4                        // tiled search: mirror blocks in the CTA's ring
#endif
#ifndef PL_KNN_TILE_NODES
#define PL_KNN_TILE_NODES 32768               // tree capacity from which the tiled search is used
#endif
#define PL_MAX_P 1024
#define PL_MAX_KEV 40                         // launches traced per iteration
#define PL_NCOUNT 14  // work counters: probe, verify, mid-probe, kNN pairs, IK starts,
                      // surrogate-routed edges, surrogate rescans, refine evaluations,
                      // goal draws by outcome (defined, speed, IK, box, singular, taper)
#define PL_CHORD_THREADS 1024

namespace fn {

// best plans of a problem's tree: (J, z) best first, at most n_fit entries
struct Archive {
  int n;
  int pad[3];
  float J[FN_ARCHIVE_MAX];
  float z[FN_ARCHIVE_MAX][9];
};

struct Incumbent {
  int id;
  float J;
  float t_best;
  int pad;
};

struct Sched {
  unsigned int queue_head;
  int n_items;        // probe items of the packed edge phase
  int n_pend[2];      // lengths of the two pending-edge lists
  int n_surv;         // probe survivors appended (may exceed surv_cap)
  int n_dyn;          // edges with probe items listed by the prep (zero between bodies)
  unsigned prep_done; // blocks of k_plan_eprep finished (zero between iterations)
  unsigned att_done;  // blocks of k_attach_scan finished (zero between iterations)
  unsigned prune_done;  // blocks of k_prune_walk finished (zero between iterations)
  unsigned tm_done;    // CTAs of k_plan_edges_tm finished (zero between bodies)
  int n_free_edges;   // free edges of all problems (the queue's first part)
  int n_edges;        // all edges
  // parent-search items (problem, query group, split), one per warp, in two
  // lists: [0] free queries, [1] goal queries (searched after the goal
  // chart has decoded them, in smaller splits)
  int knn_items[2];   // [1] unused: goal items come from the decoded-goal list
  int knn_head[2];    // next unclaimed item of each list
  int gq_n;           // decoded goal queries appended to PlanDev::gq this round
  int nsg_max;        // largest goal split count over the problems
  int free_off[PL_MAX_P + 1];
  int goal_off[PL_MAX_P + 1];
  int knn_off[2][PL_MAX_P + 1];
  int nsplit[2][PL_MAX_P];
  int pack_lo[PL_MAX_P];      // first node of problem p to (re)pack into the mirror
  int pack_off[PL_MAX_P + 1]; // flattened offsets of the nodes to pack
};

struct PlanDev {  // device pointers, passed by value to the kernels
  int P, NC, BM, KP, KN, KM, K, S, S_clear, G;
  int knn_slots;      // resident warps (CTAs when tiled) of the free queries' search grid
  int knn_tile;       // 1: the free queries' search is tiled (PL_KNN_TW queries share a CTA)
  int att_wide;       // 1: attach over many blocks per problem (large batches, few problems)
  int32_t* att_idx;   // [P][BM] a candidate's index among its chunk's attached ones, or -1
  int32_t* att_blk;   // [P][ceil(BM/PL_ATT_T)] attached per chunk, then their offsets
  int32_t* att_tot;   // [P] candidates attached
  unsigned long long* att_key;  // [P] best new rendezvous: ordered J (high), ~node (low)
  int vstages;        // packed verification stages (1 or 2)
  int goal_split;     // 1: goal edges are checked by k_plan_goal_edges, not the packed body
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
  int32_t* knn_cnt;   // [P][BM] splits finished per query (zero between iterations)
  float* e_T;         // [P][BM][KP]
  float* e_rv;
  uint8_t* e_ok;
  int32_t* e_k;       // [P][BM][KP] accepted grid index (-1 none, -2 invalid input)
  Incumbent* inc;     // [P]
  fn_problem_t* prob; // [P]
  Sched* sched;
  fn_rendezvous_t* out;  // [P]
  int* iter;
  // mapped pinned host memory: the staged problems and iteration number
  // (read by k_plan_schedule) and the rendezvous records (written by the
  // kernel that finishes them), so a replay needs no copy nodes
  const fn_problem_t* hprob;
  const int* hiter;
  fn_rendezvous_t* hout;
  int32_t* added;     // [P]
  int32_t* status;    // [P]
  // prune scratch
  int32_t* ptr;       // [P][NC]
  int32_t* newidx;    // [P][NC]
  uint8_t* alive;     // [P][NC]
  float* tmp_st;      // [P][NC][16]
  float* tmp_f;       // [P][NC][4]  (t, J, nu, eT)
  int32_t* tmp_par;   // [P][NC]
  float* tmp_z;       // [P][NC][9]  (chart parameters)
  int32_t* prune_blk; // [P][ceil(NC/PL_PRUNE_T)] kept nodes per chunk, then their offsets
  int32_t* prune_tot; // [P] nodes kept
  int32_t* prune_deep;  // [P] a parent chain longer than PL_PRUNE_WALK: single-block prune
  unsigned long long* samples;  // work counters: torque evaluations [0] probe, [1] verify,
                                // [2] mid-probe; [3] kNN (query, node) pairs; [4] IK starts;
                                // [5] edges timed by the surrogate pass, [6] of them rescanned
  // packed edge phase (flat edge index e in queue order)
  int32_t* e_ci;      // [E] candidate slot p*BM + b
  int32_t* e_par;     // [E] parent node (-1: invalid edge)
  float* e_Tp;        // [E] goal: fixed duration; free: cap
  uint8_t* e_j;       // [E] parent slot | 0x80 for goal edges
  int32_t* e_cnt;     // [E] probe items; then local exclusive offsets
  int32_t* e_klo;     // [E] grid index of the edge's first probe item
  int32_t* blk_off;   // [ceil(E/PL_SCAN)] block offsets of the item scan
  uint32_t* mask;     // [E][8] surviving grid indices of the probe
  int32_t* owner;     // [E*K] probe item -> edge
  int32_t* cur_k;     // [E] duration under verification (grid index; 0 for goals)
  uint32_t* fail;     // [E] a sample of cur_k violated a limit
  int32_t* pend;      // [2][E] edges pending verification (ping-pong lists)
  int2* surv;         // [surv_cap] probe survivors (edge, grid index)
  float* edyn;        // [Emax][2][28] end-sample torque split (alpha, beta, gamma, qd) per end
  int32_t* dyn_list;  // [Emax] edges with probe items (order of listing)
  int Emax, Kmax, surv_cap;
  // duration surrogate: free edges with admissible durations routed to the
  // window pass (sur != 0), listed in sur_list (count *sur_n)
  int sur;
  int32_t* sur_list;  // [E]
  int* sur_n;         // [1]
  // sampling densities (Sec. IV-E, batched expansion)
  fn_density_t* dens; // [P] goal density p_theta (kept across resets)
  struct Archive* arch;  // [P] best plans of the current tree
  float* cz;          // [P][BM][9] chart parameters of the goal candidates (NaN: unknown)
  float* zn;          // [P][NC][9] chart parameters of goal nodes, written at attach
  int32_t* glist;     // [P][BM] the round's valid goal candidates, in order
  int2* gq;           // [P * BM] (problem, slot) of the round's decoded goal queries
  fn_sampler_cfg_t scfg;
  // parents: node mirror laid out for lane-contiguous loads (see knn_mirror_index)
  float4* mir;        // [P][NB][7][32]
  int32_t* packed;    // [P] leading nodes whose mirror entries are current
  int NB;             // 64-node blocks per problem
};

// Programmatic dependent launch: a kernel launched with programmatic
// stream serialization may be scheduled while its predecessor drains; it
// touches nothing the predecessor writes before this wait (a no-op for a
// plain launch), and then lets its own successor be scheduled.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

// A slot in a list that every thread appends to: the lanes of a warp that
// call this together get consecutive slots from one atomic on the counter
// (a single lane's atomic per entry would serialise at the L2 when tens of
// thousands of entries arrive at once).  *n (if non-null) gets the group's
// size on the group's first lane, for a counter kept beside the list.
__device__ __forceinline__ int warp_append(int* counter, unsigned long long* n = nullptr) {
  const unsigned m = __activemask();
  const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) {
    base = atomicAdd(counter, __popc(m));
    if (n) atomicAdd(n, (unsigned long long)__popc(m));
  }
  base = __shfl_sync(m, base, leader);
  return base + __popc(m & ((1u << lane) - 1u));
}

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
  D.packed[p] = 0;
  D.inc[p] = Incumbent{-1, -INFINITY, P.t_fall, 0};
  D.status[p] = 0;
  D.arch[p].n = 0;
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
    D.packed[p] = 0;
    D.inc[p] = Incumbent{-1, -INFINITY, D.prob[p].t_fall, 0};
    D.status[p] = 0;
    D.arch[p].n = 0;
  }
}

// ---------------------------------------------------------------------------
// schedule: per-problem offsets of every flattened work list
// ---------------------------------------------------------------------------
static_assert(sizeof(fn_problem_t) % 16 == 0, "problems copied in 16-byte words");

__global__ void k_plan_schedule(PlanDev D) {
  pdl_begin();
  {   // the staged problems and iteration number, from mapped host memory
    const int nw = D.P * (int)(sizeof(fn_problem_t) / 16);
    const uint4* src = reinterpret_cast<const uint4*>(D.hprob);
    uint4* dst = reinterpret_cast<uint4*>(D.prob);
    for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = __ldcv(src + i);
    if (threadIdx.x == 0) *D.iter = __ldcv(D.hiter);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  Sched* S = D.sched;
  // free queries over all problems: with fewer query groups than resident
  // warps of the parent search, each query's nodes are split further so
  // that every warp gets an item (splits of at least PL_KNN_SPAN_MIN nodes)
  // (groups of PL_KNN_TW queries, one CTA item each, when the search is tiled)
  const int qg = D.knn_tile ? PL_KNN_TW : PL_KNN_QW;
  int qf = 0;
  for (int p = 0; p < D.P; ++p) {
    const int B = min(max(D.prob[p].batch, 0), D.BM);
    const int G = min(max(D.prob[p].n_goal, 0), B);
    if (D.KN > 0 && D.n_nodes[p] > 1) qf += (B - G + qg - 1) / qg;
  }
  const int fill = qf > 0 ? max(1, D.knn_slots / qf) : 1;
  int fo = 0, go = 0, ko = 0, kg = 0, po = 0, nsg_max = 1;
  for (int p = 0; p < D.P; ++p) {
    const fn_problem_t& P = D.prob[p];
    const int B = min(max(P.batch, 0), D.BM);
    const int G = min(max(P.n_goal, 0), B);
    S->free_off[p] = fo;
    S->goal_off[p] = go;
    S->knn_off[0][p] = ko;
    S->knn_off[1][p] = kg;
    fo += (B - G) * D.KP;
    go += G * D.KP;
    const int span = D.n_nodes[p] - 1;  // non-root nodes
    int ns = 1, nsg = 1;
    if (D.KN > 0 && span > 0) {
      ns = max((span + PL_KNN_SPAN - 1) / PL_KNN_SPAN, min(fill, span / PL_KNN_SPAN_MIN));
      ns = min(PL_NSPLIT_MAX, ns);
      nsg = min(PL_NSPLIT_MAX, (span + PL_KNN_SPAN_GOAL - 1) / PL_KNN_SPAN_GOAL);
    }
    S->nsplit[0][p] = ns;
    S->nsplit[1][p] = nsg;
    nsg_max = max(nsg_max, nsg);
    if (D.KN > 0 && span > 0) {
      ko += ((B - G + qg - 1) / qg) * ns;
      kg += ((G + PL_KNN_QW - 1) / PL_KNN_QW) * nsg;
    }
    D.added[p] = 0;
    const int lo = min(D.packed[p], D.n_nodes[p]);
    S->pack_lo[p] = lo;
    S->pack_off[p] = po;
    po += D.n_nodes[p] - lo;
    D.packed[p] = D.n_nodes[p];
  }
  S->pack_off[D.P] = po;
  S->free_off[D.P] = fo;
  S->goal_off[D.P] = go;
  S->knn_off[0][D.P] = ko;
  S->knn_off[1][D.P] = kg;
  S->n_free_edges = fo;
  S->n_edges = fo + (D.goal_split ? 0 : go);
  S->knn_items[0] = ko;
  S->knn_items[1] = kg;
  S->knn_head[0] = 0;
  S->knn_head[1] = 0;
  S->gq_n = 0;
  S->nsg_max = nsg_max;
  if (D.sur_n) *D.sur_n = 0;
  S->queue_head = 0u;
  S->n_dyn = 0;
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
// Gaussian draws folded back into the chart's cube: the angle parameters
// (z2, z3, z4) wrap modulo 1, the others reflect at 0 and 1
__device__ __forceinline__ float z_fold(int i, float z) {
  if (i == 2 || i == 3 || i == 4) return z - floorf(z);
  const float t = z - 2.f * floorf(0.5f * z);
  return t <= 1.f ? t : 2.f - t;
}

// two standard normals from two uniforms in [0, 1) (Box-Muller)
__device__ __forceinline__ void box_muller(float ua, float ub, float& n0, float& n1) {
  const float r = sqrtf(-2.f * logf(1.f - ua));
  float sn, cs;
  sincospif(2.f * ub, &sn, &cs);
  n0 = r * cs;
  n1 = r * sn;
}

// Goal parameters from p_theta: z holds the candidate's uniform draw (the
// uniform component); with probability 1 - w_u a Gaussian component, chosen
// by its weight, replaces it.  The choices are taken in single precision on
// exactly representable uniforms (Philox streams 11-14 of the candidate).
__device__ __forceinline__ void density_z(const fn_density_t& th, unsigned long long seed, int b,
                                          int it, int p, float* z) {
  if (th.C <= 0) return;
  float us[4];
  philox_u4(seed, b, it, p, 11, us);
  if (us[0] < th.w_u) return;
  const float v = (us[0] - th.w_u) / (1.f - th.w_u);
  int m = th.C - 1;
  float acc = 0.f;
  for (int c = 0; c < th.C; ++c) {
    acc += th.pi[c];
    if (v < acc) {
      m = c;
      break;
    }
  }
  float un[12], nrm[10];
#pragma unroll
  for (int s = 0; s < 3; ++s) philox_u4(seed, b, it, p, 12 + s, un + 4 * s);
#pragma unroll
  for (int k = 0; k < 5; ++k) box_muller(un[2 * k], un[2 * k + 1], nrm[2 * k], nrm[2 * k + 1]);
#pragma unroll
  for (int i = 0; i < 9; ++i) z[i] = z_fold(i, fmaf(th.sd[m][i], nrm[i], th.mu[m][i]));
}

// Free candidate (p, b): uniform in the box, |qd| <= vel_frac qdbar.
__device__ __forceinline__ void sample_free(const PlanDev& D, const ArmK& A, int p, int b) {
  const fn_problem_t& P = D.prob[p];
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

__device__ __forceinline__ void parents_prep(const PlanDev& D, long i, long stride);

__device__ __forceinline__ void sample_goal(const PlanDev& D, const ArmK& A, int p, int b, int dens);

// a goal query of this round: a decoded (valid) one joins the goal list of
// the parent search; the others get empty parent lists here
__device__ __forceinline__ void goal_query(const PlanDev& D, int p, int b, bool valid) {
  if (D.KN <= 0) return;
  const long ci = (long)p * D.BM + b;
  if (valid && D.n_nodes[p] > 1) {
    const int v = atomicAdd(&D.sched->gq_n, 1);
    D.gq[v] = make_int2(p, b);
  } else {
    for (int j = 0; j < D.KN; ++j) D.nn[ci * D.KN + j] = -1;
  }
}

// Sampling launches: warp w < nslots (P * b_max, or 0 when the caller gives
// the candidates) owns candidate slot (p, b).
//   role 0: a free slot is drawn by lane 0; the warps past the slots prepare
//           the parent search (parents_prep: tree mirror, empty lists);
//   role 1: a goal slot is decoded by the whole warp (sample_goal).
__global__ void __launch_bounds__(128) k_plan_sample(PlanDev D, ArmK A, long nslots,
                                                     int prep_warps, int dens, int role) {
  pdl_begin();
  const long gid = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (role == 0) {
    const long nsw = (nslots + 31) / 32;              // slot warps: one lane per slot
    if (gid < nsw) {
      const long x = gid * 32 + lane;
      if (x < nslots) {
        const int p = (int)(x / D.BM), b = (int)(x - (long)p * D.BM);
        const int B = min(max(D.prob[p].batch, 0), D.BM);
        if (b >= min(max(D.prob[p].n_goal, 0), B) && b < B) sample_free(D, A, p, b);
      }
    } else if (gid - nsw < prep_warps) {
      const long i = (gid - nsw) * 32 + lane, stride = (long)prep_warps * 32;
      parents_prep(D, i, stride);
      if (nslots == 0)                                // external candidates: list their goals
        for (long x = i; x < (long)D.P * D.BM; x += stride) {
          const int p = (int)(x / D.BM), b = (int)(x - (long)p * D.BM);
          const int B = min(max(D.prob[p].batch, 0), D.BM);
          if (b < min(max(D.prob[p].n_goal, 0), B)) goal_query(D, p, b, D.valid[x] != 0);
        }
    }
  } else if (gid < nslots) {
    const int p = (int)(gid / D.BM);
    const int b = (int)(gid - (long)p * D.BM);
    const int B = min(max(D.prob[p].batch, 0), D.BM);
    if (b < min(max(D.prob[p].n_goal, 0), B)) sample_goal(D, A, p, b, dens);   // warp-uniform
  }
}

// A goal slot: every lane decodes the chart pose, lane groups 0-3 (8 lanes
// each) run the four IK starts in parallel (ik_solve_group) and the lowest
// start that converges wins, the same result as trying the starts in order.
// The draw's outcome (defined, or the condition that left phi undefined) is
// counted in work counters 8..13.
__device__ __forceinline__ void sample_goal(const PlanDev& D, const ArmK& A, int p, int b,
                                            int dens) {
  const int lane = threadIdx.x & 31;
  const fn_problem_t& P = D.prob[p];
  const long ci = (long)p * D.BM + b;
  const int it = *D.iter;
  float u[12], z[9];
#pragma unroll
  for (int s = 0; s < 3; ++s) philox_u4(P.seed, b, it, p, 8 + s, u + 4 * s);
#pragma unroll
  for (int i = 0; i < 9; ++i) z[i] = u[i];
  if (dens) density_z(D.dens[p], P.seed, b, it, p, z);
#pragma unroll
  for (int i = 0; i < 9; ++i)
    if (lane == i) D.cz[ci * 9 + i] = z[i];
  ChartPose o;
  float q[7], qd[7];
  const int why = warp_decode_goal(A, P, z, o, q, qd);
  if (lane != 0) return;
  if (D.samples) {
    if (why != CHART_SPEED) atomicAdd(D.samples + 4, (unsigned long long)FN_IK_STARTS);
    atomicAdd(D.samples + 8 + why, 1ull);
  }
  if (why == CHART_SPEED || why == CHART_IK) {   // undefined before the velocity part
    D.treq[ci] = o.T;
    D.vrel[ci] = o.vrel;
    D.valid[ci] = 0;
    float4* o4 = reinterpret_cast<float4*>(D.cand + ci * 16);
    o4[0] = o4[1] = o4[2] = o4[3] = make_float4(0.f, 0.f, 0.f, 0.f);
    goal_query(D, p, b, false);
    return;
  }
  const bool ok = why == CHART_OK;
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
  goal_query(D, p, b, ok);
}

// ---------------------------------------------------------------------------
// parents: (problem, query group, split) items over all problems, claimed
// by warps one at a time.  A warp takes PL_KNN_QW queries and sweeps the
// split's nodes 64 at a time; the k best
// (d, index) pairs live across lanes 0..KM-1 in ascending order, and only
// nodes that beat the current k-th pair enter the list, one at a time (a
// ballot finds them; a shuffle-up opens their slot), or by a warp merge
// when a ballot holds many of them.
// ---------------------------------------------------------------------------

template <int KM>
struct WarpTopK {
  float d = INFINITY;                         // lane j < KM: j-th best
  int i = 0x7fffffff;
  float td = INFINITY;                        // the k-th best, on every lane
  int ti = 0x7fffffff;
  // Offer the candidates (cd, ci) of the lanes in m (each beat the k-th
  // pair when m was formed): in lane order, a candidate still better than
  // the current k-th pair takes its sorted slot and the tail shifts down.
  // Branch-free in the candidate (a candidate that no longer qualifies
  // gets pos = 32, which moves nothing).
  __device__ __forceinline__ void insert(unsigned m, float cd, int ci) {
    const int lane = threadIdx.x & 31;
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1u;
      const float nd = __shfl_sync(0xffffffffu, cd, src);
      const int ni = __shfl_sync(0xffffffffu, ci, src);
      const bool ok = knn_less(nd, ni, td, ti);
      const unsigned lt = __ballot_sync(0xffffffffu, knn_less(d, i, nd, ni)) & ((1u << KM) - 1u);
      const int pos = ok ? __popc(lt) : 32;
      const float ud = __shfl_up_sync(0xffffffffu, d, 1);
      const int ui = __shfl_up_sync(0xffffffffu, i, 1);
      d = lane < pos ? d : (lane == pos ? nd : ud);
      i = lane < pos ? i : (lane == pos ? ni : ui);
      td = __shfl_sync(0xffffffffu, d, KM - 1);
      ti = __shfl_sync(0xffffffffu, i, KM - 1);
    }
  }
  // The same for many candidates at once (the first block of a split fills
  // an empty list): the KM smallest of the list and the offered candidates
  // by KM rounds of a warp argmin, each winner taken out by its owner (node
  // indices are distinct; the empty entries (inf, max) are all alike).
  __device__ __forceinline__ void merge(unsigned m, float cd, int ci) {
    const int lane = threadIdx.x & 31;
    const bool mine = (m >> lane) & 1u;
    float ld = lane < KM ? d : INFINITY, xd = mine ? cd : INFINITY;
    int li = lane < KM ? i : 0x7fffffff, xi = mine ? ci : 0x7fffffff;
    float nd = INFINITY;
    int ni = 0x7fffffff;
#pragma unroll
    for (int r = 0; r < KM; ++r) {
      const bool fl = knn_less(ld, li, xd, xi);
      float bd = fl ? ld : xd;
      int bi = fl ? li : xi;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float od = __shfl_xor_sync(0xffffffffu, bd, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (knn_less(od, oi, bd, bi)) { bd = od; bi = oi; }
      }
      if (lane == r) { nd = bd; ni = bi; }
      if (ld == bd && li == bi) { ld = INFINITY; li = 0x7fffffff; }
      else if (xd == bd && xi == bi) { xd = INFINITY; xi = 0x7fffffff; }
    }
    d = nd;
    i = ni;
    td = __shfl_sync(0xffffffffu, d, KM - 1);
    ti = __shfl_sync(0xffffffffu, i, KM - 1);
  }
  // one at a time for a few candidates, else the merge
  __device__ __forceinline__ void offer(unsigned m, float cd, int ci) {
    if (__popc(m) >= 2 * KM) merge(m, cd, ci);
    else insert(m, cd, ci);
  }
};

// Merge of a query's split lists (run by the warp that finishes its last
// split): lane s < ns holds split s's list; KN rounds of a warp argmin.
template <int KM>
__device__ __forceinline__ void knn_merge_query(const PlanDev& D, int p, int b, int ns) {
  const int lane = threadIdx.x & 31;
  float d[KM];
  int id[KM];
#pragma unroll
  for (int j = 0; j < KM; ++j) { d[j] = INFINITY; id[j] = 0x7fffffff; }
  if (lane < ns) {
    const long off = (((long)p * PL_NSPLIT_MAX + lane) * D.BM + b) * KM;
#pragma unroll
    for (int j = 0; j < KM; ++j) { d[j] = __ldcg(D.part_d + off + j); id[j] = __ldcg(D.part_i + off + j); }
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

// asynchronous 16-byte global -> shared copy (completion tracked per thread)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

#ifndef PL_KNN_RING
#define PL_KNN_RING 3   // mirror blocks per warp in flight (shared-memory ring)
#endif
constexpr int kKnnSmem = PL_KNN_WARPS * PL_KNN_RING * 7 * 32 * 16;

// One warp per (query group, split): lane j takes nodes 2j and 2j+1 of each
// 64-node block of the split from the mirror and scores both against the
// warp's queries with paired FP32 operations (each half rounds exactly like
// the scalar knn_dist: t = q - x, dq and dv accumulated in component order,
// d = w dv + dq).  The mirror blocks stream through a per-warp ring in
// shared memory, PL_KNN_RING - 1 blocks ahead; each lane copies (cp.async)
// and later reads only its own 16-byte words, so the ring needs no barrier.
template <int KM>
__global__ void __launch_bounds__(32 * PL_KNN_WARPS) k_plan_knn(PlanDev D, int kind) {
  pdl_begin();
  extern __shared__ float4 knn_ring[];   // [warp][slot][7][32]
  const Sched* S = D.sched;
  const int items = kind == 0 ? S->knn_items[0] : S->gq_n * S->nsg_max;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float4* ring = knn_ring + (long)w * PL_KNN_RING * 7 * 32 + lane;
  const float2 w2 = make_float2(D.w_vel, D.w_vel);
  Sched* Sw = D.sched;
  // warp g's first item is g; later ones are claimed from a counter past the
  // grid's warps (a claim per warp at launch would queue every warp on one
  // address)
  const int nw = gridDim.x * PL_KNN_WARPS;
  for (int round = 0;; ++round) {
    int item = blockIdx.x * PL_KNN_WARPS + w;
    if (round > 0) {
      if (lane == 0) item = nw + atomicAdd(&Sw->knn_head[kind], 1);
      item = __shfl_sync(0xffffffffu, item, 0);
    }
    if (item >= items) break;
    int p, ns, split, b0, B;
    if (kind == 0) {   // free queries [G, B) of problem p, PL_KNN_QW per item
      p = find_problem(S->knn_off[0], D.P, item);
      const int local = item - S->knn_off[0][p];
      ns = S->nsplit[0][p];
      const int g = local / ns;
      split = local - g * ns;
      B = min(max(D.prob[p].batch, 0), D.BM);
      b0 = min(max(D.prob[p].n_goal, 0), B) + g * PL_KNN_QW;
    } else {           // one decoded goal query per item: (list entry, split)
      const int v = item / S->nsg_max;
      split = item - v * S->nsg_max;
      const int2 e = D.gq[v];
      p = e.x;
      ns = S->nsplit[1][p];
      if (split >= ns) continue;                 // warp-uniform: a smaller tree
      b0 = e.y;
      B = e.y + 1;
    }
    // candidates whose decoding failed get no parents (their edges are
    // invalid whatever the lists hold)
    bool wact = false;                         // warp-uniform
#pragma unroll
    for (int a = 0; a < PL_KNN_QW; ++a)
      wact |= b0 + a < B && D.valid[(long)p * D.BM + b0 + a];
    const int N = D.n_nodes[p];
    const int span = N - 1;
    const int per = (span + ns - 1) / ns;
    const int lo = 1 + split * per, hi = min(N, lo + per);
    float2 q2[PL_KNN_QW][14];
#pragma unroll
    for (int a = 0; a < PL_KNN_QW; ++a) {
      float qv[14];
      load_query(reinterpret_cast<const float4*>(D.cand) + 4 * ((long)p * D.BM + min(b0 + a, B - 1)),
                 qv);
#pragma unroll
      for (int c = 0; c < 14; ++c) q2[a][c] = make_float2(qv[c], qv[c]);
    }
    WarpTopK<KM> top[PL_KNN_QW];
    const float4* mir = D.mir + (long)p * D.NB * 7 * 32 + lane;
    const int blk0 = lo >> 6, nblk = wact ? ((hi + 63) >> 6) - blk0 : 0;
#pragma unroll
    for (int r = 0; r < PL_KNN_RING - 1; ++r) {   // prologue: blocks 0 .. RING-2
      if (r < nblk)
#pragma unroll
        for (int cc = 0; cc < 7; ++cc)
          cp_async16(ring + (r * 7 + cc) * 32, mir + ((blk0 + r) * 7 + cc) * 32);
      cp_async_commit();
    }
    for (int r = 0; r < nblk; ++r) {
      __syncwarp();   // last round's reads of the slot precede its refill
      {
        const int rn = r + PL_KNN_RING - 1;         // refill the slot freed last round
        if (rn < nblk) {
          const int slot = rn % PL_KNN_RING;
#pragma unroll
          for (int cc = 0; cc < 7; ++cc)
            cp_async16(ring + (slot * 7 + cc) * 32, mir + ((blk0 + rn) * 7 + cc) * 32);
        }
        cp_async_commit();
      }
      cp_async_wait<PL_KNN_RING - 1>();             // this lane's copies of block r landed
      float4 x[7];
      const int slot = r % PL_KNN_RING;
#pragma unroll
      for (int cc = 0; cc < 7; ++cc) x[cc] = ring[(slot * 7 + cc) * 32];
      const int blk = blk0 + r;
      const int n0 = blk * 64 + 2 * lane;
      const bool v0 = n0 >= lo && n0 < hi, v1 = n0 + 1 >= lo && n0 + 1 < hi;
      float2 d[PL_KNN_QW];
#pragma unroll
      for (int a = 0; a < PL_KNN_QW; ++a) {
        float2 dq = make_float2(0.f, 0.f), dv = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 14; ++c) {
          const float4 v = x[c >> 1];
          const float2 nv = (c & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
          const float2 t = __fadd2_rn(q2[a][c], nv);
          if (c < 7) dq = __ffma2_rn(t, t, dq);
          else dv = __ffma2_rn(t, t, dv);
        }
        d[a] = __ffma2_rn(w2, dv, dq);
      }
#pragma unroll
      for (int a = 0; a < PL_KNN_QW; ++a) {
        top[a].offer(__ballot_sync(0xffffffffu, v0 && knn_less(d[a].x, n0, top[a].td, top[a].ti)),
                     d[a].x, n0);
        top[a].offer(__ballot_sync(0xffffffffu, v1 && knn_less(d[a].y, n0 + 1, top[a].td, top[a].ti)),
                     d[a].y, n0 + 1);
      }
    }
    cp_async_wait<0>();
    if (D.samples && lane == 0 && wact) {
      int nq = 0;
#pragma unroll
      for (int a = 0; a < PL_KNN_QW; ++a) nq += b0 + a < B && D.valid[(long)p * D.BM + b0 + a];
      atomicAdd(D.samples + 3, (unsigned long long)nq * (unsigned long long)max(hi - lo, 0));
    }
#pragma unroll
    for (int a = 0; a < PL_KNN_QW; ++a) {
      const int b = b0 + a;
      if (b >= B || lane >= KM) continue;
      const int id = D.valid[(long)p * D.BM + b] ? top[a].i : 0x7fffffff;
      if (ns == 1) {
        if (lane < D.KN) D.nn[((long)p * D.BM + b) * D.KN + lane] = id == 0x7fffffff ? -1 : id;
      } else {
        const long off = (((long)p * PL_NSPLIT_MAX + split) * D.BM + b) * KM + lane;
        D.part_d[off] = top[a].d;
        D.part_i[off] = id;
      }
    }
    if (ns > 1) {
      // the warp that completes a query's last split merges its lists
#pragma unroll
      for (int a = 0; a < PL_KNN_QW; ++a) {
        const int b = b0 + a;
        if (b >= B) continue;
        // every lane's split-list stores are fenced, and the warp has passed
        // its fences, before lane 0 counts the split as finished
        __threadfence();
        __syncwarp();
        int last = 0;
        if (lane == 0) {
          int* cnt = D.knn_cnt + (long)p * D.BM + b;
          last = atomicAdd(cnt, 1) == ns - 1;
          if (last) *cnt = 0;   // ready for the next iteration
        }
        if (__shfl_sync(0xffffffffu, last, 0)) {
          __threadfence();
          knn_merge_query<KM>(D, p, b, ns);
        }
      }
    }
  }
}


// Tiled search of the free queries (planners whose tree capacity is at
// least PL_KNN_TILE_NODES): a CTA of PL_KNN_TW warps claims (problem, group
// of PL_KNN_TW queries, split) items, warp w takes query w of the group.
// The CTA's threads copy each 64-node mirror block of the split once into a
// shared ring (cp.async, PL_KNN_TRING - 1 blocks ahead, one barrier per
// block) and every warp scores it from there as k_plan_knn does (the same
// paired arithmetic, list and tie rule), so a split's nodes leave L2 once
// per PL_KNN_TW queries: on large trees the per-warp search is bound by the
// L2 reads of every query streaming the whole split.  Warps whose query is
// not valid keep to the copies and barriers.
constexpr int kKnnTileSmem = PL_KNN_TRING * 7 * 32 * 16;

template <int KM>
__global__ void __launch_bounds__(32 * PL_KNN_TW) k_plan_knn_tile(PlanDev D) {
  pdl_begin();
  extern __shared__ float4 knn_tring[];   // [slot][7][32]
  __shared__ int s_item;
  const Sched* S = D.sched;
  const int items = S->knn_items[0];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const float2 w2 = make_float2(D.w_vel, D.w_vel);
  Sched* Sw = D.sched;
  for (;;) {
    __syncthreads();   // the last item's ring reads and s_item reads are done
    if (threadIdx.x == 0) s_item = atomicAdd(&Sw->knn_head[0], 1);
    __syncthreads();
    const int item = s_item;
    if (item >= items) break;                  // block-uniform
    const int p = find_problem(S->knn_off[0], D.P, item);
    const int local = item - S->knn_off[0][p];
    const int ns = S->nsplit[0][p];
    const int g = local / ns, split = local - g * ns;
    const int B = min(max(D.prob[p].batch, 0), D.BM);
    const int b = min(max(D.prob[p].n_goal, 0), B) + g * PL_KNN_TW + w;
    const bool mine = b < B;                                    // warp-uniform
    const bool wact = mine && D.valid[(long)p * D.BM + b];     // warp-uniform
    const int N = D.n_nodes[p];
    const int span = N - 1;
    const int per = (span + ns - 1) / ns;
    const int lo = 1 + split * per, hi = min(N, lo + per);
    float2 q2[14];
    {
      float qv[14];
      load_query(reinterpret_cast<const float4*>(D.cand) + 4 * ((long)p * D.BM + (mine ? b : B - 1)),
                 qv);
#pragma unroll
      for (int c = 0; c < 14; ++c) q2[c] = make_float2(qv[c], qv[c]);
    }
    WarpTopK<KM> top;
    const float4* mir = D.mir + (long)p * D.NB * 7 * 32;
    const int blk0 = lo >> 6, nblk = hi > lo ? ((hi + 63) >> 6) - blk0 : 0;   // block-uniform
    auto issue = [&](int r) {   // block r of the split into ring slot r % PL_KNN_TRING
      if (r < nblk) {
        const float4* src = mir + (long)(blk0 + r) * 7 * 32;
        float4* dst = knn_tring + (r % PL_KNN_TRING) * 7 * 32;
        for (int i = threadIdx.x; i < 7 * 32; i += 32 * PL_KNN_TW) cp_async16(dst + i, src + i);
      }
      cp_async_commit();
    };
#pragma unroll
    for (int r = 0; r < PL_KNN_TRING - 1; ++r) issue(r);
    for (int r = 0; r < nblk; ++r) {
      cp_async_wait<PL_KNN_TRING - 2>();   // this thread's copies of block r landed
      __syncthreads();                     // everyone's copies of block r; slot of r - 1 read
      issue(r + PL_KNN_TRING - 1);         // into the slot block r - 1 held
      if (wact) {
        const float4* sl = knn_tring + (r % PL_KNN_TRING) * 7 * 32 + lane;
        float4 x[7];
#pragma unroll
        for (int cc = 0; cc < 7; ++cc) x[cc] = sl[cc * 32];
        const int n0 = (blk0 + r) * 64 + 2 * lane;
        const bool v0 = n0 >= lo && n0 < hi, v1 = n0 + 1 >= lo && n0 + 1 < hi;
        float2 dq = make_float2(0.f, 0.f), dv = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 14; ++c) {
          const float4 v = x[c >> 1];
          const float2 nv = (c & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
          const float2 t = __fadd2_rn(q2[c], nv);
          if (c < 7) dq = __ffma2_rn(t, t, dq);
          else dv = __ffma2_rn(t, t, dv);
        }
        const float2 d = __ffma2_rn(w2, dv, dq);
        top.offer(__ballot_sync(0xffffffffu, v0 && knn_less(d.x, n0, top.td, top.ti)), d.x, n0);
        top.offer(__ballot_sync(0xffffffffu, v1 && knn_less(d.y, n0 + 1, top.td, top.ti)), d.y,
                  n0 + 1);
      }
    }
    cp_async_wait<0>();
    if (D.samples && lane == 0 && wact)
      atomicAdd(D.samples + 3, (unsigned long long)max(hi - lo, 0));
    if (!mine) continue;                       // warp-uniform
    if (lane < KM) {
      const int id = wact ? top.i : 0x7fffffff;
      if (ns == 1) {
        if (lane < D.KN) D.nn[((long)p * D.BM + b) * D.KN + lane] = id == 0x7fffffff ? -1 : id;
      } else {
        const long off = (((long)p * PL_NSPLIT_MAX + split) * D.BM + b) * KM + lane;
        D.part_d[off] = top.d;
        D.part_i[off] = id;
      }
    }
    if (ns > 1) {
      // every lane's split-list stores are fenced, and the warp has passed
      // its fences, before lane 0 counts the split as finished
      __threadfence();
      __syncwarp();
      int last = 0;
      if (lane == 0) {
        int* cnt = D.knn_cnt + (long)p * D.BM + b;
        last = atomicAdd(cnt, 1) == ns - 1;
        if (last) *cnt = 0;   // ready for the next iteration
      }
      if (__shfl_sync(0xffffffffu, last, 0)) {
        __threadfence();
        knn_merge_query<KM>(D, p, b, ns);
      }
    }
  }
}


// Mirror of the tree for the parent search: node n sits in 64-node block
// n / 64 at pair slot j = (n % 64) / 2, half h = n % 2; for component pair
// cc (components 2cc, 2cc+1 of (q_1..q_7, qd_1..qd_7)) the float4
// (x_2j[2cc], x_2j+1[2cc], x_2j[2cc+1], x_2j+1[2cc+1]) holds the values
// negated, so that lane j loads its two nodes' component pairs with seven
// 16-byte loads (512 contiguous bytes per warp instruction) and forms
// q - x as q + (-x), exactly.
__device__ __forceinline__ float* knn_mirror_slot(const PlanDev& D, int p, int n, int cc) {
  const long f4 = (((long)p * D.NB + (n >> 6)) * 7 + cc) * 32 + ((n >> 1) & 31);
  return reinterpret_cast<float*>(D.mir + f4) + (n & 1);
}

// parents prep (thread i of `stride`): neighbour lists of single-node trees
// are empty; tree nodes added (or moved) since the last iteration enter the
// mirror
__device__ __forceinline__ void parents_prep(const PlanDev& D, long i, long stride) {
  if (stride <= 0 || i < 0 || i >= stride) return;
  const long n = (long)D.P * D.BM * D.KN;
  for (long x = i; x < n; x += stride) {
    const int p = (int)(x / ((long)D.BM * D.KN));
    if (D.n_nodes[p] <= 1) D.nn[x] = -1;
  }
  const Sched* S = D.sched;
  const int total = S->pack_off[D.P];
  for (long x = i; x < total; x += stride) {
    const int p = find_problem(S->pack_off, D.P, (int)x);
    const int node = S->pack_lo[p] + (int)(x - S->pack_off[p]);
    const float* r = D.st + ((long)p * D.NC + node) * 16;
#pragma unroll
    for (int cc = 0; cc < 7; ++cc) {
      const int c0 = 2 * cc, c1 = 2 * cc + 1;
      float* slot = knn_mirror_slot(D, p, node, cc);
      slot[0] = -r[c0 < 7 ? c0 : c0 + 1];
      slot[2] = -r[c1 < 7 ? c1 : c1 + 1];
    }
  }
}

#define PL_EDGE_WARPS 4

// ---------------------------------------------------------------------------
// packed edge phase: prep -> item scan -> probe (lanes = (edge, duration)
// items) -> verify (warp per edge, lanes = samples)
// ---------------------------------------------------------------------------
#define PL_SCAN 256
#define PL_PRUNE_T 256   // threads (and nodes) per block of the multi-block prune

// exclusive prefix sum over a block of whole warps, at most 32 (shuffles within the
// warps, one shared pass across them); *total = the block's sum
__device__ __forceinline__ int block_scan(int v, int* sh, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) sh[w] = x;
  __syncthreads();
  const int nw = blockDim.x >> 5;   // whole warps, at most 32
  if (w == 0) {
    int t = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    sh[lane] = t;
  }
  __syncthreads();
  *total = sh[nw - 1];
  const int ex = (w > 0 ? sh[w - 1] : 0) + x - v;
  __syncthreads();   // sh may be reused as soon as this returns
  return ex;
}

// decode flat edge e (queue order: free edges of all problems, then goal
// edges; parent-slot-major inside a problem) into (problem, candidate, slot)
__device__ __forceinline__ void decode_edge(const PlanDev& D, const Sched* S, int e, int& p,
                                            int& b, int& j, bool& goal) {
  const int nfree = S->n_free_edges;
  goal = e >= nfree;
  const int x = goal ? e - nfree : e;
  const int* off = goal ? S->goal_off : S->free_off;
  p = find_problem(off, D.P, x);
  const int local = x - off[p];
  const fn_problem_t& P = D.prob[p];
  const int B = min(max(P.batch, 0), D.BM);
  const int G = min(max(P.n_goal, 0), B);
  const int nc = goal ? G : B - G;
  j = local / nc;
  const int slot = local - j * nc;
  b = goal ? slot : G + slot;
}

// lists the block's edges with probe items (warp-aggregated append) for the
// end-sample torque split; every thread of the block calls it
__device__ __forceinline__ void list_dyn_edge(const PlanDev& D, int e, bool has_items) {
  const unsigned m = __ballot_sync(0xffffffffu, has_items);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == __ffs(m) - 1) base = atomicAdd(&D.sched->n_dyn, __popc(m));
  base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
  if (has_items) D.dyn_list[base + __popc(m & ((1u << lane) - 1u))] = e;
}

// exclusive scan of the per-block item totals (one block of PL_SCAN threads)
__device__ __forceinline__ void scan_block_totals(const PlanDev& D, int* sh) {
  Sched* S = D.sched;
  const int nb = (S->n_edges + PL_SCAN - 1) / PL_SCAN;
  int carry = 0;
  for (int base = 0; base < nb; base += PL_SCAN) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? __ldcg(D.blk_off + i) : 0;
    int tot;
    const int ex = block_scan(v, sh, &tot);
    if (i < nb) D.blk_off[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    S->n_items = carry;
    S->queue_head = 0u;
    S->n_pend[0] = S->n_pend[1] = 0;   // verification lists and probe survivors
    S->n_surv = 0;
  }
}

__global__ void __launch_bounds__(PL_SCAN) k_plan_eprep(PlanDev D, GridKP Gr) {
  pdl_begin();
  __shared__ float sT[FN_MAX_GRID];
  __shared__ int sh[32];
  for (int i = threadIdx.x; i < D.K; i += blockDim.x) sT[i] = Gr.T[i];
  __syncthreads();
  const Sched* S = D.sched;
  const int E = S->n_edges;
  const int e = blockIdx.x * PL_SCAN + threadIdx.x;
  int cnt = 0;
  bool routed = false;
  if (e < E) {
    int p, b, j;
    bool goal;
    decode_edge(D, S, e, p, b, j, goal);
    const long ci = (long)p * D.BM + b;
    const int pr = j == 0 ? 0 : D.nn[ci * D.KN + (j - 1)];
    const long ei = ci * D.KP + j;
    float Tp = NAN;
    const bool valid = pr >= 0 && D.valid[ci];
    if (valid) {
      const float tp = D.t[(long)p * D.NC + pr];
      Tp = goal ? __fsub_rn(D.treq[ci], tp) : __fsub_rn(D.inc[p].t_best, tp);
      if (goal) {
        cnt = (isfinite(Tp) && Tp > 0.f) ? 1 : 0;
      } else {
        int lo = 0, hi = D.K;   // #{k : T_k <= cap} on the ascending grid
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (sT[mid] <= Tp) lo = mid + 1;
          else hi = mid;
        }
        cnt = lo;
        if (D.sur && cnt > 0) {   // timed by the surrogate pass instead
          const int slot = warp_append(D.sur_n);
          if (slot < D.Emax) D.sur_list[slot] = e;
          cnt = 0;
          routed = true;
        }
      }
    }
    D.e_ci[e] = (int)ci;
    D.e_par[e] = valid ? pr : -1;
    D.e_Tp[e] = Tp;
    D.e_j[e] = (uint8_t)(j | (goal ? 0x80 : 0));
    D.e_klo[e] = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) D.mask[8L * e + w] = 0u;
    if (cnt == 0 && !routed) {   // decided without dynamics: invalid or no admissible duration
      D.e_ok[ei] = 0;
      D.e_T[ei] = goal ? Tp : INFINITY;
      D.e_rv[ei] = NAN;
      D.e_k[ei] = -1;
    }
  }
  list_dyn_edge(D, e, e < E && cnt > 0);
  // block-local exclusive scan of the item counts
  int tot;
  const int ex = block_scan(cnt, sh, &tot);
  if (e < E) D.e_cnt[e] = ex;
  // the block that finishes last scans the block totals (the planner's
  // k_plan_escan folded into this launch): each block's total is fenced
  // before the block is counted
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    D.blk_off[blockIdx.x] = tot;
    __threadfence();
    const unsigned done = atomicAdd(&D.sched->prep_done, 1u);
    s_last = done == gridDim.x - 1;
    if (s_last) D.sched->prep_done = 0u;   // ready for the next iteration
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    scan_block_totals(D, sh);
  }
}

__global__ void __launch_bounds__(PL_SCAN) k_plan_escan(PlanDev D) {
  pdl_begin();
  __shared__ int sh[32];
  scan_block_totals(D, sh);
}

__device__ __forceinline__ int item_off(const PlanDev& D, int e) {
  return D.e_cnt[e] + D.blk_off[e / PL_SCAN];
}

// For every listed edge with probe items, one lane per (edge, end, part):
// the item -> owning edge map (the edge's six lanes share its items) and the
// end-sample torque split (end_torque_part's decomposition): three torque
// evaluations per end replace two per item.  The evaluation is the rolled
// recursion (torque_at_rolled) of a cubic whose u = 0 sample is the item's
// (q, qd, qdd), with its coefficients and per-link records in the lane's
// shared-memory columns: each lane evaluates Eq. (torque) about once, so
// the one-link body, fetched once, replaces seven unrolled links the
// instruction cache would fetch cold.  Warps loop in step (every lane of a
// warp makes the same calls); sized to the resident blocks.
#define PL_EXP_WARPS 3
__global__ void __launch_bounds__(32 * PL_EXP_WARPS) k_plan_expand(PlanDev D, ArmK A) {
  pdl_begin();
  __shared__ float sCoef[PL_EXP_WARPS][FN_CUBIC_WORDS * 32];
  __shared__ float sWr[PL_EXP_WARPS][FN_LINK_WORDS * 32];
  __shared__ float4 sLink[7 * FN_LINK_F4];
  fill_links(A, sLink);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const CubicLane cb{&sCoef[w][lane]};
  const LaneLink wr{&sWr[w][lane]};
  const LinkTab L{sLink};
  const Sched* S = D.sched;
  const int E = S->n_edges;
  const int nd = min(S->n_dyn, E);
  const long n = 6L * nd;
  unsigned nsamp = 0;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long x0 = (long)blockIdx.x * blockDim.x + 32 * w; x0 < n; x0 += stride) {
    const long x = x0 + lane;
    const bool act = x < n;
    const int r = (int)(x % 6), end = r / 3, part = r - 3 * end;
    Cubic c;
    float* out = nullptr;
    c.iT = c.iT2 = 1.f;
    if (act) {
      const int e = D.dyn_list[x / 6];
      const int o = item_off(D, e);
      const int cnt = (e + 1 < E ? item_off(D, e + 1) : S->n_items) - o;
      for (int t = r; t < cnt; t += 6) D.owner[o + t] = e;
      const int p = D.e_ci[e] / D.BM;
      const float4* r0 = reinterpret_cast<const float4*>(D.st + ((long)p * D.NC + D.e_par[e]) * 16);
      const float4* r1 = reinterpret_cast<const float4*>(D.cand + (long)D.e_ci[e] * 16);
      float q0[7], qd0[7], q1[7], qd1[7];
      load_state(r0, q0, qd0);
      load_state(r1, q1, qd1);
      out = D.edyn + (2L * e + end) * 28;
#pragma unroll
      for (int j = 0; j < 7; ++j) {   // end_torque_part's (q, qd, qdd) as a cubic at u = 0
        const float d = q1[j] - q0[j];
        const float qa = end ? -6.0f * d : 6.0f * d;
        const float qb = end ? fmaf(4.0f, qd1[j], 2.0f * qd0[j]) : -fmaf(4.0f, qd0[j], 2.0f * qd1[j]);
        c.q0[j] = end ? q1[j] : q0[j];
        c.b1[j] = part == 0 ? (end ? qd1[j] : qd0[j]) : 0.f;
        c.b2[j] = 0.5f * (part == 0 ? 0.f : (part == 1 ? qa : qb));
        c.b3[j] = 0.f;
        if (part == 0) out[21 + j] = c.b1[j];   // the end velocity
      }
      ++nsamp;
    } else {
#pragma unroll
      for (int j = 0; j < 7; ++j) c.q0[j] = c.b1[j] = c.b2[j] = c.b3[j] = 0.f;
    }
    cb.store(c);
    const float on = part == 0 ? 1.f : 0.f;   // parts 1, 2: M + I_m only
    const int o = part == 0 ? 14 : 7 * (part - 1);
    torque_at_rolled(
        A, L, cb, 0.f,
        [&](int j, float tau, float, float) {
          if (act) out[o + j] = tau;
        },
        wr, on, on);
  }
  // one counter update per warp (tens of thousands of same-address atomics
  // from single lanes would serialise at the L2)
  const unsigned tot = __reduce_add_sync(0xffffffffu, nsamp);
  if (D.samples && lane == 0 && tot) atomicAdd(D.samples + 0, (unsigned long long)tot);
}

static int expand_blocks() {
  static int blocks[64] = {0};   // per device: resident blocks of k_plan_expand
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (blocks[dev] == 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plan_expand, 32 * PL_EXP_WARPS,
                                                      0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    blocks[dev] = per_sm * num_sms();
  }
  return blocks[dev];
}

// Probe: one lane per (edge, grid duration) item checks both end samples
// (u = 0, u = 1) from the edge's end-sample torque split: tau = alpha / T^2
// + beta / T + gamma per joint, then rho_tau and rho_P at the end velocity;
// a duration whose ends pass is marked in the edge's survivor mask.  Goal
// edges have one item: their fixed duration.
template <int MINB>
__global__ void __launch_bounds__(32 * PL_EDGE_WARPS, MINB) k_plan_probe(PlanDev D, ArmK A,
                                                                         GridKP Gr) {
  pdl_begin();
  __shared__ float sT[FN_MAX_GRID];
  for (int i = threadIdx.x; i < D.K; i += blockDim.x) sT[i] = Gr.T[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const Sched* S = D.sched;
  const int n_items = S->n_items;
  const long W = (long)gridDim.x * PL_EDGE_WARPS;
  for (long c = (long)blockIdx.x * PL_EDGE_WARPS + w; c * 32 < n_items; c += W) {
    const int i = (int)(c * 32) + lane;
    const bool live = i < n_items;
    int e = 0, k = 0;
    bool pass = live;
    if (live) {
      e = D.owner[i];
      k = D.e_klo[e] + (i - item_off(D, e));
      const bool goal = D.e_j[e] & 0x80;
      const float T = goal ? D.e_Tp[e] : sT[k];
      const float iT = 1.0f / T, iT2 = iT * iT;
#pragma unroll
      for (int end = 0; end < 2; ++end) {
        const float4* c4 = reinterpret_cast<const float4*>(D.edyn) + (2L * e + end) * 7;
        float f[28];
#pragma unroll
        for (int v = 0; v < 7; ++v) {
          const float4 t = __ldg(c4 + v);
          f[4 * v] = t.x; f[4 * v + 1] = t.y; f[4 * v + 2] = t.z; f[4 * v + 3] = t.w;
        }
        float r = 0.f, pw = 0.f;
#pragma unroll
        for (int j = 0; j < 7; ++j) {
          const float tau = fmaf(f[j], iT2, fmaf(f[7 + j], iT, f[14 + j]));
          r = fmaxf(r, fabsf(tau) * A.inv_tau[j]);
          pw = fmaf(tau, f[21 + j], pw);
        }
        pass = pass && r <= 1.f && fabsf(pw) * A.inv_w <= 1.f;
      }
    }
    const unsigned pm = __ballot_sync(0xffffffffu, pass);
    int slot0 = 0;
    if (lane == 0 && pm) slot0 = atomicAdd(&D.sched->n_surv, __popc(pm));
    slot0 = __shfl_sync(0xffffffffu, slot0, 0);
    if (pass) {
      // one atomic per mask word among the warp's passing lanes
      const unsigned grp = __match_any_sync(pm, (unsigned long long)(8L * e + (k >> 5)));
      const unsigned bits = __reduce_or_sync(grp, 1u << (k & 31));
      if (lane == __ffs(grp) - 1) atomicOr(&D.mask[8L * e + (k >> 5)], bits);
      const int slot = slot0 + __popc(pm & ((1u << lane) - 1u));
      if (slot < D.surv_cap) D.surv[slot] = make_int2(e, k);
    }
  }
}

// Mid-probe: lanes = (survivor, interior probe sample) items; a violation
// at any of the four interior points drops the duration from the edge's
// survivor mask before the (much costlier) full verification.  Survivors
// beyond the list's capacity are simply not filtered.
template <int MINB>
__global__ void __launch_bounds__(32 * PL_EDGE_WARPS, MINB) k_plan_mprobe(PlanDev D, ArmK A,
                                                                          GridKP Gr) {
  pdl_begin();
  __shared__ float sT[FN_MAX_GRID];
  __shared__ float sCoef[PL_EDGE_WARPS][FN_CUBIC_WORDS * 32];
  __shared__ float sWr[PL_EDGE_WARPS][FN_WRENCH_WORDS * 32];
  for (int i = threadIdx.x; i < D.K; i += blockDim.x) sT[i] = Gr.T[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const CubicLane cb{&sCoef[w][lane]};
  const LaneWrench wr{&sWr[w][lane]};
  const int ns = min(D.sched->n_surv, D.surv_cap);
  const int n = D.S > 2 ? ns * FN_MID_PROBES : 0;
  unsigned nsamp = 0;
  const long W = (long)gridDim.x * PL_EDGE_WARPS;
  for (long c = (long)blockIdx.x * PL_EDGE_WARPS + w; c * 32 < n; c += W) {
    const int i = (int)(c * 32) + lane;
    const bool live = i < n;
    int e = 0, k = 0, j = 0;
    if (live) {
      const int2 sv = D.surv[i / FN_MID_PROBES];
      j = i % FN_MID_PROBES;
      e = sv.x;
      k = sv.y;
      const bool goal = D.e_j[e] & 0x80;
      const float T = goal ? D.e_Tp[e] : sT[k];
      const int p = D.e_ci[e] / D.BM;
      const float* r0 = D.st + ((long)p * D.NC + D.e_par[e]) * 16;
      const float* r1 = D.cand + (long)D.e_ci[e] * 16;
      float es[32];
#pragma unroll
      for (int m = 0; m < 16; ++m) { es[m] = __ldg(r0 + m); es[16 + m] = __ldg(r1 + m); }
      Cubic cc;
      cubic_coef_sh<false>(es, T, cc);
      cb.store(cc);
    }
    float a = 0.f, b = 0.f;
    if (live) sample_ratios(A, cb, sample_u(mid_probe_index(j, D.S), D.S), a, b, wr);
    nsamp += __popc(__ballot_sync(0xffffffffu, live));
    if (live && !(a <= 1.f && b <= 1.f))
      atomicAnd(&D.mask[8L * e + (k >> 5)], ~(1u << (k & 31)));
  }
  if (D.samples && lane == 0 && nsamp) atomicAdd(D.samples + 2, (unsigned long long)nsamp);
}

// first survivor at or after grid index `from`; -1 if none
__device__ __forceinline__ int next_survivor(const PlanDev& D, int e, int from) {
  for (int q = from >> 5; q < 8; ++q) {
    uint32_t bits = D.mask[8L * e + q];
    if (q == (from >> 5)) bits &= ~0u << (from & 31);
    if (bits) return 32 * q + __ffs(bits) - 1;
  }
  return -1;
}

__device__ __forceinline__ void edge_slot(const PlanDev& D, int e, long& ei, bool& goal) {
  goal = D.e_j[e] & 0x80;
  ei = (long)D.e_ci[e] * D.KP + (D.e_j[e] & 0x7f);
}

// verification start: each edge with probe items either has no survivor
// (infeasible on the whole admissible grid) or joins the first pending list
__global__ void k_plan_vinit(PlanDev D) {
  pdl_begin();
  Sched* S = D.sched;
  const int E = S->n_edges;
  if (blockIdx.x == 0 && threadIdx.x == 0) S->n_dyn = 0;   // the expand consumed the list
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    const int c = (e + 1 < E ? item_off(D, e + 1) : S->n_items) - item_off(D, e);
    if (c == 0) continue;   // decided in prep
    const int k = next_survivor(D, e, 0);
    D.fail[e] = 0u;
    if (k < 0) {
      long ei;
      bool goal;
      edge_slot(D, e, ei, goal);
      D.e_ok[ei] = 0;
      D.e_T[ei] = goal ? D.e_Tp[e] : INFINITY;
      D.e_rv[ei] = NAN;
      D.e_k[ei] = -1;
      continue;
    }
    D.cur_k[e] = k;
    D.pend[warp_append(&S->n_pend[0])] = e;
  }
}

// one packed verification stage: lanes = (pending edge, sample) items; any
// violating sample marks the edge's current duration as failed
template <int MINB>
__global__ void __launch_bounds__(32 * PL_EDGE_WARPS, MINB) k_plan_vstage(PlanDev D, ArmK A,
                                                                          GridKP Gr, int list) {
  pdl_begin();
  __shared__ float sT[FN_MAX_GRID];
  __shared__ float sCoef[PL_EDGE_WARPS][FN_CUBIC_WORDS * 32];
  __shared__ float sWr[PL_EDGE_WARPS][FN_WRENCH_WORDS * 32];
  for (int i = threadIdx.x; i < D.K; i += blockDim.x) sT[i] = Gr.T[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const CubicLane cb{&sCoef[w][lane]};
  const LaneWrench wr{&sWr[w][lane]};
  Sched* S = D.sched;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->n_pend[list ^ 1] = 0;   // filled by the following selection
    S->queue_head = 0u;        // the leftover stage's queue
  }
  const int n = S->n_pend[list] * D.S;
  const int32_t* pend = D.pend + (long)list * D.Emax;
  unsigned nsamp = 0;
  const long W = (long)gridDim.x * PL_EDGE_WARPS;
  for (long c = (long)blockIdx.x * PL_EDGE_WARPS + w; c * 32 < n; c += W) {
    const int i = (int)(c * 32) + lane;
    const bool live = i < n;
    int e = 0, s = 0;
    if (live) {
      const int pi = i / D.S;
      s = i - pi * D.S;
      e = pend[pi];
      const bool goal = D.e_j[e] & 0x80;
      const float T = goal ? D.e_Tp[e] : sT[D.cur_k[e]];
      const int p = D.e_ci[e] / D.BM;
      const float* r0 = D.st + ((long)p * D.NC + D.e_par[e]) * 16;
      const float* r1 = D.cand + (long)D.e_ci[e] * 16;
      float es[32];
#pragma unroll
      for (int m = 0; m < 16; ++m) { es[m] = __ldg(r0 + m); es[16 + m] = __ldg(r1 + m); }
      Cubic cc;
      cubic_coef_sh<true>(es, T, cc);
      cb.store(cc);
    }
    float a = 0.f, b = 0.f;
    if (live) sample_ratios(A, cb, sample_u(s, D.S), a, b, wr);   // single call site
    nsamp += __popc(__ballot_sync(0xffffffffu, live));
    if (live && !(a <= 1.f && b <= 1.f)) D.fail[e] = 1u;
  }
  if (D.samples && lane == 0 && nsamp) atomicAdd(D.samples + 1, (unsigned long long)nsamp);
}

// least link-capsule clearance to problem P's obstacles along the edge
// (staged states es) at duration T, over S_clear points (lane = point)
__device__ __forceinline__ float warp_clearance(const PlanDev& D, const ArmK& A,
                                                const fn_problem_t& P, const float* es, float T) {
  const int lane = threadIdx.x & 31;
  Cubic c;
  cubic_coef_sh<true>(es, T, c);
  float mc = INFINITY;
#pragma unroll 1
  for (int s = lane; s < D.S_clear; s += 32) {
    const float u = sample_u(s, D.S_clear);
    float q[7];
#pragma unroll
    for (int jj = 0; jj < 7; ++jj) {
      float v, a;
      cubic_eval(c, jj, u, q[jj], v, a);
    }
    mc = fminf(mc, config_clearance(A, q, P));
  }
  return -warp_max(-mc);
}

// warp-wide end of an edge whose duration T passed (es: its two states
// staged in shared memory): rho_v at T (lane = joint), the clearance samples
// (lane = sample), then Clear
__device__ __forceinline__ void finish_slot(const PlanDev& D, const ArmK& A, long ei, int p, int k,
                                            float T, const float* es) {
  const int lane = threadIdx.x & 31;
  const float rv = warp_rho_v(A, es, T);
  bool ok = rv <= 1.f;
  const fn_problem_t& P = D.prob[p];
  if (ok && P.n_obs > 0) ok = warp_clearance(D, A, P, es, T) >= D.margin;
  if (lane == 0) {
    D.e_ok[ei] = ok ? 1 : 0;
    D.e_T[ei] = T;
    D.e_rv[ei] = rv;
    D.e_k[ei] = k;
  }
}
__device__ __forceinline__ void finish_edge(const PlanDev& D, const ArmK& A, int e, int k, float T,
                                            const float* es) {
  long ei;
  bool goal;
  edge_slot(D, e, ei, goal);
  finish_slot(D, A, ei, D.e_ci[e] / D.BM, k, T, es);
}

// after a stage: edges whose duration passed are finished; the others move
// to their next survivor (next list) or end with no feasible duration
__global__ void __launch_bounds__(128) k_plan_vselect(PlanDev D, ArmK A, GridKP Gr, int list) {
  pdl_begin();
  __shared__ float sEs[4][32];
  Sched* S = D.sched;
  const int n = S->n_pend[list];
  const int32_t* pend = D.pend + (long)list * D.Emax;
  int32_t* next = D.pend + (long)(list ^ 1) * D.Emax;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = gridDim.x * 4;
  for (int i = blockIdx.x * 4 + w; i < n; i += nw) {   // warp per pending edge
    const int e = pend[i];
    const bool goal = D.e_j[e] & 0x80;
    const int k = D.cur_k[e];
    const bool failed = D.fail[e];
    __syncwarp();
    if (!failed) {
      const int p = D.e_ci[e] / D.BM;
      stage_rows(D.st + ((long)p * D.NC + D.e_par[e]) * 16, D.cand + (long)D.e_ci[e] * 16, sEs[w]);
      finish_edge(D, A, e, goal ? 0 : k, goal ? D.e_Tp[e] : Gr.T[k], sEs[w]);
      continue;
    }
    if (lane != 0) continue;
    D.fail[e] = 0u;
    const int k2 = goal ? -1 : next_survivor(D, e, k + 1);
    if (k2 < 0) {
      long ei;
      bool g;
      edge_slot(D, e, ei, g);
      D.e_ok[ei] = 0;
      D.e_T[ei] = goal ? D.e_Tp[e] : INFINITY;
      D.e_rv[ei] = NAN;
      D.e_k[ei] = -1;
      continue;
    }
    D.cur_k[e] = k2;
    next[warp_append(&S->n_pend[list ^ 1])] = e;
  }
}

// Goal edges (Algorithm 1's goal branch: the cubic from parent p to a
// decoded goal at the fixed duration T_p = T_req - t(p)) checked apart from
// the packed body: every (goal candidate, parent slot) of the round, on the
// paired core with its records in tensor memory (tm_scan.cuh).  CTA b owns a
// contiguous range of the queue's goal part (goal_off).  Its threads decode
// the range a chunk at a time, one edge each: an edge whose parent is
// missing, whose candidate did not decode, or whose T_p is not positive and
// finite is decided there without dynamics (as k_plan_eprep decides it), the
// others join the CTA's list of live edges.  The warps then claim the live
// edges in groups of up to eight, shrinking towards the end of the list so
// that the warps finish together: with more than one edge to a group, one
// probe pass first evaluates eight collocation points of each (both ends and
// six between; lane 4 q + j takes points j and j + 4 of edge q, compensated
// coefficients as the full check, so a violation there is one of the check),
// and only the edges whose probes all pass get the full check at T_p (a warp
// pass per 64 samples, up to the first violating batch).  Then finish_slot's
// velocity and clearance tests.  Launched after the goal queries' parent
// search; it needs nothing of the free edges' phase, which runs beside it.
__device__ __forceinline__ int goal_probe_index(int j, int S) {
  return (int)((2 * j * (S - 1) + 7) / 14);   // round(j (S - 1) / 7), j < 8
}
struct GoalEdge {
  long ei;      // result slot
  int p;        // problem
  int pr;       // parent node (-1: none)
  long ci;      // candidate slot
  float Tp;     // fixed duration (NaN when not valid)
  bool live;    // needs dynamics
};
__device__ __forceinline__ GoalEdge decode_goal_edge(const PlanDev& D, const Sched* S, int x) {
  GoalEdge g;
  g.p = find_problem(S->goal_off, D.P, x);
  const int local = x - S->goal_off[g.p];
  const int G = min(max(D.prob[g.p].n_goal, 0), min(max(D.prob[g.p].batch, 0), D.BM));
  const int j = local / G, b = local - j * G;
  g.ci = (long)g.p * D.BM + b;
  g.ei = g.ci * D.KP + j;
  g.pr = j == 0 ? 0 : D.nn[g.ci * D.KN + (j - 1)];
  const bool valid = g.pr >= 0 && D.valid[g.ci];
  g.Tp = valid ? __fsub_rn(D.treq[g.ci], D.t[(long)g.p * D.NC + g.pr]) : NAN;
  g.live = valid && isfinite(g.Tp) && g.Tp > 0.f;
  return g;
}
__device__ __forceinline__ void goal_edge_fail(const PlanDev& D, const GoalEdge& g) {
  D.e_ok[g.ei] = 0;
  D.e_T[g.ei] = g.Tp;
  D.e_rv[g.ei] = NAN;
  D.e_k[g.ei] = -1;
}
__global__ void __launch_bounds__(32 * TM_WARPS, 1) k_plan_goal_edges(PlanDev D, ArmK A) {
  pdl_begin();
  extern __shared__ float4 tm_smem[];
  const TmBlock blk(tm_smem);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const Sched* S = D.sched;
  const int E = S->goal_off[D.P];
  fill_links2(A, blk.link);
  const int per = (E + (int)gridDim.x - 1) / (int)gridDim.x;
  const int r_lo = min((int)blockIdx.x * per, E), r_hi = min(r_lo + per, E);
  int* list = reinterpret_cast<int*>(blk.split);   // the live edges (the splits' room)
  constexpr int kChunk = (int)(kTmSplit / sizeof(int));
  int* s_n = blk.aux;
  if (w == 0) tmem_alloc(blk.tmem, kTmCols);
  tmem_sync_block();
  const uint32_t tmem = *blk.tmem;
  const PairCore<TmemStash> core = blk.core(tmem, w, lane);
  float* es_g = blk.edges_of(w);
  unsigned nscan = 0;
  for (int c0 = r_lo; c0 < r_hi; c0 += kChunk) {     // CTA-uniform
    const int c1 = min(c0 + kChunk, r_hi);
    if (threadIdx.x == 0) *s_n = 0;
    __syncthreads();
    for (int base = c0; base < c1; base += blockDim.x) {
      const int x = base + threadIdx.x;
      bool lv = false;
      if (x < c1) {
        const GoalEdge g = decode_goal_edge(D, S, x);
        lv = g.live;
        if (!lv) goal_edge_fail(D, g);
      }
      const unsigned m = __ballot_sync(0xffffffffu, lv);   // one atomic per warp
      int at = 0;
      if (m && lane == __ffs(m) - 1) at = atomicAdd(s_n, __popc(m));
      at = __shfl_sync(0xffffffffu, at, m ? __ffs(m) - 1 : 0);
      if (lv) list[at + __popc(m & ((1u << lane) - 1u))] = x;
    }
    if (threadIdx.x == 0) *blk.next = 0;
    __syncthreads();
    const int nl = *s_n;
    for (;;) {   // groups claimed from a shared counter, shrinking towards the end of the list
      int g0 = 0, gs = 0;
      if (lane == 0) {
        const int seen = atomicAdd(blk.next, 0);
        gs = min(8, max(1, (nl - seen) / (2 * TM_WARPS)));
        g0 = atomicAdd(blk.next, gs);
      }
      g0 = __shfl_sync(0xffffffffu, g0, 0);
      gs = __shfl_sync(0xffffffffu, gs, 0);
      if (g0 >= nl) break;                           // warp-uniform
      const int n = min(gs, nl - g0);
      long my_ei = 0;
      int my_p = 0;
      float my_Tp = 0.f;
      for (int i = 0; i < n; ++i) {
        const GoalEdge g = decode_goal_edge(D, S, list[g0 + i]);
        stage_rows(D.st + ((long)g.p * D.NC + g.pr) * 16, D.cand + g.ci * 16, es_g + 32 * i);
        if (lane == i) { my_ei = g.ei; my_p = g.p; my_Tp = g.Tp; }
      }
      unsigned probed = n > 1 ? 0u : 1u;   // a lone edge goes straight to its check
      if (n > 1) {
        const int q = lane >> 2;
        const bool act = q < n;
        const float T = __shfl_sync(0xffffffffu, my_Tp, act ? q : 0);
        {
          Cubic c;
          if (act) {
            cubic_coef_sh<true>(es_g + 32 * q, T, c);
          } else {                                   // an idle lane: any finite cubic
            c.iT = c.iT2 = 1.f;
#pragma unroll
            for (int m = 0; m < 7; ++m) c.q0[m] = c.b1[m] = c.b2[m] = c.b3[m] = 0.f;
          }
          core.store(c);
        }
        const float2 u = make_float2(sample_u(goal_probe_index(lane & 3, D.S), D.S),
                                     sample_u(goal_probe_index((lane & 3) + 4, D.S), D.S));
        float rx = 0.f, px = 0.f, ry = 0.f, py = 0.f;
        core.eval(A, u, dup2(1.f), dup2(1.f), [&](int m, float2 tau, float2 v, float inv_tau) {
          rx = fmaxf(rx, fabsf(tau.x) * inv_tau);
          px = fmaf(tau.x, v.x, px);
          ry = fmaxf(ry, fabsf(tau.y) * inv_tau);
          py = fmaf(tau.y, v.y, py);
        });
        const bool okl = act && rx <= 1.f && fabsf(px) * A.inv_w <= 1.f && ry <= 1.f &&
                         fabsf(py) * A.inv_w <= 1.f;
        const unsigned ok = __ballot_sync(0xffffffffu, okl);
        nscan += 8u * n;
        for (int qq = 0; qq < n; ++qq)
          if (((ok >> (4 * qq)) & 0xFu) == 0xFu) probed |= 1u << qq;
      }
      for (int i = 0; i < n; ++i) {
        const long ei = __shfl_sync(0xffffffffu, my_ei, i);
        const int p = __shfl_sync(0xffffffffu, my_p, i);
        const float Tp = __shfl_sync(0xffffffffu, my_Tp, i);
        int k = -1;
        if ((probed >> i) & 1u) {
          float rt, rp;
          k = edge_scan(A, core, es_g + 32 * i, nullptr, blk.grid, 0, D.S, true, Tp, false, rt,
                        rp, nscan);
          if (k == FN_SCAN_ABORT) {
            if (lane == 0) atomicOr(D.status + p, FN_PLAN_ERR_SCAN);
            k = -1;
          }
        }
        if (k >= 0) {
          finish_slot(D, A, ei, p, 0, Tp, es_g + 32 * i);
        } else if (lane == 0) {
          D.e_ok[ei] = 0;
          D.e_T[ei] = Tp;
          D.e_rv[ei] = NAN;
          D.e_k[ei] = -1;
        }
      }
    }
    __syncthreads();   // the list is read before the next chunk refills it
  }
  if (D.samples && lane == 0 && nscan) atomicAdd(D.samples + 1, (unsigned long long)nscan);
  tmem_sync_block();   // every warp's tensor-memory accesses precede the release
  if (w == 0) tmem_dealloc(tmem, kTmCols);
}

// The warp-per-edge edge body (schedule variant kPairEdgeVariant): the
// edges k_plan_eprep listed for dynamics are timed on the paired core with
// its records in tensor memory (tm_scan.cuh), a warp per edge in shrinking
// runs as the standalone k_time_edges_tm: the end-sample splits of a run in
// one pass, then per edge the scan of Def. "Minimum feasible time" over its
// admissible prefix (free edges: T_k <= the cap T_p) or the check at its
// fixed duration T_p (goal edges, Algorithm 1), and finish_edge's velocity
// and clearance tests.  One launch stands for the packed body's stages
// (expand, probes, verification stages, leftovers); the autotuner takes it
// where an iteration's edges are few enough that the stages' chain of
// launches, not their work, sets the time.  The CTA that finishes last
// empties the dynamics list for the next body.
__global__ void __launch_bounds__(32 * TM_WARPS, 1) k_plan_edges_tm(PlanDev D, ArmK A,
                                                                   GridKP Gr) {
  pdl_begin();
  extern __shared__ float4 tm_smem[];
  const TmBlock blk(tm_smem);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  Sched* S = D.sched;
  const int E = min(S->n_dyn, D.Emax);
  float* sT = blk.grid;
  fill_links2(A, blk.link);
  for (int i = threadIdx.x; i < D.K; i += blockDim.x) sT[i] = Gr.T[i];
  const int per = (E + (int)gridDim.x - 1) / (int)gridDim.x;
  const int r_lo = min((int)blockIdx.x * per, E), r_hi = min(r_lo + per, E);
  if (threadIdx.x == 0) *blk.next = 0;
  if (w == 0) tmem_alloc(blk.tmem, kTmCols);
  tmem_sync_block();
  const uint32_t tmem = *blk.tmem;
  const PairCore<TmemStash> core = blk.core(tmem, w, lane);
  float* es_g = blk.edges_of(w);
  float* split_g = blk.splits_of(w);
  unsigned nsplit = 0, nscan = 0;
  for (;;) {
    int n;
    const int first = tm_claim(blk.next, r_hi - r_lo, n);
    if (n == 0) break;                               // warp-uniform
    const int32_t* run = D.dyn_list + r_lo + first;
    unsigned fin = 0u;
    for (int i = 0; i < n; ++i) {
      const int e = run[i];
      const int p = D.e_ci[e] / D.BM;
      if (stage_rows(D.st + ((long)p * D.NC + D.e_par[e]) * 16, D.cand + (long)D.e_ci[e] * 16,
                     es_g + 32 * i))
        fin |= 1u << i;
    }
    split_group(A, core, es_g, split_g, n, nsplit);
    for (int i = 0; i < n; ++i) {
      const int e = run[i];
      float* es = es_g + 32 * i;
      const bool goal = D.e_j[e] & 0x80;
      const float Tp = D.e_Tp[e];
      int k = -1;
      float rt, rp;
      if ((fin >> i) & 1u) {
        k = goal ? edge_scan(A, core, es, nullptr, sT, 0, D.S, true, Tp, false, rt, rp, nscan)
                 : edge_scan(A, core, es, split_g + FN_SPLIT_WORDS * i, sT,
                             grid_prefix(sT, D.K, Tp), D.S, false, 0.f, false, rt, rp, nscan);
      }
      if (k == FN_SCAN_ABORT) {
        if (lane == 0) atomicOr(D.status + D.e_ci[e] / D.BM, FN_PLAN_ERR_SCAN);
        k = -1;
      }
      if (k >= 0) {
        finish_edge(D, A, e, k, goal ? Tp : sT[k], es);
      } else if (lane == 0) {
        long ei;
        bool g;
        edge_slot(D, e, ei, g);
        D.e_ok[ei] = 0;
        D.e_T[ei] = goal ? Tp : INFINITY;
        D.e_rv[ei] = NAN;
        D.e_k[ei] = -1;
      }
    }
  }
  if (D.samples && lane == 0) {
    if (nsplit) atomicAdd(D.samples + 0, (unsigned long long)nsplit);
    if (nscan) atomicAdd(D.samples + 1, (unsigned long long)nscan);
  }
  tmem_sync_block();   // every warp's tensor-memory accesses precede the release
  if (w == 0) tmem_dealloc(tmem, kTmCols);
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&S->tm_done, 1u) == gridDim.x - 1) {   // every CTA has read the list
      S->n_dyn = 0;
      S->tm_done = 0u;
    }
  }
}

// Leftovers after the packed stages: one block per edge; its four warps take
// the edge's next four survivors (one each, lanes = samples, exit at the
// first violating batch) and the lowest passing survivor is k*; groups of
// four continue until one passes or none remain.  Four-way parallel in the
// survivors cuts the serial depth of edges with long runs of failing
// durations, which otherwise set the kernel's tail.
template <int MINB>
__global__ void __launch_bounds__(32 * PL_EDGE_WARPS, MINB) k_plan_vseq(PlanDev D, ArmK A,
                                                                        GridKP Gr, int list) {
  pdl_begin();
  __shared__ float sT[FN_MAX_GRID];
  __shared__ float sEdge[32];
  __shared__ float sCoef[PL_EDGE_WARPS][FN_CUBIC_WORDS * 32];
  __shared__ float sWr[PL_EDGE_WARPS][FN_WRENCH_WORDS * 32];
  __shared__ int s_item, s_k[PL_EDGE_WARPS], s_pass[PL_EDGE_WARPS], s_from, s_kres, s_done,
      s_groups;
  for (int i = threadIdx.x; i < D.K; i += blockDim.x) sT[i] = Gr.T[i];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const CubicLane cb{&sCoef[w][lane]};
  const LaneWrench wr{&sWr[w][lane]};
  Sched* S = D.sched;
  const int n = S->n_pend[list];
  const int32_t* pend = D.pend + (long)list * D.Emax;
  unsigned nsamp = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (int)atomicAdd(&S->queue_head, 1u);
    __syncthreads();
    const int i = s_item;
    if (i >= n) break;
    const int e = pend[i];
    const int p = D.e_ci[e] / D.BM;
    if (w == 0) stage_rows(D.st + ((long)p * D.NC + D.e_par[e]) * 16, D.cand + (long)D.e_ci[e] * 16, sEdge);
    // Groups of four survivors: warp r verifies the r-th survivor at or after
    // s_from.  Thread 0 alone writes the group state (s_k, s_from, s_kres,
    // s_done), and only between the barriers B1 and B2 of a group; every
    // other thread reads it after B2 (or before the loop), so no write lands
    // while another thread may still read the previous value, and the block
    // leaves the loop together.
    if (threadIdx.x == 0) {
      int k = D.cur_k[e];
      for (int r = 0; r < PL_EDGE_WARPS; ++r) {
        s_k[r] = k;
        if (k >= 0) k = next_survivor(D, e, k + 1);
      }
      s_from = k;   // first survivor of the next group (or -1)
      s_kres = -1;
      s_done = 0;
      s_groups = 1;
    }
    __syncthreads();
    for (;;) {
      const int k = s_k[w];
      bool pass = false;
      if (k >= 0) {
        {
          Cubic c;
          cubic_coef_sh<true>(sEdge, sT[k], c);
          cb.store(c);
        }
        bool bad = false;
        for (int s0 = 0; s0 < D.S && !bad; s0 += 32) {   // single torque call site
          const int s = s0 + lane;
          float a = 0.f, b = 0.f;
          const bool act = s < D.S;
          if (act) sample_ratios(A, cb, sample_u(s, D.S), a, b, wr);
          bad = __any_sync(0xffffffffu, act && !(a <= 1.f && b <= 1.f));
          nsamp += (unsigned)min(32, D.S - s0);
        }
        pass = !bad;
      }
      if (lane == 0) s_pass[w] = pass ? 1 : 0;
      __syncthreads();                                      // B1
      if (threadIdx.x == 0) {
        for (int r = 0; r < PL_EDGE_WARPS && s_kres < 0; ++r)   // lowest passing survivor
          if (s_pass[r] && s_k[r] >= 0) s_kres = s_k[r];
        // next_survivor strictly increases, so an edge has at most
        // ceil(K / 4) groups; the bound stops a loop that would not progress
        const bool stuck = ++s_groups > (D.K + PL_EDGE_WARPS - 1) / PL_EDGE_WARPS + 1;
        if (stuck) atomicOr(D.status + D.e_ci[e] / D.BM, FN_PLAN_ERR_SCAN);
        const int done = s_kres >= 0 || s_from < 0 || stuck;
        if (!done) {                                        // the next group
          int kn = s_from;
          for (int r = 0; r < PL_EDGE_WARPS; ++r) {
            s_k[r] = kn;
            if (kn >= 0) kn = next_survivor(D, e, kn + 1);
          }
          s_from = kn;
        }
        s_done = done;
      }
      __syncthreads();                                      // B2
      if (s_done) break;
    }
    const int kres = s_kres;
    if (w == 0 && kres >= 0) finish_edge(D, A, e, kres, sT[kres], sEdge);
    if (threadIdx.x == 0) {
      if (kres < 0) {
        long ei;
        bool g;
        edge_slot(D, e, ei, g);
        D.e_ok[ei] = 0;
        D.e_T[ei] = INFINITY;
        D.e_rv[ei] = NAN;
        D.e_k[ei] = -1;
      }
    }
  }
  if (D.samples && lane == 0 && nsamp) atomicAdd(D.samples + 1, (unsigned long long)nsamp);
}

// Chord sampler (FN_PLAN_CHORD), one block per problem after the sampling
// launch: the round's valid goals in candidate order, then every free
// candidate whose chord draw succeeds (probability w_chord) is replaced by
// q0 + lambda (q_g - q0) + chord_sigma * half-range * n (clamped to the box)
// toward a goal chosen uniformly; its velocity as for a uniform draw.  Philox
// streams: 0-3 as the uniform draw, 4 (choice, goal, lambda), 5-6 normals.
__global__ void __launch_bounds__(PL_CHORD_THREADS) k_plan_chord(PlanDev D, ArmK A) {
  pdl_begin();
  __shared__ int sh[32];
  const int p = blockIdx.x;
  const fn_problem_t& P = D.prob[p];
  const int B = min(max(P.batch, 0), D.BM);
  const int G = min(max(P.n_goal, 0), B);
  const long cb = (long)p * D.BM;
  const int per = (G + blockDim.x - 1) / blockDim.x;
  const int c0 = min(G, threadIdx.x * per), c1 = min(G, c0 + per);
  int cnt = 0;
  for (int b = c0; b < c1; ++b) cnt += D.valid[cb + b] ? 1 : 0;
  int nv;
  int r = block_scan(cnt, sh, &nv);
  for (int b = c0; b < c1; ++b)
    if (D.valid[cb + b]) D.glist[cb + r++] = b;
  __syncthreads();
  if (nv == 0) return;                 // the free candidates keep their uniform draws
  const int it = *D.iter;
  for (int b = G + threadIdx.x; b < B; b += blockDim.x) {
    float uc[4];
    philox_u4(P.seed, b, it, p, 4, uc);
    if (!(uc[0] < D.scfg.w_chord)) continue;
    const int g = min((int)floorf(uc[1] * (float)nv), nv - 1);
    const float* qg = D.cand + (cb + D.glist[cb + g]) * 16;
    float u[16], un[8], nrm[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) philox_u4(P.seed, b, it, p, k, u + 4 * k);
#pragma unroll
    for (int k = 0; k < 2; ++k) philox_u4(P.seed, b, it, p, 5 + k, un + 4 * k);
#pragma unroll
    for (int k = 0; k < 4; ++k) box_muller(un[2 * k], un[2 * k + 1], nrm[2 * k], nrm[2 * k + 1]);
    float q[7], qd[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      const float lo = A.q_lo[j], hi = A.q_hi[j];
      const float x = P.q0[j] + uc[2] * (qg[j] - P.q0[j]) + D.scfg.chord_sigma * 0.5f * (hi - lo) * nrm[j];
      q[j] = fminf(fmaxf(x, lo), hi);
      qd[j] = fmaf(2.f, u[7 + j], -1.f) * (D.vel_frac * taper(A, j, q[j]));
    }
    float4* o4 = reinterpret_cast<float4*>(D.cand + (cb + b) * 16);
    o4[0] = make_float4(q[0], q[1], q[2], q[3]);
    o4[1] = make_float4(q[4], q[5], q[6], 0.f);
    o4[2] = make_float4(qd[0], qd[1], qd[2], qd[3]);
    o4[3] = make_float4(qd[4], qd[5], qd[6], 0.f);
  }
}

// N-ary refinement (FN_PLAN_NARY), after the verification stages: every free
// edge that found a grid duration T_k gets the rounds of the N-ary search on
// (T_{k-1}, T_k]; rho_v and the clearance are then taken at the refined T,
// which replaces the grid value (Algorithm 1: T_p = min{T <= t_best :
// rho(T) <= 1}, then Clear at T_p).  Persistent warps stride over the free
// edges.
#define PL_REFINE_WARPS 3   // static shared memory of the rolled scan within 48 KB
__global__ void __launch_bounds__(32 * PL_REFINE_WARPS, 4)
    k_plan_refine(PlanDev D, ArmK A, GridKP Gr, float eps, int max_rounds) {
  pdl_begin();
  __shared__ float sEs[PL_REFINE_WARPS][32];
  __shared__ float sSub[PL_REFINE_WARPS][32];
  __shared__ float sCoef[PL_REFINE_WARPS][FN_CUBIC_WORDS * 32];
  __shared__ float sWr[PL_REFINE_WARPS][FN_LINK_WORDS * 32];
  __shared__ __align__(16) float sSplit[PL_REFINE_WARPS][FN_SPLIT_WORDS];
  __shared__ float4 sLink[7 * FN_LINK_F4];
  fill_links(A, sLink);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const CubicLane cb{&sCoef[w][lane]};
  const LaneLink wr{&sWr[w][lane]};
  const LinkTab L{sLink};
  const int nfree = D.sched->n_free_edges;
  unsigned nsamp = 0;
  for (int e = blockIdx.x * PL_REFINE_WARPS + w; e < nfree; e += gridDim.x * PL_REFINE_WARPS) {
    long ei;
    bool goal;
    edge_slot(D, e, ei, goal);
    const int k = D.e_k[ei];
    if (goal || k < 0) continue;                        // warp-uniform
    const int ci = D.e_ci[e];
    const int p = ci / D.BM;
    stage_rows(D.st + ((long)p * D.NC + D.e_par[e]) * 16, D.cand + (long)ci * 16, sEs[w]);
    float a = k > 0 ? Gr.T[k - 1] : 0.f, b = Gr.T[k];
    float rt = NAN, rp = NAN;
    const int rounds = nary_rounds(A, ScalarCore{L, cb, wr}, sEs[w], sSplit[w], sSub[w], D.S,
                                   eps, max_rounds, a, b, -1, rt, rp, nsamp);
    if (rounds == FN_SCAN_ABORT) {                      // keep the grid duration; flag it
      a = k > 0 ? Gr.T[k - 1] : 0.f;
      b = Gr.T[k];
      if (lane == 0) atomicOr(D.status + p, FN_PLAN_ERR_SCAN);
    }
    const float rv = warp_rho_v(A, sEs[w], b);
    bool ok = rv <= 1.f;
    const fn_problem_t& P = D.prob[p];
    if (ok && P.n_obs > 0) ok = warp_clearance(D, A, P, sEs[w], b) >= D.margin;
    if (lane == 0) {
      D.e_T[ei] = b;
      D.e_rv[ei] = rv;
      D.e_ok[ei] = ok ? 1 : 0;
    }
  }
  if (D.samples && lane == 0 && nsamp) atomicAdd(D.samples + 7, (unsigned long long)nsamp);
}

// ---------------------------------------------------------------------------
// attach + score + incumbent: one block per problem
// ---------------------------------------------------------------------------
#define PL_ATTACH_THREADS 1024
#define PL_ATT_T 256             // candidates per block of the multi-block attach
#ifndef PL_ATT_WIDE_B
#define PL_ATT_WIDE_B 4096       // b_max from which (with at most PL_ATT_WIDE_P problems) attach is multi-block
#endif
#define PL_ATT_WIDE_P 16

// the caller's record of problem p: incumbent, its J and time, tree counts,
// status, and the first segment of the incumbent's path
__device__ void write_rendezvous(const PlanDev& D, int p) {
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
  if (D.hout) D.hout[p] = o;
}

// with `output`, thread 0 also writes the problem's record (k_plan_output
// folded into this launch when no later kernel of the iteration changes the
// tree or the incumbent)
__global__ void __launch_bounds__(PL_ATTACH_THREADS) k_plan_attach(PlanDev D, int output) {
  pdl_begin();
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
  // (the flags of a candidate's edges are loaded together, no early exit)
  int cnt = 0;
  for (int b = c0; b < c1; ++b) {
    const long ci = (long)p * D.BM + b;
    int any = 0;
    for (int j0 = 0; j0 < D.KP; j0 += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < D.KP) any |= D.e_ok[ci * D.KP + j0 + u];
    }
    cnt += any != 0;
  }
  int total;
  const int base = block_scan(cnt, sh, &total);
  // pass 2: attach in candidate order (Algorithm 1: argmin_p t(p) + T_p,
  // ties to the lower parent slot)
  float bestJ = -INFINITY;
  int bestI = 0x7fffffff;
  int r = base;
  for (int b = c0; b < c1; ++b) {
    const long ci = (long)p * D.BM + b;
    int bj = -1, bpar = -1;
    float bt = INFINITY;
    for (int j0 = 0; j0 < D.KP; j0 += 8) {   // eight edges' loads in flight at once
      bool ok[8];
      int pr[8];
      float te[8], tp[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + u;
        const long ei = ci * D.KP + j;
        ok[u] = j < D.KP && D.e_ok[ei];
        pr[u] = j == 0 ? 0 : (ok[u] ? D.nn[ci * D.KN + (j - 1)] : 0);
        te[u] = ok[u] ? D.e_T[ei] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) tp[u] = ok[u] ? D.t[nb + pr[u]] : 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float tt = __fadd_rn(tp[u], te[u]);
        if (ok[u] && tt < bt) { bt = tt; bj = j0 + u; bpar = pr[u]; }
      }
    }
    if (bj < 0) continue;
    const int node = N0 + r;
    ++r;
    if (node >= D.NC) {
      atomicOr(&D.status[p], FN_PLAN_TREE_FULL);
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
    if (b < G)
#pragma unroll
      for (int i = 0; i < 9; ++i) D.zn[nd * 9 + i] = D.cz[ci * 9 + i];
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
    if (output) write_rendezvous(D, p);
  }
}

// Multi-block attach (planners with large batches and few problems): the
// same attach as k_plan_attach over PL_ATT_T candidates per block.
// k_attach_scan numbers the attachable candidates of each chunk (the block
// that finishes last turns chunk counts into per-problem offsets, so node
// ids follow candidate order); k_attach_write attaches every candidate to its
// ok parent of least t(p) + T_p (ties to the lower slot) and offers each new
// rendezvous node's (J, id) as one 64-bit key, larger J first, then the lower
// id, to a per-problem atomicMax; k_attach_final sets the tree size and
// replaces the incumbent if the best key's J is strictly better.
__device__ __forceinline__ int att_chunks(const PlanDev& D) {
  return (D.BM + PL_ATT_T - 1) / PL_ATT_T;
}

__global__ void __launch_bounds__(PL_ATT_T) k_attach_scan(PlanDev D) {
  pdl_begin();
  __shared__ int sh[32];
  __shared__ bool s_last;
  const int chunks = att_chunks(D);
  const int p = blockIdx.x / chunks, ch = blockIdx.x - p * chunks;
  const int b = ch * PL_ATT_T + threadIdx.x;
  const int B = min(max(D.prob[p].batch, 0), D.BM);
  int any = 0;
  if (b < B) {
    const long ci = (long)p * D.BM + b;
    for (int j0 = 0; j0 < D.KP; j0 += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < D.KP) any |= D.e_ok[ci * D.KP + j0 + u];
    }
  }
  int tot;
  const int ex = block_scan(any != 0, sh, &tot);
  if (b < B) D.att_idx[(long)p * D.BM + b] = any ? ex : -1;
  if (threadIdx.x == 0) {
    D.att_blk[(long)p * chunks + ch] = tot;
    __threadfence();
    const unsigned done = atomicAdd(&D.sched->att_done, 1u);
    s_last = done == gridDim.x - 1;
    if (s_last) D.sched->att_done = 0u;   // ready for the next iteration
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int q = 0; q < D.P; ++q) {   // chunk counts -> offsets, per problem
    const int nq = (min(max(D.prob[q].batch, 0), D.BM) + PL_ATT_T - 1) / PL_ATT_T;
    int carry = 0;
    for (int base = 0; base < nq; base += PL_ATT_T) {
      const int j = base + threadIdx.x;
      const int v = j < nq ? __ldcg(D.att_blk + (long)q * chunks + j) : 0;
      int t;
      const int e = block_scan(v, sh, &t);
      if (j < nq) D.att_blk[(long)q * chunks + j] = carry + e;
      carry += t;
    }
    if (threadIdx.x == 0) {
      D.att_tot[q] = carry;
      D.att_key[q] = 0ull;   // no new rendezvous node yet
    }
    __syncthreads();
  }
}

// J, ordered as an unsigned integer (larger J -> larger key)
__device__ __forceinline__ unsigned ordered_f32(float x) {
  const unsigned u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void __launch_bounds__(PL_ATT_T) k_attach_write(PlanDev D) {
  pdl_begin();
  __shared__ unsigned long long s_key[PL_ATT_T / 32];
  const int chunks = att_chunks(D);
  const int p = blockIdx.x / chunks, ch = blockIdx.x - p * chunks;
  const int b = ch * PL_ATT_T + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const fn_problem_t& P = D.prob[p];
  const int B = min(max(P.batch, 0), D.BM);
  const int G = min(max(P.n_goal, 0), B);
  const int N0 = D.n_nodes[p];
  const long nb = (long)p * D.NC;
  unsigned long long key = 0ull;
  const int li = b < B ? D.att_idx[(long)p * D.BM + b] : -1;
  if (li >= 0) {
    const long ci = (long)p * D.BM + b;
    int bj = -1, bpar = -1;
    float bt = INFINITY;
    for (int j0 = 0; j0 < D.KP; j0 += 8) {   // eight edges' loads in flight at once
      bool ok[8];
      int pr[8];
      float te[8], tp[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + u;
        const long ei = ci * D.KP + j;
        ok[u] = j < D.KP && D.e_ok[ei];
        pr[u] = j == 0 ? 0 : (ok[u] ? D.nn[ci * D.KN + (j - 1)] : 0);
        te[u] = ok[u] ? D.e_T[ei] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) tp[u] = ok[u] ? D.t[nb + pr[u]] : 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float tt = __fadd_rn(tp[u], te[u]);
        if (ok[u] && tt < bt) { bt = tt; bj = j0 + u; bpar = pr[u]; }
      }
    }
    const int node = N0 + D.att_blk[(long)p * chunks + ch] + li;
    if (node >= D.NC) {
      atomicOr(&D.status[p], FN_PLAN_TREE_FULL);
    } else {
      const long nd = nb + node;
      const float4* src = reinterpret_cast<const float4*>(D.cand + ci * 16);
      float4* dst = reinterpret_cast<float4*>(D.st + nd * 16);
      dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2]; dst[3] = src[3];
      D.t[nd] = bt;
      D.par[nd] = bpar;
      const float nu = fmaxf(D.nu[nb + bpar], D.e_rv[ci * D.KP + bj]);
      D.nu[nd] = nu;
      D.eT[nd] = D.e_T[ci * D.KP + bj];
      float Jv = NAN;
      if (b < G) {
        Jv = objective(P, bt, D.vrel[ci], nu);
        key = ((unsigned long long)ordered_f32(Jv) << 32) | (unsigned)(0xffffffffu - (unsigned)node);
#pragma unroll
        for (int i = 0; i < 9; ++i) D.zn[nd * 9 + i] = D.cz[ci * 9 + i];
      }
      D.J[nd] = Jv;
    }
  }
  // the block's best key, one atomic per block
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o));
  if (lane == 0) s_key[w] = key;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long k = 0ull;
    for (int i = 0; i < PL_ATT_T / 32; ++i) k = max(k, s_key[i]);
    if (k) atomicMax(D.att_key + p, k);
  }
}

__global__ void k_attach_final(PlanDev D, int output) {
  pdl_begin();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= D.P) return;
  const long nb = (long)p * D.NC;
  const int N0 = D.n_nodes[p];
  const int add = min(D.att_tot[p], D.NC - N0);
  D.n_nodes[p] = N0 + add;
  D.added[p] = add;
  const unsigned long long key = D.att_key[p];
  if (key) {
    const int node = (int)(0xffffffffu - (unsigned)(key & 0xffffffffull));
    const float J = D.J[nb + node];
    Incumbent in = D.inc[p];
    if (J > in.J) {
      in.id = node;
      in.J = J;
      in.t_best = D.t[nb + node];
      D.inc[p] = in;
    }
  }
  if (output) write_rendezvous(D, p);
}

// ---------------------------------------------------------------------------
// goal density (FN_PLAN_DENSITY / FN_PLAN_REFIT): one block per problem after
// attach.  Thread 0 inserts the round's new rendezvous nodes whose chart
// parameters are known into the best-plans archive (best J first, a new
// entry after equal ones, at most n_fit); with `refit`, p_theta is refit to
// the archive by EM with diagonal covariances (E-step: thread per plan;
// M-step: thread per (component, parameter)).
// ---------------------------------------------------------------------------
#define PL_DENSITY_THREADS 64   // >= FN_ARCHIVE_MAX and >= 9 * FN_DENSITY_MAX_C

__global__ void __launch_bounds__(PL_DENSITY_THREADS) k_plan_density(PlanDev D, int refit) {
  pdl_begin();
  __shared__ float sz[FN_ARCHIVE_MAX][9];
  __shared__ float sr[FN_ARCHIVE_MAX][FN_DENSITY_MAX_C];
  __shared__ fn_density_t th;
  __shared__ int sn;
  const int p = blockIdx.x;
  const int t = threadIdx.x;
  Archive& ar = D.arch[p];
  if (t == 0) {
    const int N1 = D.n_nodes[p], add = D.added[p];
    const long nb = (long)p * D.NC;
    const int cap = min(max(D.scfg.n_fit, 1), FN_ARCHIVE_MAX);
    int n = min(max(ar.n, 0), cap);
    for (int nd = max(N1 - add, 0); nd < N1; ++nd) {
      const float J = D.J[nb + nd];
      const float* z = D.zn + (nb + nd) * 9;
      bool known = isfinite(J);
      for (int i = 0; i < 9; ++i) known = known && isfinite(z[i]);
      if (!known) continue;
      int pos = n;
      for (int i = 0; i < n; ++i)
        if (J > ar.J[i]) {
          pos = i;
          break;
        }
      if (pos >= cap) continue;
      for (int i = min(n, cap - 1); i > pos; --i) {
        ar.J[i] = ar.J[i - 1];
        for (int k = 0; k < 9; ++k) ar.z[i][k] = ar.z[i - 1][k];
      }
      ar.J[pos] = J;
      for (int k = 0; k < 9; ++k) ar.z[pos][k] = z[k];
      n = min(n + 1, cap);
    }
    ar.n = n;
    sn = n;
    th = D.dens[p];
    if (refit && n > 0 && th.C <= 0) {       // first fit: the best min(C, n) plans
      const int C = min(max(D.scfg.C, 1), min(n, FN_DENSITY_MAX_C));
      th.C = C;
      for (int m = 0; m < C; ++m) {
        th.pi[m] = 1.f / (float)C;
        for (int k = 0; k < 9; ++k) {
          th.mu[m][k] = ar.z[m][k];
          th.sd[m][k] = D.scfg.sd_init;
        }
      }
    }
  }
  __syncthreads();
  const int n = sn;
  if (!refit || n == 0) return;
  if (t < n)
    for (int k = 0; k < 9; ++k) sz[t][k] = ar.z[t][k];
  __syncthreads();
  const int C = th.C;
  const float floor2 = D.scfg.sd_floor * D.scfg.sd_floor;
  for (int itn = 0; itn < D.scfg.em_iters; ++itn) {
    if (t < n) {                              // E-step: responsibilities of plan t
      float lp[FN_DENSITY_MAX_C], top = -INFINITY;
      for (int m = 0; m < C; ++m) {
        float a = th.pi[m] > 0.f ? logf(th.pi[m]) : -INFINITY;
        for (int k = 0; k < 9; ++k) {
          const float d = (sz[t][k] - th.mu[m][k]) / th.sd[m][k];
          a -= 0.5f * d * d + logf(th.sd[m][k]);
        }
        lp[m] = a;
        top = fmaxf(top, a);
      }
      float sum = 0.f;
      for (int m = 0; m < C; ++m) {
        lp[m] = expf(lp[m] - top);
        sum += lp[m];
      }
      for (int m = 0; m < C; ++m) sr[t][m] = lp[m] / sum;
    }
    __syncthreads();
    float mu = 0.f, sd = 0.f, pw = 0.f;
    bool upd = false;
    const int m = t / 9, k = t - 9 * (t / 9);
    if (t < 9 * C) {                          // M-step: component m, parameter k
      float Nm = 0.f, s1 = 0.f;
      for (int i = 0; i < n; ++i) {
        Nm += sr[i][m];
        s1 += sr[i][m] * sz[i][k];
      }
      pw = Nm / (float)n;
      if (Nm >= 1e-4f) {
        mu = s1 / Nm;
        float s2 = 0.f;
        for (int i = 0; i < n; ++i) {
          const float d = sz[i][k] - mu;
          s2 += sr[i][m] * d * d;
        }
        sd = sqrtf(s2 / Nm + floor2);
        upd = true;
      }
    }
    __syncthreads();
    if (t < 9 * C) {
      if (k == 0) th.pi[m] = pw;
      if (upd) {
        th.mu[m][k] = mu;
        th.sd[m][k] = sd;
      }
    }
    __syncthreads();
  }
  if (t == 0) {
    th.w_u = D.scfg.w_u;
    D.dens[p] = th;
  }
}

// ---------------------------------------------------------------------------
// Gradient refinement of the incumbent rendezvous (FN_PLAN_GREFINE; the next
// step the paper's conclusion names: its checks and chart decoder are smooth
// in the trajectory parameters).  Reading: the variables are the node's
// chart parameters z; the objective F(z) is J of Eq. (objective) for phi(z)
// attached to the node's parent (T_p = T_req - t(p) in FP32, nu = max(nu(p),
// rho_v at T_p), J at t(p) + T_p) where phi is defined, T_p > 0 and the edge
// passes Def. "Feasibility Check" and the clearance, -inf elsewhere; the
// gradient is the central difference of the same J (without the check) with
// step h (angle coordinates z2..z4 wrap, the others are clamped, the
// difference divided by the clamped span, 0 where a side is undefined); the
// step is z' = fold(z + eta0 2^-t g / |g|), accepted when F(z') > F(z); a
// zero gradient ends the iterations.  One block per problem: warps 0..17
// take the 18 difference points in parallel, thread 0 forms the step, warp 0
// evaluates z' with the exact check.  An improved node is appended beside
// the original (same parent; a node may already have children) and becomes
// the incumbent.
// ---------------------------------------------------------------------------
#define PL_GR_WARPS 18   // one warp per central-difference point (9 coordinates x 2)

__device__ __forceinline__ bool z_angle(int i) { return i == 2 || i == 3 || i == 4; }

__device__ __forceinline__ float z_clamp_fold(int i, float v) {
  return z_angle(i) ? v - floorf(v) : fminf(fmaxf(v, 0.f), 1.f);
}

// F (check = true) or J (check = false) of phi(z) with the parent state ps
// (global [16]), time tp and nu nup; warp-wide.  es: the warp's staging slot.
// On success with check, q, qd (lane-replicated), Tp and rv describe the node.
__device__ __forceinline__ float warp_node_value(const PlanDev& D, const ArmK& A, LinkTab L,
                                                 CubicLane cb, LaneLink wr,
                                                 const fn_problem_t& P, const float* z,
                                                 const float* ps, float tp, float nup, bool check,
                                                 float* es, float* q, float* qd, float& Tp,
                                                 float& rv) {
  const int lane = threadIdx.x & 31;
  ChartPose o;
  if (warp_decode_goal(A, P, z, o, q, qd) != CHART_OK) return -INFINITY;   // warp-uniform
  Tp = __fsub_rn(o.T, tp);
  if (!(Tp > 0.f)) return -INFINITY;
  // stage the edge (parent state, goal state) as the edge kernels do
  float gv = 0.f;
  const int j = (lane - 16) & 7;
#pragma unroll
  for (int m = 0; m < 7; ++m) {
    if (j == m && lane >= 16 && lane < 24) gv = q[m];
    if (j == m && lane >= 24) gv = qd[m];
  }
  const float v = lane < 16 ? ps[lane] : ((lane & 7) == 7 ? 0.f : gv);
  __syncwarp();
  es[lane] = lane == FN_SPLIT_MARK ? 0.f : v;
  __syncwarp();
  rv = warp_rho_v(A, es, Tp);
  const float J = objective(P, __fadd_rn(tp, Tp), o.vrel, fmaxf(nup, rv));
  if (check) {
    float rt = NAN, rp = NAN;
    unsigned ns = 0;
    bool ok = edge_scan(A, ScalarCore{L, cb, wr}, es, nullptr, nullptr, 0, D.S, true, Tp, true, rt, rp, ns) == 0;
    ok = ok && rv <= 1.f;
    if (ok && P.n_obs > 0) ok = warp_clearance(D, A, P, es, Tp) >= D.margin;
    if (!ok) return -INFINITY;
  }
  return J;
}

__global__ void __launch_bounds__(32 * PL_GR_WARPS) k_plan_grefine(PlanDev D, ArmK A, int iters,
                                                                   float eta0, float h) {
  pdl_begin();
  __shared__ float sEs[PL_GR_WARPS][32];
  __shared__ float sCoef[FN_CUBIC_WORDS * 32];     // warp 0's exact check
  __shared__ float sLk[FN_LINK_WORDS * 32];
  __shared__ float4 sLink[7 * FN_LINK_F4];
  __shared__ float sz[9], szn[9], sJ[PL_GR_WARPS], sSpan[9], sF, sq[7], sqd[7], sTp, srv;
  __shared__ int s_go, s_acc;
  fill_links(A, sLink);
  const int p = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const fn_problem_t& P = D.prob[p];
  const long nb = (long)p * D.NC;
  const int N = D.n_nodes[p];
  const int node = D.inc[p].id;
  // the incumbent: a rendezvous node with known chart parameters, and room
  // for one more node
  bool go = node > 0 && node < N && N < D.NC;
  if (go)
    for (int i = 0; i < 9; ++i) go = go && isfinite(D.zn[(nb + node) * 9 + i]);
  if (!go) return;                                   // uniform over the block
  const int par = D.par[nb + node];
  const float tp = D.t[nb + par], nup = D.nu[nb + par];
  const float* ps = D.st + (nb + par) * 16;
  const LinkTab L{sLink};
  const CubicLane cb{&sCoef[lane]};
  const LaneLink wr{&sLk[lane]};
  if (threadIdx.x < 9) sz[threadIdx.x] = D.zn[(nb + node) * 9 + threadIdx.x];
  if (threadIdx.x == 0) s_acc = 0;
  __syncthreads();
  float q[7], qd[7], Tp = 0.f, rv = 0.f;
  if (w == 0) {
    float z[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) z[i] = sz[i];
    const float F = warp_node_value(D, A, L, cb, wr, P, z, ps, tp, nup, true, sEs[0], q, qd, Tp, rv);
    if (lane == 0) sF = F;
  }
  __syncthreads();
  for (int t = 0; t < iters; ++t) {
    {   // central differences: warp w takes coordinate w / 2, side + for even w
      const int i = w >> 1;
      float z[9];
#pragma unroll
      for (int m = 0; m < 9; ++m) z[m] = sz[m];
      float span;
      if (z_angle(i)) {
        z[i] = z_clamp_fold(i, (w & 1) ? z[i] - h : z[i] + h);
        span = 2.f * h;
      } else {
        const float zp = fminf(z[i] + h, 1.f), zm = fmaxf(z[i] - h, 0.f);
        z[i] = (w & 1) ? zm : zp;
        span = zp - zm;
      }
      float q2[7], qd2[7], Tp2, rv2;
      const float J = warp_node_value(D, A, L, cb, wr, P, z, ps, tp, nup, false, sEs[w], q2, qd2,
                                      Tp2, rv2);
      if (lane == 0) {
        sJ[w] = J;
        if ((w & 1) == 0) sSpan[i] = span;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float g[9], n2 = 0.f;
      for (int i = 0; i < 9; ++i) {
        const float jp = sJ[2 * i], jm = sJ[2 * i + 1];
        g[i] = (isfinite(jp) && isfinite(jm) && sSpan[i] > 0.f) ? (jp - jm) / sSpan[i] : 0.f;
        n2 = fmaf(g[i], g[i], n2);
      }
      const float n = sqrtf(n2);
      s_go = n > 0.f;
      const float step = ldexpf(eta0, -t) / n;
      for (int i = 0; i < 9; ++i) szn[i] = s_go ? z_clamp_fold(i, fmaf(step, g[i], sz[i])) : sz[i];
    }
    __syncthreads();
    if (!s_go) break;                                // uniform: read after the barrier
    if (w == 0) {
      float z[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) z[i] = szn[i];
      float Tn = 0.f, rvn = 0.f;
      const float Fn = warp_node_value(D, A, L, cb, wr, P, z, ps, tp, nup, true, sEs[0], q, qd, Tn,
                                       rvn);
      if (lane == 0 && Fn > sF) {
        sF = Fn;
        for (int i = 0; i < 9; ++i) sz[i] = z[i];
        for (int m = 0; m < 7; ++m) { sq[m] = q[m]; sqd[m] = qd[m]; }
        sTp = Tn;
        srv = rvn;
        ++s_acc;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && s_acc > 0) {               // append the refined rendezvous
    const long nd = nb + N;
    float* s = D.st + nd * 16;
    for (int m = 0; m < 7; ++m) { s[m] = sq[m]; s[8 + m] = sqd[m]; }
    s[7] = 0.f;
    s[15] = 0.f;
    D.t[nd] = __fadd_rn(tp, sTp);
    D.par[nd] = par;
    D.J[nd] = sF;
    D.nu[nd] = fmaxf(nup, srv);
    D.eT[nd] = sTp;
    for (int i = 0; i < 9; ++i) D.zn[nd * 9 + i] = sz[i];
    D.n_nodes[p] = N + 1;
    D.added[p] += 1;
    Incumbent in = D.inc[p];
    in.id = N;
    in.J = sF;
    in.t_best = D.t[nd];
    D.inc[p] = in;
  }
}

// ---------------------------------------------------------------------------
// prune (Eq. (reach)): one block per problem
// ---------------------------------------------------------------------------
// Eq. (reach) for every node of every problem (one thread per node): keep
// the root and the nodes that can reach the object by t_best
__global__ void __launch_bounds__(128) k_plan_reach(PlanDev D, ArmK A) {
  pdl_begin();
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = (int)(gid / D.NC);
  const int i = (int)(gid - (long)p * D.NC);
  if (p >= D.P || i >= D.n_nodes[p]) return;
  const long nb = (long)p * D.NC;
  bool keep = i == 0;
  if (!keep) {
    const fn_problem_t& P = D.prob[p];
    float q[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) q[j] = D.st[(nb + i) * 16 + j];
    const int g = reach_index(A, P, q, D.t[nb + i], D.G);
    if (g >= 0) {
      const float Tg = fmaf((float)g, (P.t_fall - P.t_enter) / (float)(D.G - 1), P.t_enter);
      keep = Tg <= D.inc[p].t_best;
    }
  }
  D.alive[nb + i] = keep ? 1 : 0;
  D.ptr[nb + i] = D.par[nb + i];
}

// Multi-block prune after k_plan_reach (which leaves alive_i = the node's
// own Eq. (reach) test and the root): k_prune_path keeps the incumbent's
// ancestors; k_prune_walk gives each node the AND of alive over its parent
// chain (parents have lower ids, so a chain ends at the root), and numbers the
// kept nodes of its chunk of PL_PRUNE_T (the block that finishes last turns
// the chunk counts into offsets); k_prune_scatter writes the kept nodes,
// parents remapped, to the scratch arrays and k_prune_copy moves them back.
// A chain longer than PL_PRUNE_WALK steps flags its problem, whose prune the
// single-block k_plan_prune then does instead (pointer jumping).
#define PL_PRUNE_WALK 64

__global__ void k_prune_path(PlanDev D) {
  pdl_begin();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= D.P) return;
  const int N = D.n_nodes[p];
  const long nb = (long)p * D.NC;
  int steps = 0;   // parent links point to lower ids: at most N steps
  for (int c = D.inc[p].id; c > 0 && c < N && steps < N; c = D.par[nb + c], ++steps)
    D.alive[nb + c] = 1;
  D.prune_deep[p] = 0;
}

__device__ __forceinline__ int prune_chunks(const PlanDev& D) {
  return (D.NC + PL_PRUNE_T - 1) / PL_PRUNE_T;
}

__global__ void __launch_bounds__(PL_PRUNE_T) k_prune_walk(PlanDev D) {
  pdl_begin();
  __shared__ int sh[32];
  __shared__ bool s_last;
  const int chunks = prune_chunks(D);
  const int p = blockIdx.x / chunks, ch = blockIdx.x - p * chunks;
  const int i = ch * PL_PRUNE_T + threadIdx.x;
  const int N = D.n_nodes[p];
  const long nb = (long)p * D.NC;
  int keep = 0;
  if (i < N) {
    int a = D.alive[nb + i];
    int c = D.par[nb + i];
    for (int steps = 0; a && c > 0 && steps < PL_PRUNE_WALK; ++steps) {
      a &= D.alive[nb + c];
      c = D.par[nb + c];
    }
    if (a && c > 0) atomicOr(D.prune_deep + p, 1);   // longer than the walk: fallback
    keep = a;
  }
  int tot;
  const int ex = block_scan(keep, sh, &tot);
  if (i < N) D.newidx[nb + i] = keep ? ex : -1;   // index within the chunk
  if (threadIdx.x == 0) {
    D.prune_blk[(long)p * chunks + ch] = tot;
    __threadfence();
    const unsigned done = atomicAdd(&D.sched->prune_done, 1u);
    s_last = done == gridDim.x - 1;
    if (s_last) D.sched->prune_done = 0u;   // ready for the next iteration
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int q = 0; q < D.P; ++q) {   // chunk counts -> offsets, per problem
    const int nq = (D.n_nodes[q] + PL_PRUNE_T - 1) / PL_PRUNE_T;
    int carry = 0;
    for (int base = 0; base < nq; base += PL_PRUNE_T) {
      const int j = base + threadIdx.x;
      const int v = j < nq ? __ldcg(D.prune_blk + (long)q * chunks + j) : 0;
      int t;
      const int e = block_scan(v, sh, &t);
      if (j < nq) D.prune_blk[(long)q * chunks + j] = carry + e;
      carry += t;
    }
    if (threadIdx.x == 0) D.prune_tot[q] = carry;
    __syncthreads();
  }
}

// new index of kept node i of problem p (chunk offset + index within the chunk)
__device__ __forceinline__ int prune_newidx(const PlanDev& D, int p, int i) {
  const long nb = (long)p * D.NC;
  return D.prune_blk[(long)p * prune_chunks(D) + i / PL_PRUNE_T] + D.newidx[nb + i];
}

__global__ void __launch_bounds__(PL_PRUNE_T) k_prune_scatter(PlanDev D) {
  pdl_begin();
  const int chunks = prune_chunks(D);
  const int p = blockIdx.x / chunks, ch = blockIdx.x - p * chunks;
  const int i = ch * PL_PRUNE_T + threadIdx.x;
  const long nb = (long)p * D.NC;
  if (D.prune_deep[p] || i >= D.n_nodes[p] || D.newidx[nb + i] < 0) return;
  const int ni = prune_newidx(D, p, i);
  const float4* src = reinterpret_cast<const float4*>(D.st + (nb + i) * 16);
  float4* dst = reinterpret_cast<float4*>(D.tmp_st + (nb + ni) * 16);
  dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2]; dst[3] = src[3];
  const int pa = D.par[nb + i];
  D.tmp_par[nb + ni] = pa >= 0 ? prune_newidx(D, p, pa) : -1;   // a kept node's parent is kept
  float* tf = D.tmp_f + (nb + ni) * 4;
  tf[0] = D.t[nb + i]; tf[1] = D.J[nb + i]; tf[2] = D.nu[nb + i]; tf[3] = D.eT[nb + i];
#pragma unroll
  for (int k = 0; k < 9; ++k) D.tmp_z[(nb + ni) * 9 + k] = D.zn[(nb + i) * 9 + k];
}

__global__ void __launch_bounds__(PL_PRUNE_T) k_prune_copy(PlanDev D) {
  pdl_begin();
  const int chunks = prune_chunks(D);
  const int p = blockIdx.x / chunks, ch = blockIdx.x - p * chunks;
  const int i = ch * PL_PRUNE_T + threadIdx.x;
  const long nb = (long)p * D.NC;
  if (D.prune_deep[p]) return;
  const int total = D.prune_tot[p];
  if (i < total) {
    const float4* src = reinterpret_cast<const float4*>(D.tmp_st + (nb + i) * 16);
    float4* dst = reinterpret_cast<float4*>(D.st + (nb + i) * 16);
    dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2]; dst[3] = src[3];
    D.par[nb + i] = D.tmp_par[nb + i];
    const float* tf = D.tmp_f + (nb + i) * 4;
    D.t[nb + i] = tf[0]; D.J[nb + i] = tf[1]; D.nu[nb + i] = tf[2]; D.eT[nb + i] = tf[3];
#pragma unroll
    for (int k = 0; k < 9; ++k) D.zn[(nb + i) * 9 + k] = D.tmp_z[(nb + i) * 9 + k];
  }
  if (ch == 0 && threadIdx.x == 0) {
    const int N = D.n_nodes[p];
    D.n_nodes[p] = total;
    if (total != N) D.packed[p] = 0;   // indices moved: repack the mirror
    const Incumbent in = D.inc[p];
    if (in.id >= 0 && in.id < N) {
      Incumbent o = in;
      o.id = D.newidx[nb + in.id] >= 0 ? prune_newidx(D, p, in.id) : -1;
      D.inc[p] = o;
    }
  }
}

// The single-block prune (one block per problem), for problems whose walk
// met a parent chain longer than PL_PRUNE_WALK: pointer jumping, then a
// stable compaction with parent remap (through the scratch arrays).
__global__ void __launch_bounds__(PL_ATTACH_THREADS) k_plan_prune(PlanDev D, ArmK A) {
  pdl_begin();
  __shared__ int sh[PL_ATTACH_THREADS];
  __shared__ int s_flag;
  const int p = blockIdx.x;
  if (!D.prune_deep[p]) return;   // block-uniform: the multi-block prune did it
  const int N = D.n_nodes[p];
  const long nb = (long)p * D.NC;
  const Incumbent in = D.inc[p];
  (void)A;
  if (threadIdx.x == 0) {   // parent links point to lower ids: at most N steps
    int steps = 0;
    for (int c = in.id; c > 0 && c < N && steps < N; c = D.par[nb + c], ++steps)
      D.alive[nb + c] = 1;
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
  int r = block_scan(cnt, sh, &total);
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
#pragma unroll
    for (int k = 0; k < 9; ++k) D.tmp_z[(nb + ni) * 9 + k] = D.zn[(nb + i) * 9 + k];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const float4* src = reinterpret_cast<const float4*>(D.tmp_st + (nb + i) * 16);
    float4* dst = reinterpret_cast<float4*>(D.st + (nb + i) * 16);
    dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2]; dst[3] = src[3];
    D.par[nb + i] = D.tmp_par[nb + i];
    const float* tf = D.tmp_f + (nb + i) * 4;
    D.t[nb + i] = tf[0]; D.J[nb + i] = tf[1]; D.nu[nb + i] = tf[2]; D.eT[nb + i] = tf[3];
#pragma unroll
    for (int k = 0; k < 9; ++k) D.zn[(nb + i) * 9 + k] = D.tmp_z[(nb + i) * 9 + k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    D.n_nodes[p] = total;
    if (total != N) D.packed[p] = 0;   // indices moved: repack the mirror
    if (in.id >= 0) {
      Incumbent o = in;
      o.id = D.newidx[nb + in.id];
      D.inc[p] = o;
    }
  }
}

// ---------------------------------------------------------------------------
// the incumbent plan of problem p as edges, root first (the plan that the
// full-resolution recheck of Sec. IV-E takes): edge i runs from nodes[i] to
// nodes[i + 1], with the duration stored with its end node.  *n_edges = the
// path length L (0: no incumbent), -1 if the parent links do not lead to
// the root; the arrays are written when 0 < L <= max_edges.  One thread: a
// path is a few dozen edges.
__global__ void k_plan_path(PlanDev D, int p, int max_edges, float* __restrict__ s0,
                            float* __restrict__ s1, float* __restrict__ T,
                            int32_t* __restrict__ nodes, int32_t* __restrict__ n_edges) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const long nb = (long)p * D.NC;
  const int n = D.n_nodes[p];
  const int inc = D.inc[p].id;
  int L = 0;
  if (inc >= n) {
    L = -1;
  } else if (inc > 0) {
    int v = inc;
    while (v != 0) {
      const int pv = D.par[nb + v];
      if (pv < 0 || pv >= n || L >= n) {
        L = -1;
        break;
      }
      v = pv;
      ++L;
    }
  }
  *n_edges = L;
  if (L <= 0 || L > max_edges) return;
  int v = inc;
  for (int i = L; i > 0; --i) {
    const int pv = D.par[nb + v];
    if (nodes) nodes[i] = v;
    T[i - 1] = D.eT[nb + v];
    for (int j = 0; j < 16; ++j) {
      s0[16L * (i - 1) + j] = D.st[(nb + pv) * 16 + j];
      s1[16L * (i - 1) + j] = D.st[(nb + v) * 16 + j];
    }
    v = pv;
  }
  if (nodes) nodes[0] = 0;
}

// output: the first segment of the incumbent plan (Algorithm 1's return)
// ---------------------------------------------------------------------------
__global__ void k_plan_output(PlanDev D) {
  pdl_begin();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= D.P) return;
  write_rendezvous(D, p);
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
  fn_problem_t* h_reset = nullptr;     // pinned staging of fn_planner_reset (its own copy)
  fn_rendezvous_t* h_out = nullptr;    // pinned
  int* h_iter = nullptr;               // pinned
  cudaEvent_t replay_done = nullptr;   // the last asynchronous replay (its staging and output)
  bool replay_pending = false;         // an asynchronous replay may still read the staging
  cudaEvent_t reset_done = nullptr;    // the last reset's copy of the staged problems
  bool reset_pending = false;          // that copy may still read the staging
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  unsigned graph_flags = 0;
  int edge_variant = kDefaultEdgeVariant;
  int edge_blocks = 0;
  // per-phase events: schedule, sample, parents, edge prep + scan, probe,
  // verify, attach, prune, output
  cudaEvent_t ev[10] = {};
  bool timing = false;
  // duration surrogate (fn_planner_set_surrogate): the model, the window and
  // the surrogate pass's buffers (its own schedule, compacted rows, results)
  fn_mlp* sur_mlp = nullptr;
  int sur_W = 16;
  Sched* sched2 = nullptr;
  fn_problem_t* no_obs = nullptr;       // device: a problem without obstacles
  float *g_s0 = nullptr, *g_s1 = nullptr, *g_cap = nullptr, *g_Y = nullptr;
  int32_t* g_k = nullptr;
  float *g_T = nullptr, *g_rv = nullptr;
  uint8_t *g_ok = nullptr, *g_path = nullptr;
  int2* g_win = nullptr;
  int32_t* g_fb = nullptr;
  int* g_fbn = nullptr;
  int32_t* g_slot = nullptr;
  float logT0 = 0.f, dlog = 0.f;
  // N-ary refinement of the free edges (fn_planner_set_refine)
  float nary_eps = 1e-4f;
  int nary_rounds = 8;
  // gradient refinement of the incumbent (fn_planner_set_grefine)
  int gr_iters = 8;
  float gr_eta0 = 0.05f, gr_h = 1e-3f;
  // per-launch events of a timed iteration (kev[0] before the first launch)
  cudaEvent_t kev[PL_MAX_KEV + 1] = {};
  const char* kname[PL_MAX_KEV] = {};
  int nk = 0;
  bool tracing = false;
  // the goal branch of a captured iteration (goal IK, goal queries' parent
  // search, goal edges) runs on a side stream, forked after the sampling
  // launch and joined before the attach
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool allow_fork = false;   // set by the iteration's enqueue when it is not traced
  bool forked = false;       // a fork is open (the iteration's enqueue joins it)
};

// record the end of the launch just issued (timed iterations only)
static void trace(fn_planner* pl, cudaStream_t st, const char* name) {
  if (!pl->tracing || pl->nk >= PL_MAX_KEV) return;
  pl->kname[pl->nk] = name;
  cudaEventRecord(pl->kev[++pl->nk], st);
}

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
static PlanEdgeKernel plan_probe_variant(int v) {
  switch (v) {
    case 0: return k_plan_probe<2>;
    case 1: return k_plan_probe<3>;
    default: return k_plan_probe<4>;
  }
}
static PlanEdgeKernel plan_mprobe_variant(int v) {
  switch (v) {
    case 0: return k_plan_mprobe<2>;
    case 1: return k_plan_mprobe<3>;
    default: return k_plan_mprobe<4>;
  }
}

typedef void (*PlanStageKernel)(PlanDev, ArmK, GridKP, int);
static PlanStageKernel plan_vstage_variant(int v) {
  switch (v) {
    case 0: return k_plan_vstage<2>;
    case 1: return k_plan_vstage<3>;
    default: return k_plan_vstage<4>;
  }
}
static PlanStageKernel plan_vseq_variant(int v) {
  switch (v) {
    case 0: return k_plan_vseq<2>;
    case 1: return k_plan_vseq<3>;
    default: return k_plan_vseq<4>;
  }
}

static int resident(PlanEdgeKernel k) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * PL_EDGE_WARPS, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * num_sms();
}

static int resident_stage(PlanStageKernel k) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * PL_EDGE_WARPS, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * num_sms();
}

static int plan_edge_blocks(fn_planner* pl, int v) {
  (void)pl;
  return std::min(resident(plan_probe_variant(v)),
                  std::min(resident_stage(plan_vstage_variant(v)),
                           resident_stage(plan_vseq_variant(v))));
}

// Launch with programmatic stream serialization (see pdl_begin): the
// kernel may be scheduled while the previous kernel on the stream drains.
template <class... KArgs, class... Args>
static void pl_launch_pdl(bool pdl, void (*k)(KArgs...), unsigned grid, unsigned block,
                          size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, args...);
}
template <class... KArgs, class... Args>
static void pl_launch(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem,
                      cudaStream_t st, Args... args) {
  pl_launch_pdl(true, k, grid, block, smem, st, args...);
}

template <int KM>
static int knn_blocks(fn_planner* pl) {
  (void)pl;
  static int blocks[64] = {0};   // per device: resident blocks of k_plan_knn<KM>
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (blocks[dev] == 0) {
    cudaFuncSetAttribute(k_plan_knn<KM>, cudaFuncAttributeMaxDynamicSharedMemorySize, kKnnSmem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plan_knn<KM>, 32 * PL_KNN_WARPS,
                                                      kKnnSmem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    blocks[dev] = per_sm * num_sms();
  }
  return blocks[dev];
}

// resident CTAs of the tiled free-query search (its persistent grid)
template <int KM>
static int knn_tile_blocks() {
  static int blocks[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (blocks[dev] == 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plan_knn_tile<KM>,
                                                      32 * PL_KNN_TW, kKnnTileSmem) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    blocks[dev] = per_sm * num_sms();
  }
  return blocks[dev];
}

// sampling and parents: candidates of every problem (unless given by the
// caller), then their nearest tree nodes (mark(2) between the two)
// the shared-memory request of the planner's tensor-memory kernels (the
// warp-per-edge body, the goal edges), set once per device
static bool plan_tm_ready() {
  static std::once_flag once[64];
  static bool ok[64];
  int dev = 0;
  cudaGetDevice(&dev);
  std::call_once(once[dev & 63], [&] {
    ok[dev & 63] =
        cudaFuncSetAttribute(k_plan_edges_tm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTmSmem) == cudaSuccess &&
        cudaFuncSetAttribute(k_plan_goal_edges, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTmSmem) == cudaSuccess;
  });
  return ok[dev & 63];
}

template <class Mark>
static void enqueue_front(fn_planner* pl, unsigned flags, cudaStream_t st, Mark&& mark) {
  PlanDev& D = pl->D;
  const int P = pl->cfg.P;
  const bool knn = pl->cfg.k > 1;
  // external candidates: only the parent-search preparation runs
  const long n = (flags & FN_PLAN_EXTERNAL) ? 0 : (long)P * D.BM;
  const int prep = knn ? 4 * num_sms() : 0;
  const int dens = (flags & FN_PLAN_DENSITY) ? 1 : 0;
  // launches on the side stream are plain: an early-launched (programmatic)
  // grid would hold its blocks' shared memory and warps on the SMs while it
  // waits, in the way of the free edges' launches on the other stream
  auto search = [&](int kind, cudaStream_t s) {
    if (!knn) return;
    const bool pdl = s != pl->side;
    // the goal list is short (the decoded goals): a small grid claims it
    const int gb = 2 * num_sms();
    if (kind == 0 && D.knn_tile) {   // large trees: the tiled search
      if (D.KM == 8)
        pl_launch_pdl(pdl, k_plan_knn_tile<8>, knn_tile_blocks<8>(), 32 * PL_KNN_TW, kKnnTileSmem,
                      s, D);
      else
        pl_launch_pdl(pdl, k_plan_knn_tile<16>, knn_tile_blocks<16>(), 32 * PL_KNN_TW,
                      kKnnTileSmem, s, D);
    } else if (D.KM == 8) {
      pl_launch_pdl(pdl, k_plan_knn<8>,
                    kind == 0 ? knn_blocks<8>(pl) : std::min(gb, knn_blocks<8>(pl)),
                    32 * PL_KNN_WARPS, kKnnSmem, s, D, kind);
    } else {
      pl_launch_pdl(pdl, k_plan_knn<16>,
                    kind == 0 ? knn_blocks<16>(pl) : std::min(gb, knn_blocks<16>(pl)),
                    32 * PL_KNN_WARPS, kKnnSmem, s, D, kind);
    }
    trace(pl, s, "k_plan_knn");
  };
  auto goals = [&](cudaStream_t s) {
    pl_launch_pdl(s != pl->side, k_plan_sample, (unsigned)((32 * n + 127) / 128), 128, 0, s, D,
                  pl->arm, n, 0, dens, 1);
    trace(pl, s, "k_plan_sample");
  };
  auto goal_edges = [&](cudaStream_t s) {   // after the goal queries' parent search
    if (!D.goal_split) return;
    pl_launch_pdl(s != pl->side, k_plan_goal_edges, num_sms(), 32 * TM_WARPS, kTmSmem, s, D,
                  pl->arm);
    trace(pl, s, "k_plan_goal_edges");
  };
  if (n + prep > 0) {
    const long warps = (n + 31) / 32 + prep;
    pl_launch(k_plan_sample, (unsigned)((32 * warps + 127) / 128), 128, 0, st, D, pl->arm, n,
              prep, dens, 0);
    trace(pl, st, "k_plan_prep");
  }
  if (n > 0 && knn && D.goal_split && !(flags & FN_PLAN_CHORD) && pl->allow_fork) {
    // two branches: the free queries' parent search (and, after this
    // function, the free edges) on the caller's stream; the goal chart's IK,
    // the goal queries' search and the goal edges on the side stream, joined
    // before the attach
    mark(2);
    cudaEventRecord(pl->ev_fork, st);
    cudaStreamWaitEvent(pl->side, pl->ev_fork, 0);
    search(0, st);
    goals(pl->side);
    search(1, pl->side);
    goal_edges(pl->side);
    cudaEventRecord(pl->ev_join, pl->side);
    pl->forked = true;
    return;
  }
  if (n > 0) goals(st);
  if (n > 0 && (flags & FN_PLAN_CHORD)) {
    pl_launch(k_plan_chord, P, PL_CHORD_THREADS, 0, st, D, pl->arm);
    trace(pl, st, "k_plan_chord");
  }
  mark(2);
  if (knn && D.goal_split && pl->allow_fork) {
    // chord states make the free candidates wait for the goal chart (and
    // caller-given candidates have none): the goal queries' search and the
    // goal edges still run beside the free queries' search and free edges
    cudaEventRecord(pl->ev_fork, st);
    cudaStreamWaitEvent(pl->side, pl->ev_fork, 0);
    search(0, st);
    search(1, pl->side);
    goal_edges(pl->side);
    cudaEventRecord(pl->ev_join, pl->side);
    pl->forked = true;
    return;
  }
  search(0, st);
  search(1, st);
  goal_edges(st);
}

// Packed verification stages before the sequential tail (PlanDev::vstages):
// each stage pair is two dependent launches, which pay off when thousands of
// edges fail their first duration.  Planners whose edge capacity is at least
// PL_VSTAGE_EDGES run two (a batch of many problems), smaller ones
// PL_VSTAGES_SMALL (the tail alone measured within 2 % at C2 and C5); the
// packed engine runs two (uncapped caller edges scan many durations).  At
// least one whenever goal edges are in the body (planners whose goal edges
// have their own kernel have none): they are verified at their fixed
// duration by the first stage and must not reach the tail.
#ifndef PL_VSTAGE_EDGES
#define PL_VSTAGE_EDGES 262144
#endif
#ifndef PL_VSTAGES_SMALL
#define PL_VSTAGES_SMALL 1   // stages of the smaller planners
#endif
static int vstages(const PlanDev& D) {
  return D.vstages >= 2 ? 2 : (D.goal_split ? PL_VSTAGES_SMALL : 1);
}

// the packed edge phase after the per-edge prep: item scan, probe, verify
// (over the edges of the view D; mark(i) records the phase boundaries when
// timing)
template <class Mark>
static void enqueue_edge_body(fn_planner* pl, const PlanDev& D, int v, int blocks, cudaStream_t st,
                              Mark&& mark, bool scan = true) {
  if (scan) {   // k_plan_eprep scans the block totals itself
    pl_launch(k_plan_escan, 1, PL_SCAN, 0, st, D);
    trace(pl, st, "k_plan_escan");
  }
  pl_launch(k_plan_expand, expand_blocks(), 32 * PL_EXP_WARPS, 0, st, D, pl->arm);
  trace(pl, st, "k_plan_expand");
  mark(4);
  pl_launch(plan_probe_variant(v), blocks, 32 * PL_EDGE_WARPS, 0, st, D, pl->arm, pl->grid);
  trace(pl, st, "k_plan_probe");
  pl_launch(plan_mprobe_variant(v), blocks, 32 * PL_EDGE_WARPS, 0, st, D, pl->arm, pl->grid);
  trace(pl, st, "k_plan_mprobe");
  mark(5);
  const int tb = 2 * num_sms();
  pl_launch(k_plan_vinit, tb, 256, 0, st, D);
  trace(pl, st, "k_plan_vinit");
  int list = 0;
  for (int stage = 0; stage < vstages(D); ++stage) {
    pl_launch(plan_vstage_variant(v), blocks, 32 * PL_EDGE_WARPS, 0, st, D, pl->arm, pl->grid, list);
    trace(pl, st, "k_plan_vstage");
    pl_launch(k_plan_vselect, tb, 128, 0, st, D, pl->arm, pl->grid, list);
    trace(pl, st, "k_plan_vselect");
    list ^= 1;
  }
  pl_launch(plan_vseq_variant(v), blocks, 32 * PL_EDGE_WARPS, 0, st, D, pl->arm, pl->grid, list);
  trace(pl, st, "k_plan_vseq");
}

// the planner's packed edge phase: prep of the iteration's edges, then the body
template <class Mark>
static void enqueue_edges(fn_planner* pl, int v, int blocks, cudaStream_t st, Mark&& mark) {
  PlanDev& D = pl->D;
  const int eb = (D.Emax + PL_SCAN - 1) / PL_SCAN;
  pl_launch(k_plan_eprep, eb, PL_SCAN, 0, st, D, pl->grid);
  trace(pl, st, "k_plan_eprep");
  // with the duration surrogate every free edge with an admissible duration
  // goes to the surrogate pass and the goal edges to k_plan_goal_edges: the
  // body would find no edge
  if (pl->sur_mlp && D.goal_split) {
    mark(4);
    mark(5);
    return;
  }
  if (v == kPairEdgeVariant && plan_tm_ready()) {   // the warp-per-edge body
    mark(4);
    pl_launch(k_plan_edges_tm, num_sms(), 32 * TM_WARPS, kTmSmem, st, D, pl->arm, pl->grid);
    trace(pl, st, "k_plan_edges_tm");
    mark(5);
    return;
  }
  enqueue_edge_body(pl, D, v, blocks, st, mark, false);
}

extern "C" fn_status fn_planner_destroy(fn_planner_t* pl) {
  if (!pl) return FN_EINVAL;
  for (cudaEvent_t e : pl->ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : pl->kev)
    if (e) cudaEventDestroy(e);
  if (pl->graph_exec) cudaGraphExecDestroy(pl->graph_exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  for (void* p : pl->allocs) cudaFree(p);
  if (pl->replay_done) {
    cudaEventSynchronize(pl->replay_done);
    cudaEventDestroy(pl->replay_done);
  }
  if (pl->h_prob) cudaFreeHost(pl->h_prob);
  if (pl->h_reset) cudaFreeHost(pl->h_reset);
  if (pl->h_out) cudaFreeHost(pl->h_out);
  if (pl->h_iter) cudaFreeHost(pl->h_iter);
  if (pl->reset_done) {
    cudaEventSynchronize(pl->reset_done);
    cudaEventDestroy(pl->reset_done);
  }
  if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
  if (pl->ev_join) cudaEventDestroy(pl->ev_join);
  if (pl->side) cudaStreamDestroy(pl->side);
  delete pl;
  return FN_OK;
}

static fn_sampler_cfg_t default_sampler_cfg() {
  fn_sampler_cfg_t c;
  c.w_u = 0.25f;
  c.C = 4;
  c.n_fit = 32;
  c.em_iters = 8;
  c.sd_floor = 0.02f;
  c.sd_init = 0.1f;
  c.w_chord = 0.5f;
  c.chord_sigma = 0.1f;
  return c;
}

extern "C" fn_status fn_planner_create(const fn_planner_cfg_t* cfg, const fn_arm_t* arm,
                                       fn_planner_t** out) {
  if (!cfg || !arm || !out) return FN_EINVAL;
  const fn_planner_cfg_t c = *cfg;
  if ((long)c.P * c.b_max * c.k > (1L << 28)) return FN_EINVAL;
  if ((long)c.P * c.n_cap > (1L << 30)) return FN_EINVAL;
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
  D.knn_tile = c.n_cap >= PL_KNN_TILE_NODES ? 1 : 0;
  D.att_wide = c.b_max >= PL_ATT_WIDE_B && c.P <= PL_ATT_WIDE_P ? 1 : 0;
  D.knn_slots = D.knn_tile ? (D.KM == 8 ? knn_tile_blocks<8>() : knn_tile_blocks<16>())
                           : (D.KM == 8 ? knn_blocks<8>(pl) : knn_blocks<16>(pl)) * PL_KNN_WARPS;
  D.vstages = (long)c.P * c.b_max * c.k >= PL_VSTAGE_EDGES ? 2 : 1;
  D.goal_split = 1;
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
  A_(D.e_k, P * BM * KP);
  A_(D.inc, P); A_(D.prob, P); A_(D.sched, 1); A_(D.out, P); A_(D.iter, 1);
  if (rc == FN_OK && cudaMemset(D.sched, 0, sizeof(Sched)) != cudaSuccess) rc = FN_ECUDA;
  A_(D.added, P); A_(D.status, P);
  A_(D.ptr, P * NC); A_(D.newidx, P * NC); A_(D.alive, P * NC);
  A_(D.tmp_st, P * NC * 16); A_(D.tmp_f, P * NC * 4); A_(D.tmp_par, P * NC);
  A_(D.tmp_z, P * NC * 9);
  A_(D.att_idx, P * BM); A_(D.att_blk, P * ((BM + PL_ATT_T - 1) / PL_ATT_T)); A_(D.att_tot, P);
  A_(D.att_key, P);
  A_(D.prune_blk, P * ((NC + PL_PRUNE_T - 1) / PL_PRUNE_T)); A_(D.prune_tot, P);
  A_(D.prune_deep, P);
  A_(D.samples, PL_NCOUNT);
  D.Emax = (int)(P * BM * KP);
  A_(D.e_ci, (size_t)D.Emax); A_(D.e_par, (size_t)D.Emax); A_(D.e_Tp, (size_t)D.Emax);
  A_(D.e_klo, (size_t)D.Emax);
  A_(D.e_j, (size_t)D.Emax); A_(D.e_cnt, (size_t)D.Emax);
  A_(D.blk_off, (size_t)(D.Emax + PL_SCAN - 1) / PL_SCAN + 1);
  A_(D.mask, (size_t)D.Emax * 8);
  D.Kmax = c.K;
  A_(D.owner, (size_t)D.Emax * c.K);
  A_(D.edyn, (size_t)D.Emax * 56);
  A_(D.dyn_list, (size_t)D.Emax);
  A_(D.cur_k, (size_t)D.Emax);
  A_(D.fail, (size_t)D.Emax);
  A_(D.pend, (size_t)D.Emax * 2);
  D.surv_cap = (int)std::min<long>((long)D.Emax * 16, 1L << 26);
  A_(D.surv, (size_t)D.surv_cap);
  D.NB = (NC + 63) / 64;
  A_(D.mir, (size_t)P * D.NB * 7 * 32);
  A_(D.packed, (size_t)P);
  D.sur = 0;
  D.sur_list = nullptr;
  A_(D.sur_n, 1);
  A_(D.knn_cnt, P * BM);
  A_(D.dens, P); A_(D.arch, P); A_(D.cz, P * BM * 9); A_(D.zn, P * NC * 9); A_(D.glist, P * BM); A_(D.gq, P * BM);
  D.scfg = default_sampler_cfg();
  if (rc == FN_OK) {
    std::vector<fn_density_t> th(P);
    for (auto& x : th) {
      memset(&x, 0, sizeof(x));
      x.w_u = D.scfg.w_u;
    }
    if (cudaMemcpy(D.dens, th.data(), sizeof(fn_density_t) * P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(D.arch, 0, sizeof(Archive) * P) != cudaSuccess ||
        cudaMemset(D.cz, 0xff, sizeof(float) * P * BM * 9) != cudaSuccess ||
        cudaMemset(D.zn, 0xff, sizeof(float) * P * NC * 9) != cudaSuccess)
      rc = FN_ECUDA;
  }
  if (rc == FN_OK && cudaMemset(D.knn_cnt, 0, sizeof(int32_t) * P * BM) != cudaSuccess) rc = FN_ECUDA;
  if (rc == FN_OK && cudaMemset(D.packed, 0, sizeof(int32_t) * P) != cudaSuccess) rc = FN_ECUDA;
#undef A_
  if (rc == FN_OK) {
    if (cudaHostAlloc(&pl->h_prob, P * sizeof(fn_problem_t), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostAlloc(&pl->h_reset, P * sizeof(fn_problem_t), cudaHostAllocDefault) !=
            cudaSuccess ||
        cudaHostAlloc(&pl->h_out, P * sizeof(fn_rendezvous_t), cudaHostAllocMapped) !=
            cudaSuccess ||
        cudaHostAlloc(&pl->h_iter, sizeof(int), cudaHostAllocMapped) != cudaSuccess)
      rc = FN_ENOMEM;
    else if (cudaHostGetDevicePointer((void**)&D.hprob, pl->h_prob, 0) != cudaSuccess ||
             cudaHostGetDevicePointer((void**)&D.hout, pl->h_out, 0) != cudaSuccess ||
             cudaHostGetDevicePointer((void**)&D.hiter, pl->h_iter, 0) != cudaSuccess)
      rc = FN_ECUDA;
  }
  if (rc == FN_OK && (cudaMemset(D.n_nodes, 0, P * sizeof(int)) != cudaSuccess ||
                      cudaMemset(D.samples, 0, PL_NCOUNT * sizeof(unsigned long long)) != cudaSuccess))
    rc = FN_ECUDA;
  if (rc != FN_OK) {
    fn_planner_destroy(pl);
    return rc;
  }
  for (int i = 0; i < 10; ++i)
    if (cudaEventCreate(&pl->ev[i]) != cudaSuccess) {
      fn_planner_destroy(pl);
      return FN_ECUDA;
    }
  for (int i = 0; i <= PL_MAX_KEV; ++i)
    if (cudaEventCreate(&pl->kev[i]) != cudaSuccess) {
      fn_planner_destroy(pl);
      return FN_ECUDA;
    }
  if (cudaStreamCreateWithFlags(&pl->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&pl->reset_done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      !plan_tm_ready()) {
    fn_planner_destroy(pl);
    return FN_ECUDA;
  }
  pl->edge_variant = tuned_variant(TUNE_PLAN_EDGES, (long)c.P * c.b_max * c.k, c.K, c.S);
  pl->edge_blocks = c.edge_blocks > 0 ? c.edge_blocks : plan_edge_blocks(pl, pl->edge_variant);
  *out = pl;
  return FN_OK;
}

static fn_status wait_staging(fn_planner* pl);

static bool problems_ok(const fn_planner* pl, const fn_problem_t* probs) {
  for (int p = 0; p < pl->cfg.P; ++p) {
    const fn_problem_t& q = probs[p];
    if (q.batch < 0 || q.batch > pl->cfg.b_max || q.n_goal < 0 || q.n_goal > q.batch ||
        q.n_obs < 0 || q.n_obs > FN_MAX_OBS || !(q.t_fall >= q.t_enter) || !(q.v_tip > 0.f))
      return false;
  }
  return true;
}

static fn_status stage_problems(fn_planner* pl, const fn_problem_t* probs, cudaStream_t st) {
  if (!problems_ok(pl, probs)) return FN_EINVAL;
  const fn_status rc = wait_staging(pl);
  if (rc != FN_OK) return rc;
  memcpy(pl->h_prob, probs, sizeof(fn_problem_t) * pl->cfg.P);
  if (cudaMemcpyAsync(pl->D.prob, pl->h_prob, sizeof(fn_problem_t) * pl->cfg.P,
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return FN_ECUDA;
  return FN_OK;
}

extern "C" fn_status fn_planner_reset(fn_planner_t* pl, const fn_problem_t* probs, void* stream) {
  if (!pl || !probs) return FN_EINVAL;
  if (!problems_ok(pl, probs)) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // the reset's own pinned copy of the problems (the replays' staging is
  // left alone); the previous reset's copy must have been read first
  if (pl->reset_pending) {
    if (cudaEventSynchronize(pl->reset_done) != cudaSuccess) return FN_ECUDA;
    pl->reset_pending = false;
  }
  memcpy(pl->h_reset, probs, sizeof(fn_problem_t) * pl->cfg.P);
  if (cudaMemcpyAsync(pl->D.prob, pl->h_reset, sizeof(fn_problem_t) * pl->cfg.P,
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return FN_ECUDA;
  k_plan_reset<<<(pl->cfg.P + 127) / 128, 128, 0, st>>>(pl->D);
  fn_status rc = launch_status();
  if (rc == FN_OK) {
    if (cudaEventRecord(pl->reset_done, st) != cudaSuccess) return FN_ECUDA;
    pl->reset_pending = true;
  }
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
  return launch_status();
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
  if (B > 0 && cudaMemsetAsync(D.cz + cb * 9, 0xff, sizeof(float) * 9 * B, st) != cudaSuccess)
    return FN_ECUDA;
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

static void enqueue_surrogate(fn_planner* pl, cudaStream_t st);

// enqueue one iteration (problems and iteration counter already staged)
static fn_status enqueue_iteration(fn_planner* pl, unsigned flags, cudaStream_t st,
                                   bool timed) {
  PlanDev& D = pl->D;
  const int P = pl->cfg.P;
  auto mark = [&](int i) {
    if (timed) cudaEventRecord(pl->ev[i], st);
  };
  mark(0);
  pl->tracing = timed;
  pl->allow_fork = !timed;
  pl->forked = false;
  pl->nk = 0;
  if (timed) cudaEventRecord(pl->kev[0], st);
  k_plan_schedule<<<1, 256, 0, st>>>(D);
  trace(pl, st, "k_plan_schedule");
  mark(1);
  enqueue_front(pl, flags, st, mark);
  mark(3);
  enqueue_edges(pl, pl->edge_variant, pl->edge_blocks, st, mark);
  if (pl->sur_mlp) enqueue_surrogate(pl, st);
  if (pl->forked) {            // the goal branch's edges precede the attach
    cudaStreamWaitEvent(st, pl->ev_join, 0);
    pl->forked = false;
  }
  pl->allow_fork = false;
  if (flags & FN_PLAN_NARY) {
    pl_launch(k_plan_refine, 4 * num_sms(), 32 * PL_REFINE_WARPS, 0, st, D, pl->arm, pl->grid,
              pl->nary_eps, pl->nary_rounds);
    trace(pl, st, "k_plan_refine");
  }
  mark(6);
  const bool late = flags & (FN_PLAN_DENSITY | FN_PLAN_REFIT | FN_PLAN_GREFINE | FN_PLAN_PRUNE);
  if (D.att_wide) {
    const unsigned ab = (unsigned)((long)P * ((D.BM + PL_ATT_T - 1) / PL_ATT_T));
    pl_launch(k_attach_scan, ab, PL_ATT_T, 0, st, D);
    trace(pl, st, "k_plan_attach");
    pl_launch(k_attach_write, ab, PL_ATT_T, 0, st, D);
    trace(pl, st, "k_plan_attach");
    pl_launch(k_attach_final, (unsigned)((P + 127) / 128), 128, 0, st, D, late ? 0 : 1);
    trace(pl, st, "k_plan_attach");
  } else {
    pl_launch(k_plan_attach, P, PL_ATTACH_THREADS, 0, st, D, late ? 0 : 1);
    trace(pl, st, "k_plan_attach");
  }
  if (flags & (FN_PLAN_DENSITY | FN_PLAN_REFIT)) {
    pl_launch(k_plan_density, P, PL_DENSITY_THREADS, 0, st, D, (flags & FN_PLAN_REFIT) ? 1 : 0);
    trace(pl, st, "k_plan_density");
  }
  if (flags & FN_PLAN_GREFINE) {
    pl_launch(k_plan_grefine, P, 32 * PL_GR_WARPS, 0, st, D, pl->arm, pl->gr_iters, pl->gr_eta0,
              pl->gr_h);
    trace(pl, st, "k_plan_grefine");
  }
  mark(7);
  if (flags & FN_PLAN_PRUNE) {
    const long nn = (long)P * D.NC;
    pl_launch(k_plan_reach, (unsigned)((nn + 127) / 128), 128, 0, st, D, pl->arm);
    trace(pl, st, "k_plan_reach");
    pl_launch(k_prune_path, (unsigned)((P + 127) / 128), 128, 0, st, D);
    trace(pl, st, "k_plan_prune");
    const unsigned pb = (unsigned)((long)P * ((D.NC + PL_PRUNE_T - 1) / PL_PRUNE_T));
    pl_launch(k_prune_walk, pb, PL_PRUNE_T, 0, st, D);
    trace(pl, st, "k_plan_prune");
    pl_launch(k_prune_scatter, pb, PL_PRUNE_T, 0, st, D);
    trace(pl, st, "k_plan_prune");
    pl_launch(k_prune_copy, pb, PL_PRUNE_T, 0, st, D);
    trace(pl, st, "k_plan_prune");
    pl_launch(k_plan_prune, P, PL_ATTACH_THREADS, 0, st, D, pl->arm);   // deep chains only
    trace(pl, st, "k_plan_prune");
  }
  mark(8);
  if (late) {
    pl_launch(k_plan_output, (P + 127) / 128, 128, 0, st, D);
    trace(pl, st, "k_plan_output");
  }
  pl->tracing = false;
  mark(9);
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
// events on its stream
extern "C" fn_status fn_planner_phase_ms(fn_planner_t* pl, float* ms) {
  if (!pl || !ms) return FN_EINVAL;
  if (!pl->timing) return FN_EINVAL;
  for (int i = 0; i < 9; ++i)
    if (cudaEventElapsedTime(&ms[i], pl->ev[i], pl->ev[i + 1]) != cudaSuccess) return FN_ECUDA;
  return FN_OK;
}

// durations (ms) of every kernel launch of the last fn_plan_iteration
extern "C" fn_status fn_planner_kernel_ms(fn_planner_t* pl, float* ms, const char** names, int cap,
                                          int* n) {
  if (!pl || !n || cap < 0 || (cap > 0 && (!ms || !names))) return FN_EINVAL;
  if (!pl->timing) return FN_EINVAL;
  *n = pl->nk;
  for (int i = 0; i < pl->nk && i < cap; ++i) {
    if (cudaEventElapsedTime(&ms[i], pl->kev[i], pl->kev[i + 1]) != cudaSuccess) return FN_ECUDA;
    names[i] = pl->kname[i];
  }
  return FN_OK;
}

extern "C" fn_status fn_planner_capture(fn_planner_t* pl, unsigned flags, void* stream) {
  if (!pl) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (!st) return FN_EINVAL;  // the legacy stream cannot be captured
  if (pl->graph_exec) { cudaGraphExecDestroy(pl->graph_exec); pl->graph_exec = nullptr; }
  if (pl->graph) { cudaGraphDestroy(pl->graph); pl->graph = nullptr; }
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return FN_ECUDA;
  // the staged problems and iteration counter are read by the graph's first
  // kernel from mapped host memory; the rendezvous goes back the same way
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

// the pinned staging is read by the copies of an asynchronous replay still
// in flight: wait for it before writing the staging again
static fn_status wait_staging(fn_planner* pl) {
  if (!pl->replay_pending) return FN_OK;
  if (cudaEventSynchronize(pl->replay_done) != cudaSuccess) return FN_ECUDA;
  pl->replay_pending = false;
  return FN_OK;
}

static bool replay_probs_ok(const fn_planner* pl, const fn_problem_t* probs) {
  for (int p = 0; p < pl->cfg.P; ++p) {
    const fn_problem_t& q = probs[p];
    if (q.batch < 0 || q.batch > pl->cfg.b_max || q.n_goal < 0 || q.n_goal > q.batch ||
        q.n_obs < 0 || q.n_obs > FN_MAX_OBS)
      return false;
  }
  return true;
}

extern "C" fn_status fn_plan_replay_async(fn_planner_t* pl, const fn_problem_t* probs, int iter,
                                          void* stream) {
  if (!pl || !probs || !pl->graph_exec) return FN_EINVAL;
  if (!replay_probs_ok(pl, probs)) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (!pl->replay_done &&
      cudaEventCreateWithFlags(&pl->replay_done, cudaEventDisableTiming) != cudaSuccess) {
    pl->replay_done = nullptr;
    return FN_ECUDA;
  }
  fn_status rc = wait_staging(pl);
  if (rc != FN_OK) return rc;
  memcpy(pl->h_prob, probs, sizeof(fn_problem_t) * pl->cfg.P);
  *pl->h_iter = iter;
  if (cudaGraphLaunch(pl->graph_exec, st) != cudaSuccess) return FN_ECUDA;
  if (cudaEventRecord(pl->replay_done, st) != cudaSuccess) return FN_ECUDA;
  pl->replay_pending = true;
  return FN_OK;
}

extern "C" fn_status fn_plan_result(fn_planner_t* pl, fn_rendezvous_t* out) {
  if (!pl || !out || !pl->replay_done) return FN_EINVAL;
  if (cudaEventSynchronize(pl->replay_done) != cudaSuccess) return FN_ECUDA;
  pl->replay_pending = false;
  memcpy(out, pl->h_out, sizeof(fn_rendezvous_t) * pl->cfg.P);
  return FN_OK;
}

extern "C" fn_status fn_plan_replay(fn_planner_t* pl, const fn_problem_t* probs, int iter,
                                    fn_rendezvous_t* out, void* stream) {
  if (!pl || !probs || !out || !pl->graph_exec) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (!replay_probs_ok(pl, probs)) return FN_EINVAL;
  fn_status rc = wait_staging(pl);
  if (rc != FN_OK) return rc;
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

extern "C" fn_status fn_planner_set_grid(fn_planner_t* pl, const float* T_grid, int K) {
  if (!pl || !T_grid || K != pl->cfg.K) return FN_EINVAL;
  for (int k = 0; k < K; ++k) {
    if (!(T_grid[k] > 0.f) || !std::isfinite(T_grid[k])) return FN_EINVAL;
    if (k > 0 && !(T_grid[k] > T_grid[k - 1])) return FN_EINVAL;
  }
  for (int k = 0; k < K; ++k) pl->grid.T[k] = T_grid[k];
  // a captured iteration holds the old grid in its launch parameters
  if (pl->graph_exec) { cudaGraphExecDestroy(pl->graph_exec); pl->graph_exec = nullptr; }
  if (pl->graph) { cudaGraphDestroy(pl->graph); pl->graph = nullptr; }
  return FN_OK;
}

extern "C" fn_status fn_planner_set_grefine(fn_planner_t* pl, int iters, float eta0, float h) {
  if (!pl || iters < 0 || iters > 64 || !(eta0 > 0.f) || !(eta0 <= 1.f) || !(h > 0.f) ||
      !(h <= 0.1f))
    return FN_EINVAL;
  pl->gr_iters = iters;
  pl->gr_eta0 = eta0;
  pl->gr_h = h;
  return FN_OK;
}

extern "C" fn_status fn_planner_set_refine(fn_planner_t* pl, float eps, int max_rounds) {
  if (!pl || !(eps > 0.f) || !std::isfinite(eps) || max_rounds < 0 || max_rounds > 16)
    return FN_EINVAL;
  pl->nary_eps = eps;
  pl->nary_rounds = max_rounds;
  return FN_OK;
}

extern "C" fn_status fn_planner_set_sampler(fn_planner_t* pl, const fn_sampler_cfg_t* cfg) {
  if (!pl || !cfg) return FN_EINVAL;
  const fn_sampler_cfg_t c = *cfg;
  if (!(c.w_u >= 0.f && c.w_u <= 1.f) || c.C < 1 || c.C > FN_DENSITY_MAX_C || c.n_fit < 1 ||
      c.n_fit > FN_ARCHIVE_MAX || c.em_iters < 1 || c.em_iters > 64 ||
      !(c.sd_floor >= 0.f && std::isfinite(c.sd_floor)) ||
      !(c.sd_init > 0.f && std::isfinite(c.sd_init)) || !(c.w_chord >= 0.f && c.w_chord <= 1.f) ||
      !(c.chord_sigma >= 0.f && std::isfinite(c.chord_sigma)))
    return FN_EINVAL;
  pl->D.scfg = c;
  return FN_OK;
}

extern "C" fn_status fn_planner_set_density(fn_planner_t* pl, int p, const fn_density_t* theta,
                                            void* stream) {
  if (!pl || !theta || p < 0 || p >= pl->cfg.P) return FN_EINVAL;
  const fn_density_t& t = *theta;
  if (t.C < 0 || t.C > FN_DENSITY_MAX_C || !(t.w_u >= 0.f && t.w_u <= 1.f)) return FN_EINVAL;
  double sum = 0.0;
  for (int m = 0; m < t.C; ++m) {
    if (!(t.pi[m] >= 0.f) || !std::isfinite(t.pi[m])) return FN_EINVAL;
    sum += t.pi[m];
    for (int k = 0; k < 9; ++k)
      if (!std::isfinite(t.mu[m][k]) || !(t.sd[m][k] > 0.f) || !std::isfinite(t.sd[m][k]))
        return FN_EINVAL;
  }
  if (t.C > 0 && std::fabs(sum - 1.0) > 1e-3) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(pl->D.dens + p, theta, sizeof(fn_density_t), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return FN_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? FN_OK : FN_ECUDA;
}

extern "C" fn_status fn_planner_get_density(fn_planner_t* pl, int p, fn_density_t* theta,
                                            float* archive_J, float* archive_z, int* archive_n) {
  if (!pl || p < 0 || p >= pl->cfg.P) return FN_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return FN_ECUDA;
  Archive ar;
  if (theta && cudaMemcpy(theta, pl->D.dens + p, sizeof(fn_density_t), cudaMemcpyDeviceToHost) !=
                   cudaSuccess)
    return FN_ECUDA;
  if (cudaMemcpy(&ar, pl->D.arch + p, sizeof(Archive), cudaMemcpyDeviceToHost) != cudaSuccess)
    return FN_ECUDA;
  if (archive_n) *archive_n = ar.n;
  if (archive_J) memcpy(archive_J, ar.J, sizeof(ar.J));
  if (archive_z) memcpy(archive_z, ar.z, sizeof(ar.z));
  return FN_OK;
}

extern "C" fn_status fn_planner_set_candidate_params(fn_planner_t* pl, int p, const float* z,
                                                     int n_goal, void* stream) {
  if (!pl || p < 0 || p >= pl->cfg.P || n_goal < 0 || n_goal > pl->cfg.b_max) return FN_EINVAL;
  if (n_goal == 0) return FN_OK;
  if (!z) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const long cb = (long)p * pl->cfg.b_max;
  if (cudaMemcpyAsync(pl->D.cz + cb * 9, z, sizeof(float) * 9 * n_goal, cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return FN_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? FN_OK : FN_ECUDA;
}

extern "C" fn_status fn_planner_get_candidate_params(fn_planner_t* pl, int p, float* z, int n) {
  if (!pl || p < 0 || p >= pl->cfg.P || n < 0 || n > pl->cfg.b_max || (n > 0 && !z))
    return FN_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return FN_ECUDA;
  const long cb = (long)p * pl->cfg.b_max;
  if (n > 0 && cudaMemcpy(z, pl->D.cz + cb * 9, sizeof(float) * 9 * n, cudaMemcpyDeviceToHost) !=
                   cudaSuccess)
    return FN_ECUDA;
  return FN_OK;
}

extern "C" fn_status fn_planner_incumbent_path(fn_planner_t* pl, int p, int max_edges,
                                               float* s0, float* s1, float* T, int32_t* nodes,
                                               int32_t* n_edges, void* stream) {
  if (!pl || p < 0 || p >= pl->cfg.P || max_edges < 0 || !n_edges) return FN_EINVAL;
  if (max_edges > 0 && (!s0 || !s1 || !T)) return FN_EINVAL;
  if ((s0 && !aligned16(s0)) || (s1 && !aligned16(s1))) return FN_EINVAL;
  k_plan_path<<<1, 32, 0, (cudaStream_t)stream>>>(pl->D, p, max_edges, s0, s1, T, nodes, n_edges);
  return launch_status();
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

extern "C" fn_status fn_planner_get_parents(fn_planner_t* pl, int p, int32_t* nn, int cap) {
  if (!pl || !nn || p < 0 || p >= pl->cfg.P || cap < 0) return FN_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return FN_ECUDA;
  const int KN = pl->D.KN;
  const long m = std::min(cap, pl->cfg.b_max);
  if (KN == 0 || m == 0) return FN_OK;
  return cudaMemcpy(nn, pl->D.nn + (long)p * pl->cfg.b_max * KN, sizeof(int32_t) * m * KN,
                    cudaMemcpyDeviceToHost) == cudaSuccess
             ? FN_OK
             : FN_ECUDA;
}

extern "C" fn_status fn_planner_get_node_params(fn_planner_t* pl, int p, float* z, int cap) {
  if (!pl || !z || p < 0 || p >= pl->cfg.P || cap < 0) return FN_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return FN_ECUDA;
  const long m = std::min(cap, pl->cfg.n_cap);
  if (m == 0) return FN_OK;
  return cudaMemcpy(z, pl->D.zn + (long)p * pl->cfg.n_cap * 9, sizeof(float) * 9 * m,
                    cudaMemcpyDeviceToHost) == cudaSuccess
             ? FN_OK
             : FN_ECUDA;
}

extern "C" fn_status fn_planner_get_edges(fn_planner_t* pl, int p, int32_t* k_star, float* T,
                                          float* rho_v, uint8_t* ok, int cap) {
  if (!pl || p < 0 || p >= pl->cfg.P || cap < 0) return FN_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return FN_ECUDA;
  const long KP = pl->D.KP;
  const long m = (long)std::min(cap, pl->cfg.b_max) * KP;
  const long e0 = (long)p * pl->cfg.b_max * KP;
  if (m == 0) return FN_OK;
  bool good = true;
  if (k_star) good &= cudaMemcpy(k_star, pl->D.e_k + e0, sizeof(int32_t) * m, cudaMemcpyDeviceToHost) == cudaSuccess;
  if (T) good &= cudaMemcpy(T, pl->D.e_T + e0, sizeof(float) * m, cudaMemcpyDeviceToHost) == cudaSuccess;
  if (rho_v) good &= cudaMemcpy(rho_v, pl->D.e_rv + e0, sizeof(float) * m, cudaMemcpyDeviceToHost) == cudaSuccess;
  if (ok) good &= cudaMemcpy(ok, pl->D.e_ok + e0, m, cudaMemcpyDeviceToHost) == cudaSuccess;
  return good ? FN_OK : FN_ECUDA;
}

// work counters of the edge kernels (torque evaluations since the last
// reset): count[0] probe, count[1] verify
extern "C" fn_status fn_planner_work_counts(fn_planner_t* pl, unsigned long long* count, int n,
                                            int reset) {
  if (!pl || !count || n < 0) return FN_EINVAL;
  unsigned long long c[PL_NCOUNT];
  if (cudaMemcpy(c, pl->D.samples, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
    return FN_ECUDA;
  for (int i = 0; i < n && i < PL_NCOUNT; ++i) count[i] = c[i];
  if (reset && cudaMemset(pl->D.samples, 0, sizeof(c)) != cudaSuccess) return FN_ECUDA;
  return FN_OK;
}

extern "C" fn_status fn_planner_sample_count(fn_planner_t* pl, unsigned long long* count,
                                             int reset) {
  if (!pl || !count) return FN_EINVAL;
  unsigned long long c[PL_NCOUNT];
  const fn_status rc = fn_planner_work_counts(pl, c, PL_NCOUNT, reset);
  if (rc != FN_OK) return rc;
  count[0] = c[0] + c[2];   // both probe stages
  count[1] = c[1];
  return FN_OK;
}

// Autotuner of the planner's edge kernel: runs the iteration's prefix
// (schedule, samplers unless FN_PLAN_EXTERNAL, parents) once, then times
// every register-budget variant of the persistent edge kernel on that edge
// batch (`reps` runs each, after one warm-up) and keeps the fastest for this
// planner and for planners created later with the same shape.  The tree is
// not modified.  chosen: host (may be NULL); variant_ms: host [3] (may be NULL).
extern "C" fn_status fn_planner_set_schedule(fn_planner_t* pl, int variant) {
  if (!pl || variant < 0 || variant >= kPlanEdgeVariants) return FN_EINVAL;
  pl->edge_variant = variant;
  pl->edge_blocks = pl->cfg.edge_blocks > 0 ? pl->cfg.edge_blocks : plan_edge_blocks(pl, variant);
  return FN_OK;
}

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
  k_plan_schedule<<<1, 256, 0, st>>>(D);
  enqueue_front(pl, flags, st, [](int) {});
  if ((rc = launch_status()) != FN_OK) return rc;
  float best_ms = INFINITY;
  int best = pl->edge_variant;
  for (int v = 0; v < kPlanEdgeVariants; ++v) {
    const int blocks = pl->cfg.edge_blocks > 0 ? pl->cfg.edge_blocks : plan_edge_blocks(pl, v);
    float tot = 0.f;
    for (int r = 0; r <= reps; ++r) {
      cudaEventRecord(pl->ev[0], st);
      enqueue_edges(pl, v, blocks, st, [](int) {});
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

// ---------------------------------------------------------------------------
// Packed edge engine (fn_edges_*): the planner's packed edge pipeline over
// edge arrays given by the caller.  A private planner (one problem, one
// parent slot) owns the buffers and the tuned schedule; a view of its
// device state points the rows at the caller's s0 / s1 and the results at
// the caller's outputs (edge e's result slot is e).
// ---------------------------------------------------------------------------
namespace fn {

// Per-edge prep of one pass: admissible count Kadm = #{k : T_k <= cap},
// probe-item range, mask reset, and the result of edges decided without
// dynamics (non-finite input: k = -2; empty range: k = -1).
//   mode 0: full scan [0, Kadm)
//   mode 1: window [lo, min(lo + W, Kadm)) around the prediction's centre c
//           (window_centre over the admissible range, the window clamped
//           into [0, Kadm)), scanned from klo = max(lo - 1, c -
//           FN_WINDOW_BELOW, 0); win[e] = (klo, whether "none" over [klo,
//           Kadm) is certified: the scan reaches the top admissible duration)
//   mode 2: full scan of the listed edges (list)
// n_list (device, may be NULL): the number of edges of the pass, at most E.
__global__ void __launch_bounds__(PL_SCAN) k_edges_prep(PlanDev D, GridKP Gr, int mode, int E,
                                                        const float* __restrict__ cap,
                                                        const float* __restrict__ Y, int W,
                                                        float logT0, float dlog,
                                                        const int32_t* __restrict__ list,
                                                        const int* __restrict__ n_list,
                                                        int2* __restrict__ win) {
  pdl_begin();
  __shared__ float sT[FN_MAX_GRID];
  __shared__ int sh[32];
  for (int i = threadIdx.x; i < D.K; i += blockDim.x) sT[i] = Gr.T[i];
  __syncthreads();
  const int n = n_list ? min(*n_list, E) : E;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    D.sched->n_edges = n;
    D.sched->n_free_edges = n;
  }
  const int e = blockIdx.x * PL_SCAN + threadIdx.x;
  int cnt = 0;
  if (e < n) {
    const int src = mode == 2 ? list[e] : e;
    const float* r0 = D.st + 16L * src;
    const float* r1 = D.cand + 16L * src;
    bool finite = true;
#pragma unroll
    for (int m = 0; m < 16; ++m)
      if ((m & 7) != 7) finite = finite && isfinite(r0[m]) && isfinite(r1[m]);
    const float c = cap ? cap[src] : INFINITY;
    int lo = 0, hi = D.K;   // Kadm = #{k : T_k <= c} on the ascending grid
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sT[mid] <= c) lo = mid + 1;
      else hi = mid;
    }
    const int Kadm = lo;
    int klo = 0, khi = Kadm;
    if (mode == 1) {
      // the window is clamped into the admissible range, so that a
      // prediction above the cap puts it at the top admissible duration
      const int top = max(Kadm, 1);
      const int ctr = window_centre(Y[2L * src], Y[2L * src + 1], logT0, dlog, top);
      const int wlo = min(max(ctr - W / 2, 0), max(top - W, 0));
      klo = max(max(wlo - 1, 0), ctr - FN_WINDOW_BELOW);
      khi = min(wlo + W, Kadm);
      win[src] = make_int2(klo, (klo < khi && khi == Kadm) ? 1 : 0);
    }
    cnt = finite ? max(khi - klo, 0) : 0;
    D.e_ci[e] = src;
    D.e_par[e] = src;
    D.e_Tp[e] = c;
    D.e_j[e] = 0;
    D.e_klo[e] = klo;
#pragma unroll
    for (int w = 0; w < 8; ++w) D.mask[8L * e + w] = 0u;
    if (cnt == 0) {
      D.e_ok[src] = 0;
      D.e_T[src] = finite ? INFINITY : NAN;
      D.e_rv[src] = NAN;
      D.e_k[src] = finite ? -1 : -2;
    }
  }
  list_dyn_edge(D, e, e < n && cnt > 0);
  int tot;
  const int ex = block_scan(cnt, sh, &tot);
  if (e < n) D.e_cnt[e] = ex;
  if (threadIdx.x == 0) D.blk_off[blockIdx.x] = tot;
}

// Window certificate (exact under monotone rho_tau, rho_P): the first
// feasible index k of the scanned range [klo, khi) is accepted if k = 0 or
// k > klo (T_{k-1} was shown infeasible); "none" is accepted if the scan
// reached the top admissible duration.  Any other edge joins the list for
// the exact scan.
__global__ void k_edges_cert(PlanDev D, int E, const int2* __restrict__ win,
                             int32_t* __restrict__ list, int* __restrict__ n_list,
                             uint8_t* __restrict__ path, const int* __restrict__ n_dev) {
  pdl_begin();
  if (n_dev) E = min(E, *n_dev);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    const int k = D.e_k[e];
    bool cert;
    if (k == -2) {
      cert = true;                                   // invalid input, decided
    } else if (k >= 0) {
      cert = k > win[e].x || k == 0;
    } else {
      cert = win[e].y != 0;
    }
    if (path) path[e] = cert ? 0 : 1;
    if (!cert) list[warp_append(n_list, D.samples ? D.samples + 6 : nullptr)] = e;
  }
}

// ---- the planner's surrogate pass (free edges routed by k_plan_eprep)

// rows, caps and result slots of the routed edges, compacted (the pass's
// prep reuses the per-edge arrays, so the slots are recorded here)
__global__ void k_sur_gather(PlanDev D, float* __restrict__ s0, float* __restrict__ s1,
                             float* __restrict__ cap, int32_t* __restrict__ slot) {
  pdl_begin();
  const long n = (long)min(*D.sur_n, D.Emax) * 16;
  for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (long)gridDim.x * blockDim.x) {
    const int i = (int)(x >> 4), m = (int)(x & 15);
    const int e = D.sur_list[i];
    const int p = D.e_ci[e] / D.BM;
    s0[x] = D.st[((long)p * D.NC + D.e_par[e]) * 16 + m];
    s1[x] = D.cand[(long)D.e_ci[e] * 16 + m];
    if (m == 0) {
      long ei;
      bool goal;
      edge_slot(D, e, ei, goal);
      cap[i] = D.e_Tp[e];
      slot[i] = (int32_t)ei;
    }
  }
}

// results of the surrogate pass into the edges' slots (a lane per edge), with
// the clearance check of the edge's own problem for accepted durations
__global__ void __launch_bounds__(128) k_sur_scatter(PlanDev D, ArmK A, const int32_t* __restrict__ gk,
                                                     const float* __restrict__ gT,
                                                     const float* __restrict__ grv,
                                                     const uint8_t* __restrict__ gok,
                                                     const float* __restrict__ s0,
                                                     const float* __restrict__ s1,
                                                     const int32_t* __restrict__ slot) {
  pdl_begin();
  __shared__ float sEs[4][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = min(*D.sur_n, D.Emax);
  if (D.samples && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(D.samples + 5, (unsigned long long)n);
  // a warp takes 32 edges, a lane each; the accepted edges of problems with
  // obstacles then get the warp-wide clearance check one at a time
  for (int i0 = (blockIdx.x * 4 + w) * 32; i0 < n; i0 += gridDim.x * 4 * 32) {
    const int i = i0 + lane;
    long ei = 0;
    bool ok = false;
    float T = 0.f;
    bool clear = false;
    if (i < n) {
      ei = slot[i];
      ok = gok[i] != 0;
      T = gT[i];
      clear = ok && D.prob[ei / ((long)D.KP * D.BM)].n_obs > 0;
    }
    for (unsigned m = __ballot_sync(0xffffffffu, clear); m; m &= m - 1u) {
      const int l = __ffs(m) - 1;
      const int il = i0 + l;
      const long el = __shfl_sync(0xffffffffu, ei, l);
      const float Tl = __shfl_sync(0xffffffffu, T, l);
      const fn_problem_t& P = D.prob[el / ((long)D.KP * D.BM)];
      stage_rows(s0 + 16L * il, s1 + 16L * il, sEs[w]);
      const bool okl = warp_clearance(D, A, P, sEs[w], Tl) >= D.margin;
      if (lane == l) ok = okl;
    }
    if (i < n) {
      D.e_ok[ei] = ok ? 1 : 0;
      D.e_T[ei] = T;
      D.e_rv[ei] = grv[i];
      D.e_k[ei] = gk[i];
    }
  }
}

}  // namespace fn

using namespace fn;

struct fn_edges {
  fn_planner* pl = nullptr;
  int maxE = 0;
  int2* win = nullptr;
  int32_t* list = nullptr;
  int* n_list = nullptr;
  float logT0 = 0.f, dlog = 0.f;
  // N-ary refinement of the free edges (fn_planner_set_refine)
  float nary_eps = 1e-4f;
  int nary_rounds = 8;
};

extern "C" fn_status fn_edges_destroy(fn_edges_t* eg) {
  if (!eg) return FN_EINVAL;
  if (eg->pl) fn_planner_destroy(eg->pl);
  if (eg->win) cudaFree(eg->win);
  if (eg->list) cudaFree(eg->list);
  if (eg->n_list) cudaFree(eg->n_list);
  delete eg;
  return FN_OK;
}

extern "C" fn_status fn_edges_create(const fn_arm_t* arm, const float* T_grid, int K, int S,
                                     int max_E, fn_edges_t** out) {
  if (!arm || !T_grid || !out || K < 2 || K > FN_MAX_GRID || S < 2 || S > FN_MAX_S || max_E < 1 ||
      max_E > (1 << 16))
    return FN_EINVAL;
  for (int k = 0; k < K; ++k) {
    if (!(T_grid[k] > 0.f) || !std::isfinite(T_grid[k])) return FN_EINVAL;
    if (k > 0 && !(T_grid[k] > T_grid[k - 1])) return FN_EINVAL;
  }
  fn_planner_cfg_t c = {};
  c.P = 1; c.n_cap = 2; c.b_max = max_E; c.k = 1; c.K = K;
  c.T_lo = T_grid[0]; c.T_hi = T_grid[K - 1]; c.S = S; c.S_clear = 2; c.reach_grid = 2;
  c.w_vel = 0.1f; c.vel_frac = 0.5f; c.clear_margin = 0.f; c.edge_blocks = 0;
  fn_edges* eg = new fn_edges();
  eg->maxE = max_E;
  fn_status rc = fn_planner_create(&c, arm, &eg->pl);
  if (rc != FN_OK) {
    delete eg;
    return rc;
  }
  for (int k = 0; k < K; ++k) eg->pl->grid.T[k] = T_grid[k];
  eg->pl->D.vstages = 2;
  eg->logT0 = std::log(T_grid[0]);
  eg->dlog = (std::log(T_grid[K - 1]) - eg->logT0) / (float)(K - 1);
  fn_problem_t prob = {};   // no obstacles: the clearance check is off
  prob.t_fall = 1.f;
  prob.v_tip = 1.f;
  if ((rc = fn_planner_reset(eg->pl, &prob, nullptr)) != FN_OK ||
      cudaMalloc(&eg->win, sizeof(int2) * max_E) != cudaSuccess ||
      cudaMalloc(&eg->list, sizeof(int32_t) * max_E) != cudaSuccess ||
      cudaMalloc(&eg->n_list, sizeof(int)) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    fn_edges_destroy(eg);
    return rc != FN_OK ? rc : FN_ENOMEM;
  }
  *out = eg;
  return FN_OK;
}

// the planner's device state viewed over a chunk of the caller's edges
static PlanDev edges_view(fn_edges* eg, const float* s0, const float* s1, int32_t* k_star,
                          float* T_star, float* rho_v, uint8_t* ok) {
  PlanDev D = eg->pl->D;
  D.st = const_cast<float*>(s0);
  D.cand = const_cast<float*>(s1);
  D.NC = eg->maxE;
  D.BM = eg->maxE;
  D.KP = 1;
  D.e_k = k_star;
  D.e_T = T_star;
  D.e_rv = rho_v;
  D.e_ok = ok;
  return D;
}

static fn_status edges_check(fn_edges* eg, const float* s0, const float* s1, int E,
                             const int32_t* k_star, const float* T_star, const float* rho_v,
                             const uint8_t* ok) {
  if (!eg || E < 0) return FN_EINVAL;
  if (E > 0 && (!s0 || !s1 || !k_star || !T_star || !rho_v || !ok)) return FN_EINVAL;
  if (E > 0 && (!aligned16(s0) || !aligned16(s1))) return FN_EINVAL;
  return FN_OK;
}

extern "C" fn_status fn_edges_time(fn_edges_t* eg, const float* s0, const float* s1, int E,
                                   const float* T_cap, int32_t* k_star, float* T_star, float* rho_v,
                                   uint8_t* ok, void* stream) {
  fn_status rc = edges_check(eg, s0, s1, E, k_star, T_star, rho_v, ok);
  if (rc != FN_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  fn_planner* pl = eg->pl;
  for (int e0 = 0; e0 < E; e0 += eg->maxE) {
    const int n = std::min(eg->maxE, E - e0);
    const PlanDev D = edges_view(eg, s0 + 16L * e0, s1 + 16L * e0, k_star + e0, T_star + e0,
                                 rho_v + e0, ok + e0);
    pl_launch(k_edges_prep, (n + PL_SCAN - 1) / PL_SCAN, PL_SCAN, 0, st, D, pl->grid, 0, n,
              T_cap ? T_cap + e0 : (const float*)nullptr, (const float*)nullptr, 0, 0.f, 0.f,
              (const int32_t*)nullptr, (const int*)nullptr, (int2*)nullptr);
    enqueue_edge_body(pl, D, pl->edge_variant, pl->edge_blocks, st, [](int) {});
  }
  return launch_status();
}

extern "C" fn_status fn_edges_time_window(fn_edges_t* eg, const float* s0, const float* s1, int E,
                                          const float* Y, int W, int32_t* k_star, float* T_star,
                                          float* rho_v, uint8_t* ok, uint8_t* path, void* stream) {
  fn_status rc = edges_check(eg, s0, s1, E, k_star, T_star, rho_v, ok);
  if (rc != FN_OK) return rc;
  if (E > 0 && !Y) return FN_EINVAL;
  if (W < 1) return FN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  fn_planner* pl = eg->pl;
  W = std::min(W, pl->D.K);
  for (int e0 = 0; e0 < E; e0 += eg->maxE) {
    const int n = std::min(eg->maxE, E - e0);
    const PlanDev D = edges_view(eg, s0 + 16L * e0, s1 + 16L * e0, k_star + e0, T_star + e0,
                                 rho_v + e0, ok + e0);
    const unsigned pb = (unsigned)((n + PL_SCAN - 1) / PL_SCAN);
    // pass 1: the predicted windows (and their certificate index)
    pl_launch(k_edges_prep, pb, PL_SCAN, 0, st, D, pl->grid, 1, n, (const float*)nullptr, Y + 2L * e0,
              W, eg->logT0, eg->dlog, (const int32_t*)nullptr, (const int*)nullptr, eg->win);
    enqueue_edge_body(pl, D, pl->edge_variant, pl->edge_blocks, st, [](int) {});
    // certificate; uncertified edges -> exact scan of their full range
    if (cudaMemsetAsync(eg->n_list, 0, sizeof(int), st) != cudaSuccess) return FN_ECUDA;
    k_edges_cert<<<2 * num_sms(), 256, 0, st>>>(D, n, eg->win, eg->list, eg->n_list,
                                                 path ? path + e0 : nullptr, nullptr);
    k_edges_prep<<<pb, PL_SCAN, 0, st>>>(D, pl->grid, 2, n, nullptr, nullptr, 0, 0.f, 0.f, eg->list,
                                          eg->n_list, nullptr);
    enqueue_edge_body(pl, D, pl->edge_variant, pl->edge_blocks, st, [](int) {});
  }
  return launch_status();
}

extern "C" fn_status fn_edges_work_counts(fn_edges_t* eg, unsigned long long* count, int n,
                                          int reset) {
  if (!eg) return FN_EINVAL;
  return fn_planner_work_counts(eg->pl, count, n, reset);
}

// ---------------------------------------------------------------------------
// Duration surrogate inside the planner iteration: the free edges routed by
// k_plan_eprep go through the packed window pass (predicted windows, their
// certificate, an exact rescan of the uncertified ones), on a view of the
// planner's buffers with its own schedule; their results land in the edges'
// slots before attach.
// ---------------------------------------------------------------------------
static void enqueue_surrogate(fn_planner* pl, cudaStream_t st) {
  PlanDev& D = pl->D;
  const int E = D.Emax;
  pl_launch(k_sur_gather, 4 * num_sms(), 256, 0, st, D, pl->g_s0, pl->g_s1, pl->g_cap,
            pl->g_slot);
  trace(pl, st, "k_sur_gather");
  mlp_forward_rows(pl->sur_mlp, pl->arm, pl->g_s0, pl->g_s1, E, D.sur_n, pl->g_Y, st);
  trace(pl, st, "k_mlp_tc");
  PlanDev V = D;                       // the pass's view
  V.sched = pl->sched2;
  V.st = pl->g_s0;
  V.cand = pl->g_s1;
  V.NC = E;
  V.BM = E;
  V.KP = 1;
  V.prob = pl->no_obs;                 // clearance: checked per problem in the scatter
  V.e_k = pl->g_k;
  V.e_T = pl->g_T;
  V.e_rv = pl->g_rv;
  V.e_ok = pl->g_ok;
  const unsigned pb = (unsigned)((E + PL_SCAN - 1) / PL_SCAN);
  const int v = pl->edge_variant, blocks = pl->edge_blocks;
  k_edges_prep<<<pb, PL_SCAN, 0, st>>>(V, pl->grid, 1, E, pl->g_cap, pl->g_Y, pl->sur_W, pl->logT0,
                                        pl->dlog, nullptr, D.sur_n, pl->g_win);
  trace(pl, st, "k_edges_prep");
  enqueue_edge_body(pl, V, v, blocks, st, [](int) {});
  cudaMemsetAsync(pl->g_fbn, 0, sizeof(int), st);
  k_edges_cert<<<2 * num_sms(), 256, 0, st>>>(V, E, pl->g_win, pl->g_fb, pl->g_fbn,
                                               pl->g_path, D.sur_n);
  trace(pl, st, "k_edges_cert");
  k_edges_prep<<<pb, PL_SCAN, 0, st>>>(V, pl->grid, 2, E, pl->g_cap, nullptr, 0, 0.f, 0.f, pl->g_fb,
                                        pl->g_fbn, nullptr);
  trace(pl, st, "k_edges_prep");
  enqueue_edge_body(pl, V, v, blocks, st, [](int) {});
  pl_launch(k_sur_scatter, 4 * num_sms(), 128, 0, st, D, pl->arm, pl->g_k, pl->g_T, pl->g_rv,
            pl->g_ok, pl->g_s0, pl->g_s1, pl->g_slot);
  trace(pl, st, "k_sur_scatter");
}

extern "C" fn_status fn_planner_set_surrogate(fn_planner_t* pl, fn_mlp_t* mlp, int W) {
  if (!pl || (mlp && (W < 1 || W > pl->D.K))) return FN_EINVAL;
  if (!mlp) {
    pl->sur_mlp = nullptr;
    pl->D.sur = 0;
    return FN_OK;
  }
  const size_t E = (size_t)pl->D.Emax;
  if (!pl->sched2) {
    fn_status rc = FN_OK;
#define B_(ptr, n) if (rc == FN_OK) rc = pl_alloc_n(pl, &(ptr), (n))
    B_(pl->sched2, 1); B_(pl->no_obs, 1);
    B_(pl->g_s0, E * 16); B_(pl->g_s1, E * 16); B_(pl->g_cap, E); B_(pl->g_Y, E * 2);
    B_(pl->g_k, E); B_(pl->g_T, E); B_(pl->g_rv, E); B_(pl->g_ok, E); B_(pl->g_path, E);
    B_(pl->g_win, E); B_(pl->g_fb, E); B_(pl->g_fbn, 1); B_(pl->D.sur_list, E);
    B_(pl->g_slot, E);
#undef B_
    if (rc != FN_OK) return rc;
    fn_problem_t z = {};
    z.t_fall = 1.f;
    z.v_tip = 1.f;
    if (cudaMemcpy(pl->no_obs, &z, sizeof(z), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(pl->sched2, 0, sizeof(Sched)) != cudaSuccess)
      return FN_ECUDA;
  }
  pl->logT0 = std::log(pl->grid.T[0]);
  pl->dlog = (std::log(pl->grid.T[pl->D.K - 1]) - pl->logT0) / (float)(pl->D.K - 1);
  pl->sur_mlp = reinterpret_cast<fn_mlp*>(mlp);
  pl->sur_W = W;
  pl->D.sur = 1;
  return FN_OK;
}
