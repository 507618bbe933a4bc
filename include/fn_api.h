/*
 * fn_api.h -- C ABI of the GB300 edge-timing planner library
 * (libfruitninja.so), after "Becoming a Fruit Ninja: Real-Time Probabilistic
 * Kinodynamic Planning for Manipulator Projectile Interception"
 * (arxiv 2609.22608).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers documented as "device" must point to CUDA device memory of the
 *    current device; "host" pointers are ordinary CPU memory.  The caller owns
 *    every buffer it passes; the library never frees caller memory.  Only the
 *    *_create functions allocate, and *_destroy frees what they allocated.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream unless stated.
 *  - The return value covers argument validation (FN_EINVAL, nothing is
 *    launched) and launch errors (FN_ECUDA).  Faults inside a kernel surface
 *    at the caller's next synchronising CUDA call.  No C++ exception crosses
 *    this boundary.
 *  - Per-edge numerical problems are reported per edge (k_star = -2), not as
 *    call failures.
 *  - States are packed rows of 16 floats: q[7], pad, qdot[7], pad (64 bytes,
 *    16-byte aligned rows).
 *  - Every routine computes in FP32.
 */
#ifndef FN_API_H
#define FN_API_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FN_DOF 7
#define FN_STATE_STRIDE 16
#define FN_MAX_GRID 256 /* largest duration grid K */
#define FN_MAX_S 256    /* largest number of collocation points S */
#define FN_MAX_KNN 16   /* largest k of the nearest-parent search */

typedef enum {
  FN_OK = 0,
  FN_EINVAL = -1,    /* invalid argument; nothing was launched */
  FN_ECUDA = -2,     /* a CUDA call or launch failed */
  FN_ENOMEM = -3,    /* allocation failed (only *_create allocate) */
  FN_ETIMEOUT = -4,  /* a bounded device-side wait gave up */
  FN_EDEADLINE = -5  /* a host-side deadline expired */
} fn_status;

/* Human-readable name of a status code (static storage). */
const char* fn_status_str(int status);
/* Library version string (static storage). */
const char* fn_version(void);

/*
 * Robot model.  Eq. (torque) of Sec. IV-C: rigid-body inverse dynamics by
 * recursive Newton-Euler (modified DH, Craig: T_{j-1,j} = Rx(alpha_j)
 * Tx(a_j) Rz(theta0_j + q_j) Tz(d_j)), plus reflected rotor inertia
 * I_m,j qdd_j (`armature`) and the sigmoid friction of Eq. (friction)
 * with (psi1, psi2, psi3) per joint.  Link inertias are diagonal about the
 * link's centre of mass, in the link frame.  Limits of Def. 1: |tau_j| <=
 * tau_max_j, |sum_j tau_j qd_j| <= w_max, |qd_j| <= qdbar_j(q_j) with the
 * taper qdbar_j(q) = min(qd_max_j, sqrt(2 qd_taper_a_j max(0, min(q - q_lo_j,
 * q_hi_j - q)))).  The end-effector frame is frame 7 moved `flange_d` along
 * its z axis; the blade edge (Sec. IV-A, 30 cm) starts at `blade_base` and
 * runs `blade_len` along `blade_axis`, cutting towards `blade_normal` (all in
 * the end-effector frame).  `link_radius` are the capsule radii used by the
 * clearance check.  Passed by host pointer to each call; `dof` must be 7.
 */
typedef struct {
  int dof;
  float dh_a[7], dh_alpha[7], dh_d[7], dh_theta0[7];
  float mass[7], com[7][3], inertia[7][3];
  float armature[7];
  float fric[7][3];
  float q_lo[7], q_hi[7], qd_max[7], qd_taper_a[7];
  float tau_max[7], w_max;
  float gravity[3];
  float flange_d;
  float blade_base[3], blade_axis[3], blade_normal[3], blade_len;
  float link_radius[7];
} fn_arm_t;

/* Edge-timing modes of fn_time_edges. */
#define FN_MODE_FULL 0  /* first feasible index over the whole grid        */
#define FN_MODE_FIXED 1 /* one given duration per edge (goal candidates)   */

/*
 * fn_time_edges -- minimum feasible duration of cubic edges (Sec. IV-D).
 *
 * Each edge is the cubic of Def. "Cubic edge" / Eq. (cubic) from state s0[e]
 * to state s1[e].  For a duration T the check of Def. "Feasibility Check" /
 * Eq. (rho) evaluates Eq. (torque) at the S equally spaced times
 * t_s = s T/(S-1), s = 0..S-1 (both ends included) and forms
 *   rho_tau = max_{j,s} |tau_j(t_s)| / tau_max_j,
 *   rho_P   = max_s |sum_j tau_j(t_s) qd_j(t_s)| / w_max,
 *   rho_v   = max_j over the exact extremum of the quadratic velocity
 *             (t in {0, T, stationary point}) of |qd_j(t)| / qdbar_j(q_j(t)).
 *
 * FN_MODE_FULL: Def. "Minimum feasible time" on the ascending duration grid
 *   T_grid[0..K-1]: k_star[e] = the FIRST k with rho_tau(T_k) <= 1 and
 *   rho_P(T_k) <= 1 (every lower index is shown infeasible; no monotonicity
 *   is assumed), restricted to T_k <= T_cap[e] when T_cap is non-NULL (the
 *   incumbent bound of Algorithm 1).  rho_v is then checked once at
 *   T_{k*} (Sec. IV-D): ok[e] = (k* >= 0) && rho_v <= 1.
 * FN_MODE_FIXED: Algorithm 1's goal-candidate check: the single duration
 *   T_fixed[e] with all three ratios; k_star[e] = 0 if rho_tau, rho_P <= 1,
 *   else -1; ok[e] = (k_star == 0) && rho_v <= 1.  T_grid/K are ignored.
 *
 * Arguments
 *   arm        host, robot model (dof == 7).
 *   s0, s1     device [E][16] f32, start / end states.
 *   E          number of edges (0 is allowed: nothing is launched).
 *   T_grid     host [K] f32, strictly ascending, positive (FULL mode).
 *   K          1..FN_MAX_GRID (FULL mode).
 *   S          2..FN_MAX_S collocation points.
 *   mode       FN_MODE_FULL or FN_MODE_FIXED.
 *   T_fixed    device [E] f32 (FIXED mode; ignored otherwise).
 *   T_cap      device [E] f32 or NULL (FULL mode cap; ignored otherwise).
 * Outputs (device, [E] unless noted)
 *   k_star     i32: grid index (FULL) / 0 (FIXED) when rho_tau, rho_P <= 1;
 *              -1 if no admissible duration passes; -2 if the edge is
 *              invalid (a non-finite state, or T_fixed not finite and > 0).
 *   T_star     f32: T_grid[k*] (FULL), T_fixed[e] (FIXED, also when -1);
 *              +inf when FULL finds none; NaN when invalid.
 *   rho3       [E][3] f32 (rho_tau, rho_P, rho_v) at T_star; NaN when
 *              k_star is -1 in FULL mode or -2.
 *   ok         u8: 1 iff the edge is feasible at T_star including rho_v.
 * Errors: FN_EINVAL for dof != 7, E < 0, S out of range, K out of range or a
 * non-ascending / non-positive grid in FULL mode, a NULL required pointer,
 * unknown mode.
 */
fn_status fn_time_edges(const fn_arm_t* arm, const float* s0, const float* s1, int E,
                        const float* T_grid, int K, int S, int mode, const float* T_fixed,
                        const float* T_cap, int32_t* k_star, float* T_star, float* rho3,
                        uint8_t* ok, void* stream);

/*
 * fn_time_edges_counted -- fn_time_edges plus a work counter: when
 * `sample_count` (device, one u64) is non-NULL, the number of torque
 * evaluations (edge, duration, sample) the kernels performed is ADDED to it
 * (the caller zeroes it).  Used to state the algorithmic work of a launch.
 */
fn_status fn_time_edges_counted(const fn_arm_t* arm, const float* s0, const float* s1, int E,
                                const float* T_grid, int K, int S, int mode,
                                const float* T_fixed, const float* T_cap, int32_t* k_star,
                                float* T_star, float* rho3, uint8_t* ok,
                                unsigned long long* sample_count, void* stream);

/*
 * fn_rnea_dump -- torques of Eq. (torque) along each edge (diagnostic hook
 * for torque parity).  tau[e][s][j] = tau_j(t_s) of the cubic from s0[e] to
 * s1[e] with duration T[e], t_s = s T[e]/(S-1).
 *   arm host; s0, s1 device [E][16]; T device [E] (finite, > 0);
 *   tau device [E][S][7] f32.  E >= 0, 2 <= S <= FN_MAX_S.
 */
fn_status fn_rnea_dump(const fn_arm_t* arm, const float* s0, const float* s1, const float* T,
                       int E, int S, float* tau, void* stream);

/*
 * fn_knn_tree -- Parents of Algorithm 1 (Sec. IV-E): brute-force parallel
 * scan for the k nearest tree nodes of each query under the velocity-weighted
 * squared joint distance
 *   d2(a, b) = sum_j (q_a,j - q_b,j)^2 + w_vel * sum_j (qd_a,j - qd_b,j)^2.
 * Candidates are nodes [first, N) (first = 1 excludes the root, which the
 * planner always adds as parent 0).  Results are sorted ascending by
 * (d2, node index); slots beyond the number of candidates get idx -1 and
 * d2 = +inf.
 *   tree       device [N][16] f32 node states.
 *   N, first   0 <= first <= N.
 *   queries    device [B][16] f32.
 *   B          >= 0.
 *   k          1..FN_MAX_KNN.
 *   w_vel      >= 0.
 *   idx        device [B][k] i32 out;  d2  device [B][k] f32 out.
 *   workspace  device scratch of at least fn_knn_workspace_bytes(B, N, k)
 *              bytes, 256-byte aligned, or NULL (then a single-pass kernel
 *              with less parallelism is used).  Its contents on entry do
 *              not matter; concurrent calls must not share one workspace.
 */
size_t fn_knn_workspace_bytes(int B, int N, int k);
fn_status fn_knn_tree(const float* tree, int N, int first, const float* queries, int B, int k,
                      float w_vel, int32_t* idx, float* d2, void* workspace,
                      size_t workspace_bytes, void* stream);

/*
 * fn_make_edges -- the (candidate, parent) edges of Algorithm 1's inner loop.
 * Each candidate b has the parent set {root} + its k_nn nearest tree nodes
 * (Sec. IV-E "Parents"): edge e = b (k_nn + 1) + j joins parent p (p = 0 for
 * j = 0, else nn_idx[b][j-1]) to the candidate.  The first n_goal candidates
 * are goal candidates whose edge duration is fixed at T_req[b] - t(p)
 * (Algorithm 1, goal branch); the others are free candidates whose duration
 * scan is capped at t_best - t(p) (Algorithm 1, free branch).  Differences
 * are rounded in FP32.  A parent index of -1 yields an invalid edge (NaN s0).
 *   tree    device [N][16] node states;  t_node device [N] time-to-come.
 *   cand    device [B][16];  nn_idx device [B][k_nn];  T_req device [n_goal].
 *   s0, s1  device [B (k_nn+1)][16] out;  T_param device [B (k_nn+1)] out
 *           (fixed duration for goal edges, cap for free edges);
 *   parent  device [B (k_nn+1)] out or NULL.
 */
fn_status fn_make_edges(const float* tree, const float* t_node, const float* cand, int B,
                        int n_goal, const int32_t* nn_idx, int k_nn, const float* T_req,
                        float t_best, float* s0, float* s1, float* T_param, int32_t* parent,
                        void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FN_API_H */
