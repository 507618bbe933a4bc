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
 * Schedule: unless fn_autotune_time_edges chose otherwise for the shape, one
 * warp per edge with two samples per lane (paired FP32 arithmetic) and the
 * torque recursion's per-link records in tensor memory (one CTA of 12 warps
 * per SM, which allocates all of the SM's 512 tensor-memory columns for the
 * duration of the call; a kernel of another stream holding columns on the
 * same SM delays it until they are released).
 * Errors: FN_EINVAL for dof != 7, E < 0, S out of range, K out of range or a
 * non-ascending / non-positive grid in FULL mode, a NULL required pointer,
 * unknown mode.  FN_ECUDA if the kernel's shared-memory size cannot be set.
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
 * fn_time_edges_nary -- minimum feasible duration refined by the N-ary
 * search of Sec. IV-D (the search after Def. "Minimum feasible time").
 *
 * First the grid scan of FN_MODE_FULL (same grid, cap and k_star rule).
 * For an edge with k* >= 0 the bracket [a, b] = [T_{k*-1}, T_{k*}]
 * (a = 0 for k* = 0) is then refined in rounds while b - a > eps and fewer
 * than max_rounds rounds ran: with w = (b - a) / 32 the interior points
 * t_j = fmaf(j, w, a), j = 1..31 (single precision) are checked in
 * ascending order (rho_tau <= 1 and rho_P <= 1, S samples each), and the
 * bracket becomes [t_{j-1}, t_j] for the first passing t_j (t_0 = a), or
 * [t_31, b] if none passes.  No monotonicity is assumed, as in the grid
 * scan.  rho_v is checked once at the refined T* = b.  A round takes about
 * log2(32) = 5 bits of T*: ceil(log_32(width / eps)) rounds in all.
 *
 * Arguments (as fn_time_edges unless stated)
 *   T_grid, K   host [K] f32 ascending grid, 1 <= K <= FN_MAX_GRID.
 *   T_cap       device [E] f32 or NULL.
 *   eps         bracket width to reach (seconds, f32, > 0, finite).
 *   max_rounds  0..16 (0: the grid result).
 *   k_star      device [E] i32: the grid index (-1 none, -2 invalid input).
 *   T_star      device [E] f32: refined duration b (+inf none, NaN invalid).
 *   T_lo        device [E] f32 or NULL: the bracket's lower end a, the last
 *               duration shown infeasible (0 if none was); NaN if k* < 0.
 *   rho3, ok    device: (rho_tau, rho_P, rho_v) and ok at T_star.
 *   rounds      device [E] i32 or NULL: rounds run.
 *   sample_count device, one u64 or NULL: torque evaluations are ADDED.
 *   stream      cudaStream_t or NULL.
 * Ownership: all device buffers are the caller's; nothing is allocated.
 * Errors: FN_EINVAL for a bad argument (nothing launched), FN_ECUDA on a
 * launch error.  Non-finite states give k_star = -2 for that edge only.
 */
fn_status fn_time_edges_nary(const fn_arm_t* arm, const float* s0, const float* s1, int E,
                             const float* T_grid, int K, int S, const float* T_cap, float eps,
                             int max_rounds, int32_t* k_star, float* T_star, float* T_lo,
                             float* rho3, uint8_t* ok, int32_t* rounds,
                             unsigned long long* sample_count, void* stream);

/*
 * fn_check_edges_full -- the full-resolution recheck of a plan's edges
 * (Sec. IV-E: clearance and dynamics are checked coarsely during the search
 * and the plan sent to the controller is rechecked at full resolution).
 * Each edge at its own duration T[e]: rho_tau, rho_P over all S samples and
 * rho_v (Def. "Feasibility Check", Eq. (rho)), and the least link-capsule
 * clearance to the obstacle spheres over S_clear equally spaced points
 * (both ends included).  ok[e] = rho_tau, rho_P, rho_v <= 1 and (no
 * obstacles, or clearance >= margin).
 *   s0, s1     device [E][16] f32 (16-byte aligned); T device [E] f32.
 *   E          capacity; E_dev (device, one int, or NULL): the edges actually
 *              present (min(E, *E_dev) are checked), for chaining after
 *              fn_planner_incumbent_path without a host synchronisation.
 *   S          2..FN_MAX_S; S_clear >= 2 when n_obs > 0.
 *   n_obs, obs 0..FN_MAX_OBS spheres, host [n_obs][4] (centre, radius).
 *   rho3       device [E][3] f32; clearance device [E] f32 (+inf without
 *              obstacles); ok device [E] u8.
 * Non-finite states or T <= 0 give NaN ratios and clearance and ok = 0.
 * Errors: FN_EINVAL for a bad argument, FN_ECUDA on a launch error.
 */
fn_status fn_check_edges_full(const fn_arm_t* arm, const float* s0, const float* s1,
                              const float* T, int E, const int* E_dev, int S, int S_clear,
                              int n_obs, const float* obs, float margin, float* rho3,
                              float* clearance, uint8_t* ok, void* stream);

/*
 * fn_controller_torque -- one cycle of the tracking controller of
 * Eq. (controller) for B independent instances.
 *
 * From the measured state (q, qd) the cubic is refitted to the rendezvous
 * (q_g, qd_g) over the horizon T; its initial acceleration
 * 6 (q_g - q) / T^2 - (4 qd + 2 qd_g) / T is clipped per joint to [l, u],
 * the box that keeps the velocity after one control period dt inside the
 * taper: l = (-qdbar(q) - qd) / dt, u = (qdbar(q) - qd) / dt.  Eq. (torque)
 * (RNEA + armature + friction) at (q, qd, qdd_des) gives the command, which
 * is clipped to the arm's torque limits, then scaled as a whole onto W_max
 * if |sum_j tau_j qd_j| exceeds it, then (with tau_prev) held within
 * tau_rate_max dt of the previous command.
 *   state, goal  device [B][16] f32: (q, pad, qd, pad) measured / rendezvous.
 *   T            device [B] f32 horizons (> 0).
 *   tau_prev     device [B][7] f32 or NULL (no slew clip).
 *   dt           control period (s, > 0).
 *   tau_rate_max host [7] f32 (N m/s, >= 0); required with tau_prev.
 *   tau          device [B][7] f32; qdd_des device [B][7] f32 or NULL.
 *   flags        device [B] u8 or NULL: bit 0 acceleration clipped, 1 torque,
 *                2 power, 3 slew; 0x80 invalid input (non-finite values or
 *                T <= 0), whose tau and qdd_des are NaN.
 * Errors: FN_EINVAL for a bad argument, FN_ECUDA on a launch error.
 */
fn_status fn_controller_torque(const fn_arm_t* arm, int B, const float* state, const float* goal,
                               const float* T, const float* tau_prev, float dt,
                               const float* tau_rate_max, float* tau, float* qdd_des,
                               uint8_t* flags, void* stream);

/*
 * fn_autotune_time_edges -- the schedule autotuner for fn_time_edges: runs
 * the call (same arguments) with every compiled schedule variant of the edge
 * kernel, `reps` timed runs each after one warm-up, and records the fastest
 * for this (mode, E bucket, K, S) on the current device; later fn_time_edges
 * calls of that shape use it.  Variants 0-2: the scalar scan (one sample per
 * lane) at three register budgets (resident blocks per SM), identical
 * results; variant 3 (the default of untuned shapes): the paired scan (two
 * samples per lane, paired FP32 arithmetic, the torque recursion's per-link
 * records in tensor memory), whose torques round differently in the last
 * bits, so k* can differ from the scalar scan's only where a limit ratio is
 * within FP32 rounding of 1.  The outputs are left as computed by the last
 * variant.  chosen: host, the winning variant index (may be NULL);
 * variant_ms: host [4] mean ms per variant (may be NULL).  Synchronous.
 */
fn_status fn_autotune_time_edges(const fn_arm_t* arm, const float* s0, const float* s1, int E,
                                 const float* T_grid, int K, int S, int mode,
                                 const float* T_fixed, const float* T_cap, int32_t* k_star,
                                 float* T_star, float* rho3, uint8_t* ok, int reps, int* chosen,
                                 float* variant_ms, void* stream);

/*
 * fn_time_edges_set_variant -- pin the schedule variant (0..3, as listed
 * under fn_autotune_time_edges) that fn_time_edges uses for calls of this
 * shape (mode, E's bucket, K, S) on the current device, e.g. to restore a
 * choice fn_autotune_time_edges made in an earlier process.  The N-ary
 * refinement follows a FULL-mode choice of 0-2 (its default otherwise).
 * Every variant's k* equals the oracle's up to the feasibility margin.
 * Errors: FN_EINVAL for an unknown mode, a
 * variant outside 0..3, E < 1, S out of range or (FULL) K out of range.
 */
fn_status fn_time_edges_set_variant(int mode, int E, int K, int S, int variant);

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
 * fn_knn_tree_static -- fn_knn_tree for callers that cannot allocate device
 * memory.  (The paper has no counterpart; this is a property of the library.)
 *
 * Who needs it: a real-time planning thread must not enter the CUDA
 * allocator mid-cycle, because cudaMalloc can synchronise the device and take
 * milliseconds inside a 20 ms budget; an embedded host may have all device
 * memory budgeted at start-up.  Such callers cannot provide fn_knn_tree's
 * workspace.  This entry point takes the same arguments minus the workspace
 * and computes the same result: its split pass uses a fixed file-scope device
 * array of 16 MiB that every GPU loading the library holds until the process
 * exits.  The call itself allocates nothing (no cudaMalloc, no library
 * allocator).
 *
 * Limits and caveats:
 *  - B <= FN_KNN_STATIC_MAX_QUERIES (65536); larger B returns FN_EINVAL.
 *    Within the limit the number of node splits is reduced to what fits.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, once per device, with that device current).
 *    Make that first call before any stream capture.  The address is kept
 *    for the life of the process: after cudaDeviceReset (or any teardown of
 *    the device's primary context) the library must be unloaded and loaded
 *    again before this entry point is called on that device.
 *  - The split pass uses at most nsplit * B * (8 or 16) * 8 bytes of the
 *    array (about 5 MiB for any B: the split count falls as B grows); the
 *    array is sized for two splits of the largest B.
 *  - All calls share the one array.  Calls that overlap on the GPU (other
 *    streams, other host threads) race on it and must be serialised by the
 *    caller.  The array keeps the last call's contents; nothing in it needs
 *    to start at zero, because every entry is written before it is read.
 */
#define FN_KNN_STATIC_MAX_QUERIES 65536
fn_status fn_knn_tree_static(const float* tree, int N, int first, const float* queries, int B,
                             int k, float w_vel, int32_t* idx, float* d2, void* stream);

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


/* ------------------------------------------------------------------------
 * Planner: batched expansion of Algorithm 1 over P independent problems.
 * ------------------------------------------------------------------------ */

/* Static sizes of a planner (Sec. IV-E: the tree is preallocated as a
 * struct of arrays; every buffer is sized here, once). */
typedef struct {
  int P;              /* independent problems (1..1024)                      */
  int n_cap;          /* tree capacity per problem (2..1<<22; P*n_cap <= 2^30) */
  int b_max;          /* largest candidate batch per problem (1..1<<16)      */
  int k;              /* parents per candidate incl. the root (1..17)        */
  int K;              /* duration grid size (1..FN_MAX_GRID)                 */
  float T_lo, T_hi;   /* log grid T_i = T_lo (T_hi/T_lo)^(i/(K-1))           */
  int S;              /* collocation points of the dynamics check            */
  int S_clear;        /* collocation points of the clearance check (>= 2)    */
  int reach_grid;     /* points of the Eq. (reach) grid (>= 2)               */
  float w_vel;        /* velocity weight of the parent distance              */
  float vel_frac;     /* free samples: |qd_j| <= vel_frac * qdbar_j(q_j)     */
  float clear_margin; /* minimum clearance of an edge, metres                */
  int edge_blocks;    /* persistent blocks of the edge kernel (0 = auto)     */
} fn_planner_cfg_t;

#define FN_MAX_OBS 8

/* One planning problem (Def. "Interception planning"): the measured root
 * state, the ballistic flight estimate of Eq. (ballistic) with the reach
 * window, latency compensation (Sec. IV-F: plan time t corresponds to flight
 * time t + t_offset), the uncertainty model of Sec. IV-B, the manifold
 * thresholds of Def. 2, the objective constants of Eq. (objective), the
 * end-effector speed bound of Eq. (reach), obstacle spheres, the batch of
 * this problem and its goal share, and the Philox seed. */
typedef struct {
  float q0[7], qd0[7];
  float x0[3], v0[3], g[3];
  float t_enter, t_fall, t_offset;
  float sig_p, sig_v, sig_a;
  int sig_linear;            /* 1: sigma(t) = sig_lin_a + sig_lin_b t */
  float sig_lin_a, sig_lin_b;
  float a_min, v_min;
  float w_v, v_target, w_p, w_r, w_x, r_catch, nu0, lam;
  float v_tip;
  int batch;                 /* candidates this round (<= b_max)      */
  int n_goal;                /* goal candidates among them            */
  int n_obs;                 /* obstacle spheres (<= FN_MAX_OBS)      */
  float obs[FN_MAX_OBS][4];  /* centre xyz, radius                    */
  unsigned long long seed;
} fn_problem_t;

/* Output of one iteration per problem (Algorithm 1's return value, D9). */
/* fn_rendezvous_t.status bits: candidates dropped because the tree reached
 * n_cap; a duration search hit its pass bound (an internal error, never
 * expected: the search state machine progresses every pass, and the bound
 * stops a scan that would not, leaving that edge's grid result in place) */
#define FN_PLAN_TREE_FULL 1
#define FN_PLAN_ERR_SCAN 2

typedef struct {
  float q_g[7], qd_g[7];  /* end state of the incumbent plan's first edge  */
  float T;                /* that edge's duration from the root            */
  float J;                /* incumbent score (-inf if none)                */
  float t_best;           /* incumbent arrival time (t_fall if none)       */
  int incumbent;          /* incumbent node id (-1 if none)                */
  int n_nodes;            /* tree size after the iteration                 */
  int n_added;            /* nodes attached in this iteration              */
  int status;             /* 0, or FN_PLAN_TREE_FULL | FN_PLAN_ERR_SCAN     */
} fn_rendezvous_t;

typedef struct fn_planner fn_planner_t;

/* Allocates every device and pinned host buffer of the planner (the only
 * allocating call).  `arm` is copied.  FN_ENOMEM if an allocation fails. */
fn_status fn_planner_create(const fn_planner_cfg_t* cfg, const fn_arm_t* arm,
                            fn_planner_t** out);
fn_status fn_planner_destroy(fn_planner_t* pl);

/* Algorithm 1, first line: each problem's tree becomes its root
 * (q0, qd0, t = 0); the incumbent is cleared and t_best = t_fall.
 * probs: host [P], copied into the reset's own pinned staging before the
 * call returns.  Asynchronous on `stream`: the call returns once the work is
 * enqueued (the next reset waits, on the host, for this one's copy). */
fn_status fn_planner_reset(fn_planner_t* pl, const fn_problem_t* probs, void* stream);

/* Replace problem p's tree with n host nodes (states [n][16], time-to-come
 * t[n], parent[n] with parent[0] = -1 and parent[i] < i): used to start an
 * iteration from a given tree.  Nodes carry no score and nu = 0.
 * Asynchronous on `stream`: the copies are enqueued and the call returns, as
 * cudaMemcpyAsync does; host arrays in page-locked memory must stay
 * unchanged until the stream has executed the copies (pageable arrays may be
 * reused at once). */
fn_status fn_planner_load_tree(fn_planner_t* pl, int p, const float* states, const float* t,
                               const int32_t* parent, int n, void* stream);

/* Give problem p an explicit candidate batch for the next iteration that
 * runs with FN_PLAN_EXTERNAL: host states [B][16]; the first n_goal are goal
 * candidates with required arrival T_req[n_goal] and relative speed
 * v_rel[n_goal] (|v_b - xdot(T)| of Eq. (terms)). */
fn_status fn_planner_set_candidates(fn_planner_t* pl, int p, const float* states, int B,
                                    int n_goal, const float* T_req, const float* v_rel,
                                    void* stream);

#define FN_PLAN_EXTERNAL 1u /* use the candidates given by fn_planner_set_candidates */
#define FN_PLAN_PRUNE 2u    /* prune the trees after the round (Eq. (reach))          */
#define FN_PLAN_DENSITY 4u  /* goal parameters drawn from p_theta (else uniform); the
                               best-plans archive is updated after the round        */
#define FN_PLAN_CHORD 8u    /* free candidates from the chord sampler (else uniform) */
#define FN_PLAN_REFIT 16u   /* update the archive and refit p_theta to it after the
                               round (the last round of an anytime iteration)       */
#define FN_PLAN_NARY 32u    /* refine the free edges' durations by the N-ary search
                               (fn_planner_set_refine)                              */
#define FN_PLAN_GREFINE 64u /* gradient refinement of the incumbent rendezvous
                               (fn_planner_set_grefine)                             */

/*
 * fn_plan_iteration -- one round of Algorithm 1 for all P problems:
 *   sample B_p candidates (unless FN_PLAN_EXTERNAL): the first n_goal by
 *     the goal chart (Def. "Goal chart"), the rest uniform in the joint box
 *     with |qd| <= vel_frac qdbar(q); Philox4x32-10 counter
 *     (candidate, iter, problem, stream), key = seed;
 *   Parents: root + (k-1) nearest nodes (fn_knn_tree's metric);
 *   goal edges: one check at T_req - t(p); free edges: first feasible grid
 *     duration with t(p) + T <= t_best (FN_MODE_FULL with a cap);
 *   Clear: link capsules vs obstacle spheres at S_clear points of the edge,
 *     rejected below clear_margin;
 *   attach each candidate to the ok parent of least t(p) + T_p (ties: lower
 *     parent slot), appended in candidate order;
 *   incumbent = argmax J (Eq. (objective)) over rendezvous nodes (ties: lower
 *     node id); t_best = its arrival time;
 *   with FN_PLAN_PRUNE, Eq. (reach) pruning (root kept, descendants of
 *     pruned nodes removed, order and parents preserved).
 * Enqueued on `stream`; returns after the stream has finished and `out`
 * (host [P]) holds each problem's rendezvous.  probs: host [P].
 */
fn_status fn_plan_iteration(fn_planner_t* pl, const fn_problem_t* probs, int iter,
                            unsigned flags, fn_rendezvous_t* out, void* stream);

/*
 * CUDA-graph form of fn_plan_iteration: fn_planner_capture records one
 * iteration (with `flags`) into a graph; fn_plan_replay refreshes the
 * problems and the iteration counter through the planner's pinned staging
 * buffer, launches the graph on `stream` and returns like fn_plan_iteration.
 */
fn_status fn_planner_capture(fn_planner_t* pl, unsigned flags, void* stream);
fn_status fn_plan_replay(fn_planner_t* pl, const fn_problem_t* probs, int iter,
                         fn_rendezvous_t* out, void* stream);

/*
 * fn_plan_replay_async -- fn_plan_replay without waiting: stages `probs` and
 * `iter` and launches the captured graph on `stream`, then returns; the
 * rendezvous records are read with fn_plan_result.  The staging is pinned
 * host memory that the graph's own copies read, so a call waits (on the host)
 * for the previous asynchronous replay's graph to finish before staging
 * again; fn_plan_iteration and fn_plan_replay do the same (fn_planner_reset
 * stages into its own buffer).
 * Everything else is as fn_plan_replay (Algorithm 1's loop body, one
 * iteration per call).  Errors as fn_plan_replay.
 */
fn_status fn_plan_replay_async(fn_planner_t* pl, const fn_problem_t* probs, int iter,
                               void* stream);

/*
 * fn_plan_result -- wait for the last fn_plan_replay_async and copy its
 * rendezvous records (host [P]) to `out`.  FN_EINVAL if no asynchronous
 * replay was launched on this planner.
 */
fn_status fn_plan_result(fn_planner_t* pl, fn_rendezvous_t* out);

/* Schedule autotuner of the planner (the work pattern of an iteration is
 * data dependent, so variants are timed on the caller's own problems): runs
 * the iteration's sampling and parent search once, then times every
 * schedule of the edge phase on that edge batch (`reps` runs each after a
 * warm-up) and keeps the fastest for this planner and later planners of the
 * same shape.  Schedules 0-2: the packed stages (lanes over probe and
 * verification items) at three register budgets; 3: one warp per edge on
 * the paired core with its records in tensor memory, one launch.  The trees
 * are not modified.  chosen: host (may be NULL); variant_ms: host [4] (may
 * be NULL).
 * Synchronous. */
fn_status fn_planner_autotune(fn_planner_t* pl, const fn_problem_t* probs, int iter,
                              unsigned flags, int reps, int* chosen, float* variant_ms,
                              void* stream);

/* Sets the planner's edge-phase schedule (the index fn_planner_autotune
 * reports: 0-2 the packed stages, 3 one warp per edge on the paired core)
 * for its later iterations and captures; a graph captured earlier keeps the
 * schedule it was captured with.  FN_EINVAL for an index outside [0, 4). */
fn_status fn_planner_set_schedule(fn_planner_t* pl, int variant);

/* Durations in ms of the last fn_plan_iteration's phases, from CUDA events
 * recorded on its stream: [0] schedule, [1] sample, [2] parents (kNN),
 * [3] edge prep + item scan, [4] probe (the end-sample torque split of every
 * edge with admissible durations, then both end samples of every admissible
 * (edge, duration) item), [5] verify (surviving durations, rho_v, Clear),
 * [6] attach + score, [7] prune, [8] output.  ms: host [9].  FN_EINVAL
 * before the first fn_plan_iteration. */
fn_status fn_planner_phase_ms(fn_planner_t* pl, float* ms);

/* Durations in ms of every kernel launch of the last fn_plan_iteration, in
 * launch order, from CUDA events recorded on its stream after each launch
 * (so a launch's time includes its wait for the previous one to drain).
 * names[i]: the kernel's name (static strings owned by the library).
 * ms, names: host [cap]; *n = launches traced (up to 40; min(n, cap)
 * written).  FN_EINVAL before the first fn_plan_iteration. */
fn_status fn_planner_kernel_ms(fn_planner_t* pl, float* ms, const char** names, int cap, int* n);

/* Torque evaluations (edge, duration, sample) performed by the planner's
 * edge kernels since creation or the last reset (reset != 0 zeroes every
 * work counter): count[0] by the probe stages (end and interior samples),
 * count[1] by the verify stages.  count: host [2]. */
fn_status fn_planner_sample_count(fn_planner_t* pl, unsigned long long* count, int reset);

/* All work counters of the planner's kernels since creation or the last
 * reset: [0] torque evaluations of the end-sample probe (three per end of
 * every edge with admissible durations: the split of Eq. (torque) into
 * alpha / T^2 + beta / T + gamma that the per-duration checks then use), [1]
 * of the verify
 * stages, [2] of the interior-sample probe, [3] (query, node) distance
 * evaluations of the parent search, [4] IK starts run by the goal sampler,
 * [5] edges timed by the surrogate's window pass, [6] of those rescanned
 * in full (certificate failed), [7] torque evaluations of the N-ary
 * refinement (FN_PLAN_NARY), [8..13] goal-chart draws by outcome (Def. "Goal
 * chart": phi is undefined where the IK has no solution or qd_g exceeds its
 * bounds): [8] defined, [9] |v_rel| below v_min, [10] no IK start converged,
 * [11] IK solution outside the joint box, [12] singular contact-point
 * Jacobian, [13] qd_g over the velocity taper.  count: host [n] (n <= 14
 * written).  reset != 0 zeroes them all. */
fn_status fn_planner_work_counts(fn_planner_t* pl, unsigned long long* count, int n, int reset);

/* Copy problem p's tree to host (any pointer may be NULL): states [n][16],
 * t[n], parent[n], J[n] (NaN for non-rendezvous nodes), nu[n]; *n = size.
 * Synchronous. */
fn_status fn_planner_get_tree(fn_planner_t* pl, int p, float* states, float* t,
                              int32_t* parent, float* J, float* nu, int* n, int cap);
/*
 * fn_planner_set_refine -- the N-ary refinement of rounds run with
 * FN_PLAN_NARY: every free edge that found a grid duration T_k is refined on
 * (T_{k-1}, T_k] as fn_time_edges_nary does (N = 32, rounds while the
 * bracket is wider than eps, at most max_rounds), and its rho_v and
 * clearance are taken at the refined duration, which the attach then uses
 * (Algorithm 1: T_p = min{T <= t_best : rho(T) <= 1}, then Clear at T_p).
 * Defaults: eps = 1e-4 s, 8 rounds.  Set before fn_planner_capture.
 * Errors: FN_EINVAL unless eps > 0 finite and 0 <= max_rounds <= 16.
 */
fn_status fn_planner_set_refine(fn_planner_t* pl, float eps, int max_rounds);

/*
 * fn_planner_set_grefine -- parameters of the rounds run with
 * FN_PLAN_GREFINE: after attach, the incumbent rendezvous node of each
 * problem is refined by gradient ascent on its chart parameters z (the
 * paper's conclusion: the checks and the chart decoder are smooth in the
 * trajectory parameters, and gradient-based refinement of tree nodes is the
 * next step; it fixes no objective, variables or step rule).  Reading:
 * F(z) = J of Eq. (objective) for phi(z) attached to the node's parent
 * (T_p = T_req(z) - t(p), nu = max(nu(parent), rho_v at T_p)) where phi(z)
 * is defined, T_p > 0 and the edge passes Def. "Feasibility Check" at T_p
 * and the clearance, -inf elsewhere; the gradient is the central difference
 * of the same J without the check, step h per coordinate (z2..z4 wrap, the
 * others are clamped); iteration t moves z by eta0 2^-t along the normalised
 * gradient (folded into the cube) and keeps the move when F improves; a zero
 * gradient stops.  A node that improved is appended with the original's
 * parent (the original stays: it may have children) and becomes the
 * incumbent, which the rendezvous then reports.  Nothing happens without an
 * incumbent whose chart parameters are known, or with a full tree.
 * Defaults: iters 8, eta0 0.05, h 1e-3.  Set before fn_planner_capture.
 * Errors: FN_EINVAL unless 0 <= iters <= 64, 0 < eta0 <= 1, 0 < h <= 0.1.
 */
fn_status fn_planner_set_grefine(fn_planner_t* pl, int iters, float eta0, float h);

/*
 * fn_planner_set_grid -- replace the planner's duration grid (Def. "Minimum
 * feasible time" searched over the N-ary slots laid out on one grid) by the
 * caller's K values, host T_grid[K] in seconds, positive, finite and strictly
 * ascending (K = the planner's K).  fn_planner_create builds the log grid
 * T_lo (T_hi/T_lo)^(k/(K-1)) itself; callers that hold the exact single-
 * precision grid another component uses give it here so that both examine
 * the same durations.  A captured iteration is discarded (capture again).
 * Errors: FN_EINVAL for a bad argument.
 */
fn_status fn_planner_set_grid(fn_planner_t* pl, const float* T_grid, int K);

/*
 * The sampling densities of Sec. IV-E ("Batched expansion").
 *
 * p_theta: goal parameters z in the chart's cube [0, 1]^9 come from a
 * Gaussian mixture (C <= FN_DENSITY_MAX_C diagonal components) mixed with a
 * uniform component of weight w_u.  A Gaussian draw is folded back into the
 * cube (the angle parameters z2, z3, z4 wrap modulo 1, the others reflect
 * at 0 and 1).  p_theta is kept per problem on the device; fn_planner_reset
 * does not clear it (it persists across planning cycles).  C = 0 draws every
 * z uniformly, exactly as without FN_PLAN_DENSITY.
 *
 * Best-plans archive: per problem, the FN_ARCHIVE_MAX (at most n_fit) best
 * (J, z) of the rendezvous nodes attached since the last reset, best first
 * (an earlier plan wins a tie).  It is updated after every round run with
 * FN_PLAN_DENSITY or FN_PLAN_REFIT, from the new nodes whose z is known
 * (device-drawn goals, or external ones given fn_planner_set_candidate_params).
 *
 * Refit (FN_PLAN_REFIT): em_iters EM iterations with diagonal covariances
 * on the archive's z, starting from the current mixture (or, the first
 * time, from the min(C, n) best z with deviation sd_init and equal weights);
 * sd_floor^2 is added to every variance; a component whose responsibility
 * sum falls below 1e-4 keeps its mean and deviation.  w_u is set from the
 * configuration, not fit.
 *
 * Chord sampler (FN_PLAN_CHORD): a free candidate is, with probability
 * w_chord and if the round decoded any valid goal, the point
 * q0 + lambda (q_g - q0) + chord_sigma * half-range * n on the chord from the
 * root q0 to a goal q_g of the round chosen uniformly (lambda uniform, n
 * standard normal), clamped to the joint box; otherwise a uniform draw.
 * Its velocity is drawn as for a uniform candidate.
 */
#define FN_DENSITY_MAX_C 4
#define FN_ARCHIVE_MAX 64

typedef struct {
  int C;                          /* Gaussian components (0: uniform only)   */
  float w_u;                      /* weight of the uniform component         */
  float pi[FN_DENSITY_MAX_C];     /* component weights (sum 1)               */
  float mu[FN_DENSITY_MAX_C][9];  /* means over the chart parameters         */
  float sd[FN_DENSITY_MAX_C][9];  /* standard deviations (> 0)               */
} fn_density_t;

typedef struct {
  float w_u;          /* uniform weight of p_theta (default 0.25)             */
  int C;              /* components of a refit, 1..4 (4)                       */
  int n_fit;          /* archive size, 1..FN_ARCHIVE_MAX (32)                  */
  int em_iters;       /* EM iterations per refit, 1..64 (8)                    */
  float sd_floor;     /* added in quadrature to every deviation (0.02)         */
  float sd_init;      /* deviation of a first fit's components (0.1)           */
  float w_chord;      /* probability of a chord draw for a free candidate (0.5) */
  float chord_sigma;  /* chord spread, fraction of the joint half-range (0.1)  */
} fn_sampler_cfg_t;

/* Set the sampling configuration (before fn_planner_capture: a captured
 * iteration keeps the configuration it was captured with). */
fn_status fn_planner_set_sampler(fn_planner_t* pl, const fn_sampler_cfg_t* cfg);

/* Set problem p's p_theta (host struct; validated: 0 <= C <= 4,
 * 0 <= w_u <= 1, pi >= 0 summing to 1 within 1e-3, sd > 0, finite). */
fn_status fn_planner_set_density(fn_planner_t* pl, int p, const fn_density_t* theta,
                                 void* stream);

/* Read problem p's p_theta and best-plans archive (host outputs, any may be
 * NULL: archive_J [FN_ARCHIVE_MAX], archive_z [FN_ARCHIVE_MAX][9],
 * archive_n).  Synchronises the device. */
fn_status fn_planner_get_density(fn_planner_t* pl, int p, fn_density_t* theta,
                                 float* archive_J, float* archive_z, int* archive_n);

/* Chart parameters z (host [n_goal][9]) of the external goal candidates
 * given by fn_planner_set_candidates (call after it), so that their plans
 * can enter the archive; without it their z is unknown (NaN). */
fn_status fn_planner_set_candidate_params(fn_planner_t* pl, int p, const float* z, int n_goal,
                                          void* stream);

/* Read the chart parameters of problem p's first n candidate slots (host
 * [n][9]; NaN where unknown: free slots, external goals without parameters).
 * Synchronises the device. */
fn_status fn_planner_get_candidate_params(fn_planner_t* pl, int p, float* z, int n);

/*
 * fn_planner_incumbent_path -- the incumbent plan of problem p as a list of
 * edges, root first: edge i runs from node nodes[i] to nodes[i + 1] with the
 * duration stored with its end node (the plan that Sec. IV-E rechecks at
 * full resolution before it goes to the controller).
 *   max_edges  capacity of the outputs (edges).
 *   s0, s1     device [max_edges][16] f32 (16-byte aligned): edge states.
 *   T          device [max_edges] f32: edge durations (NaN for edges into
 *              nodes given by fn_planner_load_tree, which carry none).
 *   nodes      device [max_edges + 1] i32 or NULL.
 *   n_edges    device, one i32: the path length L (0: no incumbent; -1: the
 *              parent links do not reach the root).  The arrays are written
 *              only when 0 < L <= max_edges.
 * Stream-ordered after the iteration that produced the incumbent; no host
 * synchronisation (chain fn_check_edges_full with E_dev = n_edges).
 * Errors: FN_EINVAL for a bad argument.
 */
fn_status fn_planner_incumbent_path(fn_planner_t* pl, int p, int max_edges, float* s0, float* s1,
                                    float* T, int32_t* nodes, int32_t* n_edges, void* stream);

/* Copy problem p's last candidate batch to host: states [B][16], T_req[B],
 * v_rel[B], valid[B] (goal candidates whose chart decoding succeeded, and
 * every free candidate).  Synchronous. */
fn_status fn_planner_get_candidates(fn_planner_t* pl, int p, float* states, float* T_req,
                                    float* v_rel, uint8_t* valid, int cap);
/* Copy problem p's last parent lists to host: nn [B][k-1] int32, row b the
 * tree indices of candidate b's k-1 nearest non-root nodes under the
 * distance of Sec. IV-E "Parents" (ascending, ties to the lower index; -1
 * where the tree has fewer nodes).  The root, parent slot 0, is implicit.
 * Rows beyond the batch of the last iteration are stale.  Synchronous. */
fn_status fn_planner_get_parents(fn_planner_t* pl, int p, int32_t* nn, int cap);
/* Copy problem p's per-edge results of the last iteration to host, row b
 * slot j = the edge from candidate b's parent j (slot 0 the root, slot j > 0
 * the node nn[b][j-1] of fn_planner_get_parents) to the candidate; arrays
 * [cap][k], any pointer may be NULL:
 *   k_star  free edge: the first feasible grid index with t(p) + T_k <=
 *           t_best (Def. "Minimum feasible time" under Algorithm 1's bound),
 *           -1 if none; goal edge: 0 if rho_tau, rho_P <= 1 at T_p, else -1;
 *           -2 for non-finite states (the edge is invalid);
 *   T       free edge: T_{k*} (+inf if none); goal edge: T_p = T_req - t(p)
 *           in single precision (NaN where the candidate or the parent does
 *           not exist);
 *   rho_v   Eq. (rho)'s velocity term at T (NaN where not evaluated);
 *   ok      1 iff the edge passed every check of Def. "Feasibility Check"
 *           at T and the clearance (Algorithm 1's Clear): the edges the
 *           attach chooses from.
 * Rows beyond the batch of the last iteration are stale.  Synchronous.
 * Errors: FN_EINVAL for a bad argument, FN_ECUDA for a failed copy. */
fn_status fn_planner_get_edges(fn_planner_t* pl, int p, int32_t* k_star, float* T, float* rho_v,
                               uint8_t* ok, int cap);
/* Copy problem p's per-node chart parameters to host: z [cap][9] f32, row n
 * the z of rendezvous node n (Def. "Goal chart"), NaN for free nodes and
 * for goal nodes whose z is unknown (candidates given without parameters).
 * Synchronous.  Errors: FN_EINVAL for a bad argument, FN_ECUDA. */
fn_status fn_planner_get_node_params(fn_planner_t* pl, int p, float* z, int cap);

/* Routes the free edges of the following iterations (those with an
 * admissible duration) through the duration surrogate: the model predicts a
 * window of W grid durations per edge, the window is scanned with its
 * certificate and uncertified edges are rescanned in full (as
 * fn_edges_time_window); goal edges keep their fixed-duration check.  The
 * planner keeps the pointer (the model must outlive the planner or be
 * detached with mlp = NULL) and uses the weights current at each iteration.
 * Capture graphs after setting it.  Allocates on the first call. */
struct fn_mlp;
fn_status fn_planner_set_surrogate(fn_planner_t* pl, struct fn_mlp* mlp, int W);

/* ------------------------------------------------------------------------
 * Packed edge engine: the planner's edge pipeline (Sec. IV-D search as a
 * probe of both end samples of every admissible (edge, duration), a probe of
 * four interior samples of the survivors, then verification of each edge's
 * lowest surviving duration, all with lanes packed over items) applied to
 * edge arrays given by the caller.  Same result as fn_time_edges mode FULL
 * (first feasible grid index, rho_v at it), without the (rho_tau, rho_P)
 * ratios.
 * ------------------------------------------------------------------------ */
typedef struct fn_edges fn_edges_t;

/* Sizes the engine once (up to max_E <= 65536 edges per pass; longer calls
 * run in passes) for the grid T_grid (host [K], ascending, positive) and S
 * collocation points.  Allocates; synchronous. */
fn_status fn_edges_create(const fn_arm_t* arm, const float* T_grid, int K, int S, int max_E,
                          fn_edges_t** out);
fn_status fn_edges_destroy(fn_edges_t* eg);

/* First feasible grid index with T_k <= T_cap[e] (T_cap device [E] or NULL
 * for no cap) of each edge (device s0, s1 [E][16], 16-byte aligned).
 * Outputs (device [E]): k_star (-1 none, -2 non-finite input), T_star
 * (T_{k*}; +inf none; NaN invalid), rho_v (at k*; NaN otherwise), ok (k* >= 0
 * and rho_v <= 1).  Asynchronous on `stream`; one engine serves one call at
 * a time. */
fn_status fn_edges_time(fn_edges_t* eg, const float* s0, const float* s1, int E,
                        const float* T_cap, int32_t* k_star, float* T_star, float* rho_v,
                        uint8_t* ok, void* stream);

/* The windowed scan of the duration surrogate: per edge, the window of W
 * grid durations around the prediction Y (device [E][2], fn_mlp_predict's
 * output) plus the index below it; the window's first feasible index is
 * accepted if it is 0 or the index below was infeasible, "none" if the
 * window reached the top of the grid; every other edge is rescanned in
 * full.  path (device [E] or NULL): 0 certified by the window, 1 rescanned.
 * Outputs as fn_edges_time. */
fn_status fn_edges_time_window(fn_edges_t* eg, const float* s0, const float* s1, int E,
                               const float* Y, int W, int32_t* k_star, float* T_star,
                               float* rho_v, uint8_t* ok, uint8_t* path, void* stream);

/* The engine's work counters (as fn_planner_work_counts). */
fn_status fn_edges_work_counts(fn_edges_t* eg, unsigned long long* count, int n, int reset);

/* ------------------------------------------------------------------------
 * Duration surrogate (the project's addition; the paper has no learned
 * component).  An MLP 28 -> 256 -> 256 -> 256 -> 2 with ReLU predicts
 * (log T*, feasibility logit) of an edge from its boundary states; the
 * windowed scan uses it to examine a few durations instead of the whole
 * grid, with the exact scan as fallback.
 *
 * Features: q scaled by the joint box to [-1, 1], qdot by qd_max, for s0 and
 * s1 (28 values, padded to 32).  Precision: features, weights and hidden
 * activations in bf16 on the tensor cores with FP32 accumulation; outputs,
 * losses and gradients of the outputs in FP32; Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8) on FP32 master weights.  Loss over a batch of n edges with labels
 * k* from the exact scan: (1/n) sum [f (y0 - log T_{k*})^2 + BCE(y1, f)],
 * f = (k* >= 0).  Weights W_l are [in][out] row-major.
 * ------------------------------------------------------------------------ */
typedef struct fn_mlp fn_mlp_t;

/* Allocates the weights (He-uniform from `seed`, zero biases), Adam state
 * and a workspace for batches of up to max_batch edges. */
fn_status fn_mlp_create(int max_batch, unsigned long long seed, fn_mlp_t** out);
fn_status fn_mlp_destroy(fn_mlp_t* m);

/* Y[e] = (log T*_pred, feasibility logit) for E edges (device s0, s1 [E][16],
 * 16-byte aligned; device Y [E][2]), any E.  Runs on the 5th-generation
 * tensor cores (tcgen05, accumulators in tensor memory), one fused launch;
 * the packed weights are refreshed on the stream after any weight change.
 * A timeout inside the kernel raises the flag read by fn_mlp_error. */
fn_status fn_mlp_predict(fn_mlp_t* m, const fn_arm_t* arm, const float* s0, const float* s1,
                         int E, float* Y, void* stream);

/* The same forward on the training kernels' path (mma.sync GEMMs through
 * the model's workspace, chunks of max_batch).  Same rounding points; the
 * two differ only by FP32 summation order. */
fn_status fn_mlp_predict_ref(fn_mlp_t* m, const fn_arm_t* arm, const float* s0, const float* s1,
                             int E, float* Y, void* stream);

/* Error flag of the tensor-core kernel (1 after a timed-out wait); reset
 * != 0 clears it.  Synchronous. */
fn_status fn_mlp_error(fn_mlp_t* m, int* flag, int reset);

/* Loss and gradients of one batch (E <= max_batch; k_star device [E] from
 * the exact scan over the host grid T_grid [K]); *loss (host, may be NULL)
 * receives the loss.  Gradients stay on the device (fn_mlp_get_grads). */
fn_status fn_mlp_backward(fn_mlp_t* m, const fn_arm_t* arm, const float* s0, const float* s1,
                          const int32_t* k_star, const float* T_grid, int K, int E,
                          float* loss, void* stream);
/* One Adam step with learning rate lr from the stored gradients. */
fn_status fn_mlp_adam_step(fn_mlp_t* m, float lr, void* stream);
/* fn_mlp_backward followed by fn_mlp_adam_step; synchronous when loss != NULL. */
fn_status fn_mlp_train_step(fn_mlp_t* m, const fn_arm_t* arm, const float* s0, const float* s1,
                            const int32_t* k_star, const float* T_grid, int K, int E, float lr,
                            float* loss, void* stream);

/* Host access to layer l (0..3): W [in][out], b [out] (in = 32, 256, 256,
 * 256; out = 256, 256, 256, 2).  Any pointer may be NULL.  Synchronous. */
fn_status fn_mlp_get_params(fn_mlp_t* m, int l, float* W, float* b);
fn_status fn_mlp_set_params(fn_mlp_t* m, int l, const float* W, const float* b);
fn_status fn_mlp_get_grads(fn_mlp_t* m, int l, float* gW, float* gb);
fn_status fn_mlp_set_grads(fn_mlp_t* m, int l, const float* gW, const float* gb);
/* Weights to / from a binary file (magic "FNMLP1", step count, W and b of
 * every layer as little-endian f32). */
fn_status fn_mlp_save(fn_mlp_t* m, const char* path);
fn_status fn_mlp_load(fn_mlp_t* m, const char* path);

/*
 * fn_time_edges_window -- minimum feasible duration with a predicted window.
 * For each edge the window [lo, lo+W) is centred on the grid index nearest
 * exp(Y[e][0]) (the top of the grid if Y[e][1] < 0), clamped into [0, K).
 * The scan of Def. "Minimum feasible time" runs on the window first, from
 * four grid steps below the predicted index (never below lo-1) up to lo+W,
 * and on down to lo-1 only if that starting duration is feasible:
 *  - its first feasible k is accepted if k = 0 or T_{k-1} was shown
 *    infeasible and k >= lo (certified: exact whenever rho_tau, rho_P are
 *    monotone in T, as the paper states for fixed boundary states);
 *  - "no feasible duration" is accepted if the window and T_{K-1} are
 *    infeasible (same certificate);
 *  - otherwise the indices not yet examined are scanned exactly.
 * path[e] (device u8, may be NULL) = 0 when the certificate decided, 1 when
 * the fallback scan ran.  Other arguments and outputs as fn_time_edges
 * (FN_MODE_FULL, no cap); sample_count as fn_time_edges_counted.
 */
fn_status fn_time_edges_window(const fn_arm_t* arm, const float* s0, const float* s1, int E,
                               const float* T_grid, int K, int S, const float* Y, int W,
                               int32_t* k_star, float* T_star, float* rho3, uint8_t* ok,
                               uint8_t* path, unsigned long long* sample_count, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FN_API_H */
