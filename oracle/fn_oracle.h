/*
 * FP64 CPU oracle for the edge-timing planner of "Becoming a Fruit Ninja"
 * (arxiv 2609.22608).  TEST INFRASTRUCTURE ONLY: this library exists so that
 * the tests, the smoke check and the benchmark's CPU-baseline leg can check
 * the CUDA path against plain definitions.  The product path never calls it,
 * and it shares no header, helper or table with the CUDA sources.
 *
 * Every routine evaluates the paper's definitions directly, in double
 * precision, with no blocking or reordering:
 *   cubic edge ............ Def. "Cubic edge", Eq. (cubic)
 *   torque ................ Eq. (torque) = RNEA + reflected rotor inertia + Eq. (friction)
 *   feasibility ratios .... Def. "Feasibility Check", Eq. (rho)
 *   minimum feasible time . Def. "Minimum feasible time" over a duration grid,
 *                           refined by the N-ary search that follows it
 *   nearest parents ....... Sec. IV-E "Batched expansion" (brute-force scan)
 *   goal chart ............ Def. "Goal chart" and the decoding described after it
 *   objective ............. Eq. (objective), Eq. (terms)
 *   arrival-time pruning .. Eq. (reach)
 *   tracking controller ... Eq. (controller) with the torque, power and slew clips
 *   plan recheck .......... Sec. IV-E (the plan sent to the controller, full resolution)
 *   sampling densities .... Sec. IV-E "Batched expansion" (p_theta, chord sampler)
 * Readings of passages that the paper leaves open are listed beside each
 * function in fn_oracle.c.
 */
#ifndef FN_ORACLE_H
#define FN_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int dof;                                   /* 1..7 joints used              */
  double a[7], alpha[7], d[7], theta0[7];    /* modified DH (Craig)           */
  double mass[7], com[7][3], inertia[7][3];  /* link frame, diag about COM    */
  double armature[7];                        /* I_m = J_m n^2                 */
  double fric[7][3];                         /* psi1, psi2, psi3              */
  double q_lo[7], q_hi[7], qd_max[7], taper_a[7];
  double tau_max[7], w_max;
  double gravity[3];
  double flange_d;                           /* EE frame = frame 7 + flange_d z7 */
  double blade_base[3], blade_axis[3], blade_normal[3], blade_len;
  double link_radius[7];
} or_arm;

typedef struct {
  double x0[3], v0[3];          /* flight estimate at measurement time      */
  double t_enter, t_fall;       /* window, plan time                         */
  double t_offset;              /* latency compensation: flight time = T + t_offset */
  double sig_p, sig_v, sig_a;   /* sigma^2(t) = sig_p^2 + (sig_v t)^2 + (sig_a t^2/2)^2 */
  int    sig_linear;            /* 1: sigma(t) = sig_lin_a + sig_lin_b t     */
  double sig_lin_a, sig_lin_b;
  double a_min, v_min;          /* manifold thresholds                       */
  double w_v, v_target, w_p, w_r, w_x, r_catch, nu0, lam;
  double v_tip;                 /* end-effector speed bound for Eq. (reach)  */
  double g[3];                  /* gravity of the flight, Eq. (ballistic)    */
} or_problem;

void or_set_threads(int n);

/* sigma_T(t), its first and second derivative for `n` joints. */
void or_cubic(int n, const double* q0, const double* qd0, const double* q1,
              const double* qd1, double T, double t, double* s, double* sd, double* sdd);

/* rigid-body inverse dynamics only (RNEA, base acceleration = -gravity) */
void or_rnea(const or_arm* arm, const double* q, const double* qd, const double* qdd,
             double* tau);
/* Eq. (torque): RNEA + armature + friction */
void or_torque(const or_arm* arm, const double* q, const double* qd, const double* qdd,
               double* tau);
double or_friction(const double* psi, double qd);
double or_taper(const or_arm* arm, int j, double q);

/* (rho_tau, rho_P, rho_v) of one edge at duration T, S samples incl. both ends */
void or_rho(const or_arm* arm, const float* s0, const float* s1, double T, int S, double* rho3);

/* Edge timing over an ascending duration grid.  mode 0 = full scan (first
 * feasible index), mode 1 = fixed duration per edge (T_fixed[e]).  T_cap may
 * be NULL (no cap).  Outputs as in the library: k_star (-1 none, -2 invalid),
 * T_star, rho3 [E][3], ok. */
void or_time_edges(const or_arm* arm, int E, const float* s0, const float* s1,
                   const float* T_grid, int K, int S, int mode, const float* T_fixed,
                   const float* T_cap, int* k_star, float* T_star, double* rho3,
                   unsigned char* ok);

/* The grid scan refined by the N-ary search (N = 32) to a bracket
 * (T_lo, T_star] no wider than eps (at most max_rounds rounds; rounds[e]
 * counts them).  k_star is the grid scan's index; rho3 and ok are taken at
 * the refined T_star.  margin (may be NULL) reports the smallest
 * |max(rho_tau, rho_P) - 1| over the durations checked. */
void or_time_edges_nary(const or_arm* arm, int E, const float* s0, const float* s1,
                        const float* T_grid, int K, int S, const float* T_cap, float eps,
                        int max_rounds, int* k_star, float* T_star, float* T_lo, double* rho3,
                        unsigned char* ok, int* rounds, double* margin);

/* rho3 at an arbitrary per-edge duration T[e] (all S samples). */
void or_rho_batch(const or_arm* arm, int E, const float* s0, const float* s1,
                  const double* T, int S, double* rho3);

/* torques tau[E][S][7] along each edge at its duration T[e] */
void or_torque_dump(const or_arm* arm, int E, const float* s0, const float* s1,
                    const float* T, int S, double* tau);

/* brute-force kNN over nodes [first, N) of tree [N][16]; output sorted by
 * (d2, index); missing slots get idx -1 / d2 +inf */
void or_knn(const float* tree, int N, int first, const float* queries, int B, int k,
            double w_vel, int* idx, double* d2);

/* forward kinematics: world rotation R[f] and origin o[f] of frames 1..7 (f=0..6)
 * and the end-effector frame (f=7) */
void or_fk(const or_arm* arm, const double* q, double R[8][3][3], double o[8][3]);
void or_blade(const or_arm* arm, const double* q, double b0[3], double b1[3]);
/* geometric 6 x dof Jacobian (row-major [6][7]) of the point p (world) */
void or_jacobian_point(const or_arm* arm, const double* q, const double* p, double J[6][7]);

/* Philox4x32-10 (Salmon et al., SC'11) */
void or_philox4x32(const unsigned int ctr[4], const unsigned int key[2], unsigned int out[4]);

/* why phi(z) is undefined (the first failing condition), or OR_CHART_OK */
enum { OR_CHART_OK = 0, OR_CHART_SPEED = 1, OR_CHART_IK = 2, OR_CHART_BOX = 3,
       OR_CHART_SINGULAR = 4, OR_CHART_TAPER = 5 };
/* goal chart phi(z): out_state[16] (q, pad, qd, pad), T_req, |v_rel|, v_b[3];
 * returns 1 if defined, 0 otherwise; reason (may be NULL) gets an OR_CHART_* code */
int or_goal_chart(const or_arm* arm, const or_problem* pr, const double* z,
                  double* out_state, double* T_req, double* vrel, double* vb, int* reason);

/* samplers drawing Philox uniforms with counter (index, iter, problem, stream) */
void or_sample_uniform(const or_arm* arm, unsigned long long seed, int iter, int problem,
                       int first_index, int n, double vel_frac, double* states);
void or_sample_goals(const or_arm* arm, const or_problem* pr, unsigned long long seed,
                     int iter, int problem, int first_index, int n, double* states,
                     double* T_req, double* vrel, int* valid, int* reason);

/* Eq. (objective) of a rendezvous at arrival T with relative speed vrel and
 * peak velocity fraction nu */
double or_objective(const or_problem* pr, double T, double vrel, double nu);

/* Eq. (reach): earliest T on a G-point grid of [t_enter, t_fall] that node
 * (q, t_n) can reach; returns -1 if none.  Writes T_n. */
int or_reach_time(const or_arm* arm, const or_problem* pr, const double* q, double t_n,
                  int G, double* T_n);

/* minimum clearance of the arm's link capsules to obstacle spheres [n_obs][4]
 * along an edge at duration T over S collocation points (incl. both ends) */
double or_edge_clearance(const or_arm* arm, const float* s0, const float* s1, double T,
                         int S, const float* obs, int n_obs);

/* Eq. (controller) for B instances: state/goal [B][16] (q, pad, qd, pad),
 * horizon T [B], tau_prev [B][7] and rate [7] (both NULL: no slew limit),
 * control period dt; outputs tau, qdd [B][7] and flags [B] (bit 0 acc,
 * 1 torque, 2 power, 3 slew clipped; 0x80 invalid input). */
void or_controller_torque(const or_arm* arm, int B, const float* state, const float* goal,
                          const float* T, const float* tau_prev, double dt, const double* rate,
                          double* tau, double* qdd, unsigned char* flags);

/* Full-resolution recheck: ratios over S samples, clearance over S_clear
 * points (obs [n_obs][4]), ok per edge at its own duration T[e]. */
void or_check_edges(const or_arm* arm, int E, const float* s0, const float* s1, const float* T,
                    int S, int S_clear, const float* obs, int n_obs, double margin, double* rho3,
                    double* clearance, unsigned char* ok);

/* The goal density p_theta: C (<= 4) diagonal Gaussians over Z = [0, 1]^9
 * with weights pi (summing to 1) mixed with the uniform component of weight
 * w_u; single-precision parameters, as the planner keeps them. */
typedef struct {
  int C;
  float w_u;
  float pi[4];
  float mu[4][9];
  float sd[4][9];
} or_density;

/* chart parameters z [9] of goal candidate (seed, index, iter, problem) */
void or_density_z(const or_density* th, unsigned long long seed, int index, int iter, int problem,
                  double* z);
/* goal candidates drawn from p_theta and decoded (as or_sample_goals; zs
 * [n][9] may be NULL) */
void or_sample_goals_density(const or_arm* arm, const or_problem* pr, const or_density* th,
                             unsigned long long seed, int iter, int problem, int first_index,
                             int n, double* states, double* T_req, double* vrel, int* valid,
                             double* zs);
/* free candidates from the chord sampler: goals [n_goals][16] are the
 * round's valid decoded goals in candidate order, q0 [7] the root */
void or_sample_chord(const or_arm* arm, unsigned long long seed, int iter, int problem,
                     int first_index, int n, double vel_frac, const double* q0,
                     const double* goals, int n_goals, float w_chord, double sigma,
                     double* states);

#ifdef __cplusplus
}
#endif
#endif
