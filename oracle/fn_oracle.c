/*
 * FP64 CPU oracle for the edge-timing planner of "Becoming a Fruit Ninja"
 * (arxiv 2609.22608).  TEST INFRASTRUCTURE ONLY (see fn_oracle.h): used by the
 * tests, the smoke check and the benchmark's CPU-baseline leg, never by the
 * product path.  Plain loops, double precision, the paper's definitions in
 * the paper's order.
 */
#include "fn_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */
static void cross3(const double* a, const double* b, double* c) {
  double x = a[1] * b[2] - a[2] * b[1];
  double y = a[2] * b[0] - a[0] * b[2];
  double z = a[0] * b[1] - a[1] * b[0];
  c[0] = x; c[1] = y; c[2] = z;
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double* a) { return sqrt(dot3(a, a)); }
/* y = R x  (R row-major 3x3) */
static void matvec(double R[3][3], const double* x, double* y) {
  double t[3];
  for (int i = 0; i < 3; ++i) t[i] = R[i][0] * x[0] + R[i][1] * x[1] + R[i][2] * x[2];
  y[0] = t[0]; y[1] = t[1]; y[2] = t[2];
}
/* y = R^T x */
static void matTvec(double R[3][3], const double* x, double* y) {
  double t[3];
  for (int i = 0; i < 3; ++i) t[i] = R[0][i] * x[0] + R[1][i] * x[1] + R[2][i] * x[2];
  y[0] = t[0]; y[1] = t[1]; y[2] = t[2];
}
static void matmul(double A[3][3], double B[3][3], double C[3][3]) {
  double T[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) T[i][j] = A[i][0] * B[0][j] + A[i][1] * B[1][j] + A[i][2] * B[2][j];
  memcpy(C, T, sizeof(T));
}

/* Modified DH link transform of joint j (Craig):
 *   T_{j-1,j} = Rx(alpha_j) Tx(a_j) Rz(theta0_j + q_j) Tz(d_j)
 * R maps frame-j vectors into frame j-1; p is frame j's origin in frame j-1. */
static void link_transform(const or_arm* arm, int j, double q, double R[3][3], double p[3]) {
  double th = q + arm->theta0[j];
  double ct = cos(th), st = sin(th);
  double ca = cos(arm->alpha[j]), sa = sin(arm->alpha[j]);
  R[0][0] = ct;      R[0][1] = -st;     R[0][2] = 0.0;
  R[1][0] = st * ca; R[1][1] = ct * ca; R[1][2] = -sa;
  R[2][0] = st * sa; R[2][1] = ct * sa; R[2][2] = ca;
  p[0] = arm->a[j];
  p[1] = -sa * arm->d[j];
  p[2] = ca * arm->d[j];
}

/* ------------------------------------------------------------------ */
/* Def. "Cubic edge", Eq. (cubic)                                       */
/*   sigma(t) = q0 + qd0 t + (3 d1/T^2 - d2/T) t^2 + (d2/T^2 - 2 d1/T^3) t^3 */
/*   d1 = q1 - q0 - qd0 T,  d2 = qd1 - qd0                               */
/* ------------------------------------------------------------------ */
void or_cubic(int n, const double* q0, const double* qd0, const double* q1,
              const double* qd1, double T, double t, double* s, double* sd, double* sdd) {
  for (int i = 0; i < n; ++i) {
    double d1 = q1[i] - q0[i] - qd0[i] * T;
    double d2 = qd1[i] - qd0[i];
    double c2 = 3.0 * d1 / (T * T) - d2 / T;
    double c3 = d2 / (T * T) - 2.0 * d1 / (T * T * T);
    s[i] = q0[i] + qd0[i] * t + c2 * t * t + c3 * t * t * t;
    sd[i] = qd0[i] + 2.0 * c2 * t + 3.0 * c3 * t * t;
    sdd[i] = 2.0 * c2 + 6.0 * c3 * t;
  }
}

/* ------------------------------------------------------------------ */
/* Eq. (torque): recursive Newton-Euler with the base accelerating at   */
/* -gravity (Craig's outward/inward iterations, modified DH).           */
/* ------------------------------------------------------------------ */
void or_rnea(const or_arm* arm, const double* q, const double* qd, const double* qdd,
             double* tau) {
  int n = arm->dof;
  double R[7][3][3], p[7][3];
  double w[7][3], wd[7][3], vd[7][3], F[7][3], N[7][3];
  double w_prev[3] = {0, 0, 0}, wd_prev[3] = {0, 0, 0};
  double vd_prev[3] = {-arm->gravity[0], -arm->gravity[1], -arm->gravity[2]};
  for (int j = 0; j < n; ++j) {
    link_transform(arm, j, q[j], R[j], p[j]);
    double z[3] = {0, 0, 1};
    double Rw[3], Rwd[3], tmp[3], tmp2[3];
    matTvec(R[j], w_prev, Rw);
    matTvec(R[j], wd_prev, Rwd);
    /* omega_j = R^T omega_{j-1} + qd_j z */
    for (int k = 0; k < 3; ++k) w[j][k] = Rw[k] + qd[j] * z[k];
    /* omegadot_j = R^T omegadot_{j-1} + (R^T omega_{j-1}) x (qd_j z) + qdd_j z */
    double qz[3] = {0, 0, qd[j]};
    cross3(Rw, qz, tmp);
    for (int k = 0; k < 3; ++k) wd[j][k] = Rwd[k] + tmp[k] + qdd[j] * z[k];
    /* vdot_j = R^T (omegadot_{j-1} x p + omega_{j-1} x (omega_{j-1} x p) + vdot_{j-1}) */
    double a1[3], a2[3], a3[3];
    cross3(wd_prev, p[j], a1);
    cross3(w_prev, p[j], tmp);
    cross3(w_prev, tmp, a2);
    for (int k = 0; k < 3; ++k) a3[k] = a1[k] + a2[k] + vd_prev[k];
    matTvec(R[j], a3, vd[j]);
    /* COM acceleration, F = m vdot_c, N = I omegadot + omega x I omega */
    double vc[3];
    cross3(wd[j], arm->com[j], a1);
    cross3(w[j], arm->com[j], tmp);
    cross3(w[j], tmp, a2);
    for (int k = 0; k < 3; ++k) vc[k] = a1[k] + a2[k] + vd[j][k];
    for (int k = 0; k < 3; ++k) F[j][k] = arm->mass[j] * vc[k];
    double Iw[3], Iwd[3];
    for (int k = 0; k < 3; ++k) { Iw[k] = arm->inertia[j][k] * w[j][k]; Iwd[k] = arm->inertia[j][k] * wd[j][k]; }
    cross3(w[j], Iw, tmp2);
    for (int k = 0; k < 3; ++k) N[j][k] = Iwd[k] + tmp2[k];
    for (int k = 0; k < 3; ++k) { w_prev[k] = w[j][k]; wd_prev[k] = wd[j][k]; vd_prev[k] = vd[j][k]; }
  }
  /* inward: f_j = R_{j+1} f_{j+1} + F_j;
   *         n_j = N_j + R_{j+1} n_{j+1} + c_j x F_j + p_{j+1} x (R_{j+1} f_{j+1}) */
  double f_next[3] = {0, 0, 0}, n_next[3] = {0, 0, 0};
  for (int j = n - 1; j >= 0; --j) {
    double Rf[3] = {0, 0, 0}, Rn[3] = {0, 0, 0}, pxRf[3] = {0, 0, 0};
    if (j + 1 < n) {
      matvec(R[j + 1], f_next, Rf);
      matvec(R[j + 1], n_next, Rn);
      cross3(p[j + 1], Rf, pxRf);
    }
    double cxF[3];
    cross3(arm->com[j], F[j], cxF);
    double f[3], nn[3];
    for (int k = 0; k < 3; ++k) {
      f[k] = Rf[k] + F[j][k];
      nn[k] = N[j][k] + Rn[k] + cxF[k] + pxRf[k];
    }
    tau[j] = nn[2];
    memcpy(f_next, f, sizeof(f));
    memcpy(n_next, nn, sizeof(nn));
  }
}

/* Eq. (friction): psi1/(1+exp(-psi2 (qd + psi3))) - psi1/(1+exp(-psi2 psi3)) */
double or_friction(const double* psi, double qd) {
  return psi[0] / (1.0 + exp(-psi[1] * (qd + psi[2]))) - psi[0] / (1.0 + exp(-psi[1] * psi[2]));
}

/* Eq. (torque): [M qdd + c + g]_i + I_m,i qdd_i + tau_f,i(qd_i) */
void or_torque(const or_arm* arm, const double* q, const double* qd, const double* qdd,
               double* tau) {
  or_rnea(arm, q, qd, qdd, tau);
  for (int j = 0; j < arm->dof; ++j)
    tau[j] += arm->armature[j] * qdd[j] + or_friction(arm->fric[j], qd[j]);
}

/* Position-dependent velocity bound (Def. 1 names it; the paper gives no
 * formula).  Reading: a deceleration taper to the joint box,
 *   qdbar(q) = min(qd_max, sqrt(2 a max(0, min(q - q_lo, q_hi - q)))). */
double or_taper(const or_arm* arm, int j, double q) {
  double m = fmin(q - arm->q_lo[j], arm->q_hi[j] - q);
  if (m < 0.0) m = 0.0;
  return fmin(arm->qd_max[j], sqrt(2.0 * arm->taper_a[j] * m));
}

static int state_finite(const float* s, int n) {
  for (int i = 0; i < n; ++i)
    if (!isfinite(s[i]) || !isfinite(s[8 + i])) return 0;
  return 1;
}

static void unpack(const float* s, int n, double* q, double* qd) {
  for (int i = 0; i < n; ++i) { q[i] = (double)s[i]; qd[i] = (double)s[8 + i]; }
}

/* rho_v: the velocity of a cubic is quadratic in t, so its extremum over
 * [0, T] is at an end or at the stationary point -b/(2c).  Reading: each
 * joint's ratio is |sigma_dot| over the taper evaluated at the position the
 * joint has at that same time; zero taper with nonzero speed gives +inf. */
static double rho_v_of(const or_arm* arm, const double* q0, const double* qd0,
                       const double* q1, const double* qd1, double T) {
  int n = arm->dof;
  double rv = 0.0;
  for (int i = 0; i < n; ++i) {
    double d1 = q1[i] - q0[i] - qd0[i] * T;
    double d2 = qd1[i] - qd0[i];
    double c2 = 3.0 * d1 / (T * T) - d2 / T;
    double c3 = d2 / (T * T) - 2.0 * d1 / (T * T * T);
    double cand[3];
    int nc = 0;
    cand[nc++] = 0.0;
    cand[nc++] = T;
    /* sigma_dot = qd0 + 2 c2 t + 3 c3 t^2; stationary at t = -2c2/(6c3) */
    if (c3 != 0.0) {
      double ts = -(2.0 * c2) / (2.0 * 3.0 * c3);
      if (ts > 0.0 && ts < T) cand[nc++] = ts;
    }
    for (int c = 0; c < nc; ++c) {
      double t = cand[c];
      double pos = q0[i] + qd0[i] * t + c2 * t * t + c3 * t * t * t;
      double vel = qd0[i] + 2.0 * c2 * t + 3.0 * c3 * t * t;
      double bound = or_taper(arm, i, pos);
      double r;
      if (bound > 0.0) r = fabs(vel) / bound;
      else r = (vel != 0.0) ? INFINITY : 0.0;
      if (r > rv) rv = r;
    }
  }
  return rv;
}

/* Def. "Feasibility Check", Eq. (rho).  Reading: the S equally spaced times
 * include both ends, t_s = s T / (S - 1). */
static void rho_tp(const or_arm* arm, const double* q0, const double* qd0, const double* q1,
                   const double* qd1, double T, int S, double* rt, double* rp) {
  int n = arm->dof;
  double rho_tau = 0.0, rho_p = 0.0;
  for (int s = 0; s < S; ++s) {
    double t = (double)s * T / (double)(S - 1);
    double q[7], qd[7], qdd[7], tau[7];
    or_cubic(n, q0, qd0, q1, qd1, T, t, q, qd, qdd);
    or_torque(arm, q, qd, qdd, tau);
    double pw = 0.0;
    for (int i = 0; i < n; ++i) {
      double r = fabs(tau[i]) / arm->tau_max[i];
      if (r > rho_tau) rho_tau = r;
      pw += tau[i] * qd[i];
    }
    double r = fabs(pw) / arm->w_max;
    if (r > rho_p) rho_p = r;
  }
  *rt = rho_tau;
  *rp = rho_p;
}

void or_rho(const or_arm* arm, const float* s0, const float* s1, double T, int S, double* rho3) {
  double q0[7], qd0[7], q1[7], qd1[7];
  unpack(s0, arm->dof, q0, qd0);
  unpack(s1, arm->dof, q1, qd1);
  rho_tp(arm, q0, qd0, q1, qd1, T, S, &rho3[0], &rho3[1]);
  rho3[2] = rho_v_of(arm, q0, qd0, q1, qd1, T);
}

void or_rho_batch(const or_arm* arm, int E, const float* s0, const float* s1,
                  const double* T, int S, double* rho3) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int e = 0; e < E; ++e) or_rho(arm, s0 + 16 * (size_t)e, s1 + 16 * (size_t)e, T[e], S, rho3 + 3 * (size_t)e);
}

/* Def. "Minimum feasible time" on a grid: k* = min{k : rho_tau(T_k) <= 1 and
 * rho_P(T_k) <= 1}, scanning every grid index in ascending order (no
 * monotonicity is assumed), then rho_v checked once at T_{k*}.  With a cap,
 * only T_k <= T_cap[e] are admissible (the incumbent bound of Alg. 1). */
void or_time_edges(const or_arm* arm, int E, const float* s0, const float* s1,
                   const float* T_grid, int K, int S, int mode, const float* T_fixed,
                   const float* T_cap, int* k_star, float* T_star, double* rho3,
                   unsigned char* ok) {
  int n = arm->dof;
#pragma omp parallel for schedule(dynamic, 1)
  for (int e = 0; e < E; ++e) {
    const float* a = s0 + 16 * (size_t)e;
    const float* b = s1 + 16 * (size_t)e;
    double* r3 = rho3 + 3 * (size_t)e;
    k_star[e] = -1;
    T_star[e] = INFINITY;
    r3[0] = r3[1] = r3[2] = NAN;
    ok[e] = 0;
    if (!state_finite(a, n) || !state_finite(b, n)) { k_star[e] = -2; T_star[e] = NAN; continue; }
    double q0[7], qd0[7], q1[7], qd1[7];
    unpack(a, n, q0, qd0);
    unpack(b, n, q1, qd1);
    if (mode == 1) {
      float Tf = T_fixed[e];
      if (!(isfinite(Tf) && Tf > 0.0f)) { k_star[e] = -2; T_star[e] = NAN; continue; }
      double T = (double)Tf;
      rho_tp(arm, q0, qd0, q1, qd1, T, S, &r3[0], &r3[1]);
      r3[2] = rho_v_of(arm, q0, qd0, q1, qd1, T);
      T_star[e] = Tf;
      k_star[e] = (r3[0] <= 1.0 && r3[1] <= 1.0) ? 0 : -1;
      ok[e] = (k_star[e] == 0 && r3[2] <= 1.0) ? 1 : 0;
      continue;
    }
    for (int k = 0; k < K; ++k) {
      if (T_cap && !(T_grid[k] <= T_cap[e])) break;
      double rt, rp;
      rho_tp(arm, q0, qd0, q1, qd1, (double)T_grid[k], S, &rt, &rp);
      if (rt <= 1.0 && rp <= 1.0) {
        k_star[e] = k;
        T_star[e] = T_grid[k];
        r3[0] = rt;
        r3[1] = rp;
        r3[2] = rho_v_of(arm, q0, qd0, q1, qd1, (double)T_grid[k]);
        ok[e] = r3[2] <= 1.0 ? 1 : 0;
        break;
      }
    }
  }
}

/* Def. "Minimum feasible time" refined by the N-ary search that the paper
 * describes after it: the bracket is split into N equal slots, every slot
 * boundary is checked, and the slot where the check first passes is split
 * again, until the bracket is no wider than eps.  Readings:
 *   - the first bracket is the grid cell of the grid scan's k*:
 *     (T_{k*-1}, T_{k*}], with T_{-1} = 0; its upper end is feasible;
 *   - a round checks the N - 1 interior points t_j = a + j w (w = (b - a)/N)
 *     in ascending order and keeps [t_{j-1}, t_j] for the first feasible t_j
 *     (or [t_{N-1}, b] if none is); like the grid scan, it assumes no
 *     monotonicity;
 *   - N = 32; the points are formed in single precision (w = (b - a) * 2^-5,
 *     t_j = fmaf(j, w, a)) so that both implementations check the same
 *     durations; the checks themselves are in double precision here;
 *   - rounds run while b - a > eps (single precision), at most max_rounds;
 *   - rho_v is checked once, at the refined T* = b.
 * margin[e] (may be NULL): the smallest |max(rho_tau, rho_P) - 1| over every
 * duration this routine checked for the edge (grid and rounds), +inf if none. */
#define OR_NARY_N 32
void or_time_edges_nary(const or_arm* arm, int E, const float* s0, const float* s1,
                        const float* T_grid, int K, int S, const float* T_cap, float eps,
                        int max_rounds, int* k_star, float* T_star, float* T_lo, double* rho3,
                        unsigned char* ok, int* rounds, double* margin) {
  int n = arm->dof;
#pragma omp parallel for schedule(dynamic, 1)
  for (int e = 0; e < E; ++e) {
    const float* sa = s0 + 16 * (size_t)e;
    const float* sb = s1 + 16 * (size_t)e;
    double* r3 = rho3 + 3 * (size_t)e;
    double mg = INFINITY;
    k_star[e] = -1;
    T_star[e] = INFINITY;
    T_lo[e] = NAN;
    rounds[e] = 0;
    r3[0] = r3[1] = r3[2] = NAN;
    ok[e] = 0;
    if (!state_finite(sa, n) || !state_finite(sb, n)) {
      k_star[e] = -2;
      T_star[e] = NAN;
      if (margin) margin[e] = mg;
      continue;
    }
    double q0[7], qd0[7], q1[7], qd1[7];
    unpack(sa, n, q0, qd0);
    unpack(sb, n, q1, qd1);
    double rt = NAN, rp = NAN;
    for (int k = 0; k < K; ++k) {
      if (T_cap && !(T_grid[k] <= T_cap[e])) break;
      double t_rt, t_rp;
      rho_tp(arm, q0, qd0, q1, qd1, (double)T_grid[k], S, &t_rt, &t_rp);
      double m = fmax(t_rt, t_rp);
      if (fabs(m - 1.0) < mg) mg = fabs(m - 1.0);
      if (t_rt <= 1.0 && t_rp <= 1.0) {
        k_star[e] = k;
        rt = t_rt;
        rp = t_rp;
        break;
      }
    }
    if (k_star[e] < 0) {
      if (margin) margin[e] = mg;
      continue;
    }
    float a = k_star[e] > 0 ? T_grid[k_star[e] - 1] : 0.0f;
    float b = T_grid[k_star[e]];
    int r = 0;
    while (r < max_rounds && (b - a) > eps) {
      float w = (b - a) * 0.03125f;
      int js = OR_NARY_N;
      for (int j = 1; j < OR_NARY_N; ++j) {
        float t = fmaf((float)j, w, a);
        double t_rt, t_rp;
        rho_tp(arm, q0, qd0, q1, qd1, (double)t, S, &t_rt, &t_rp);
        double m = fmax(t_rt, t_rp);
        if (fabs(m - 1.0) < mg) mg = fabs(m - 1.0);
        if (t_rt <= 1.0 && t_rp <= 1.0) {
          js = j;
          rt = t_rt;
          rp = t_rp;
          break;
        }
      }
      float lo = js == 1 ? a : fmaf((float)(js - 1), w, a);
      float hi = js == OR_NARY_N ? b : fmaf((float)js, w, a);
      a = lo;
      b = hi;
      ++r;
    }
    T_star[e] = b;
    T_lo[e] = a;
    rounds[e] = r;
    r3[0] = rt;
    r3[1] = rp;
    r3[2] = rho_v_of(arm, q0, qd0, q1, qd1, (double)b);
    ok[e] = r3[2] <= 1.0 ? 1 : 0;
    if (margin) margin[e] = mg;
  }
}

void or_torque_dump(const or_arm* arm, int E, const float* s0, const float* s1,
                    const float* T, int S, double* tau) {
  int n = arm->dof;
#pragma omp parallel for schedule(dynamic, 4)
  for (int e = 0; e < E; ++e) {
    double q0[7], qd0[7], q1[7], qd1[7];
    unpack(s0 + 16 * (size_t)e, n, q0, qd0);
    unpack(s1 + 16 * (size_t)e, n, q1, qd1);
    double Te = (double)T[e];
    for (int s = 0; s < S; ++s) {
      double t = (double)s * Te / (double)(S - 1);
      double q[7], qd[7], qdd[7], tq[7];
      or_cubic(n, q0, qd0, q1, qd1, Te, t, q, qd, qdd);
      or_torque(arm, q, qd, qdd, tq);
      for (int i = 0; i < 7; ++i) tau[((size_t)e * S + s) * 7 + i] = i < n ? tq[i] : 0.0;
    }
  }
}

/* ------------------------------------------------------------------ */
/* Parents (Sec. IV-E): brute-force scan of the tree, velocity-weighted  */
/* squared joint distance (the metric is a reading; the paper gives none). */
/* ------------------------------------------------------------------ */
typedef struct { double d; int i; } dpair;
static int dpair_cmp(const void* x, const void* y) {
  const dpair* a = (const dpair*)x;
  const dpair* b = (const dpair*)y;
  if (a->d < b->d) return -1;
  if (a->d > b->d) return 1;
  return (a->i > b->i) - (a->i < b->i);
}

void or_knn(const float* tree, int N, int first, const float* queries, int B, int k,
            double w_vel, int* idx, double* d2) {
#pragma omp parallel
  {
    dpair* buf = (dpair*)malloc(sizeof(dpair) * (size_t)(N > 0 ? N : 1));
#pragma omp for schedule(dynamic, 8)
    for (int b = 0; b < B; ++b) {
      const float* qv = queries + 16 * (size_t)b;
      int m = 0;
      for (int n = first; n < N; ++n) {
        const float* t = tree + 16 * (size_t)n;
        double dq = 0.0, dv = 0.0;
        for (int j = 0; j < 7; ++j) {
          double a = (double)qv[j] - (double)t[j];
          double c = (double)qv[8 + j] - (double)t[8 + j];
          dq += a * a;
          dv += c * c;
        }
        buf[m].d = dq + w_vel * dv;
        buf[m].i = n;
        ++m;
      }
      qsort(buf, (size_t)m, sizeof(dpair), dpair_cmp);
      for (int j = 0; j < k; ++j) {
        if (j < m) { idx[(size_t)b * k + j] = buf[j].i; d2[(size_t)b * k + j] = buf[j].d; }
        else { idx[(size_t)b * k + j] = -1; d2[(size_t)b * k + j] = INFINITY; }
      }
    }
    free(buf);
  }
}

/* ------------------------------------------------------------------ */
/* Forward kinematics and Jacobians (used by the goal chart, clearance  */
/* and pruning).                                                       */
/* ------------------------------------------------------------------ */
void or_fk(const or_arm* arm, const double* q, double R[8][3][3], double o[8][3]) {
  double Rc[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  double oc[3] = {0, 0, 0};
  int n = arm->dof;
  for (int j = 0; j < 7; ++j) {
    if (j < n) {
      double Rj[3][3], pj[3], wp[3];
      link_transform(arm, j, q[j], Rj, pj);
      matvec(Rc, pj, wp);
      for (int k = 0; k < 3; ++k) oc[k] += wp[k];
      matmul(Rc, Rj, Rc);
    }
    memcpy(R[j], Rc, sizeof(Rc));
    memcpy(o[j], oc, sizeof(oc));
  }
  /* end-effector frame: frame 7 (or the last frame) moved flange_d along its z */
  memcpy(R[7], Rc, sizeof(Rc));
  for (int k = 0; k < 3; ++k) o[7][k] = oc[k] + arm->flange_d * Rc[k][2];
}

void or_blade(const or_arm* arm, const double* q, double b0[3], double b1[3]) {
  double R[8][3][3], o[8][3];
  or_fk(arm, q, R, o);
  double w[3], ax[3];
  matvec(R[7], arm->blade_base, w);
  matvec(R[7], arm->blade_axis, ax);
  for (int k = 0; k < 3; ++k) {
    b0[k] = o[7][k] + w[k];
    b1[k] = b0[k] + arm->blade_len * ax[k];
  }
}

void or_jacobian_point(const or_arm* arm, const double* q, const double* p, double J[6][7]) {
  double R[8][3][3], o[8][3];
  or_fk(arm, q, R, o);
  for (int j = 0; j < 7; ++j) {
    double z[3] = {R[j][0][2], R[j][1][2], R[j][2][2]};
    double r[3] = {p[0] - o[j][0], p[1] - o[j][1], p[2] - o[j][2]};
    double v[3];
    cross3(z, r, v);
    int used = j < arm->dof;
    for (int k = 0; k < 3; ++k) {
      J[k][j] = used ? v[k] : 0.0;
      J[3 + k][j] = used ? z[k] : 0.0;
    }
  }
}

/* Solve A x = b (n <= 6) by Gaussian elimination with partial pivoting.
 * Returns 0 if a pivot is (numerically) zero. */
static int solve_gepp(int n, double A[6][6], double* b, double* x) {
  double M[6][7];
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) M[i][j] = A[i][j];
    M[i][n] = b[i];
  }
  double scale = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) scale = fmax(scale, fabs(A[i][j]));
  for (int c = 0; c < n; ++c) {
    int pr = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(M[r][c]) > fabs(M[pr][c])) pr = r;
    if (!(fabs(M[pr][c]) > 1e-12 * scale)) return 0;
    if (pr != c)
      for (int j = 0; j <= n; ++j) { double t = M[c][j]; M[c][j] = M[pr][j]; M[pr][j] = t; }
    for (int r = c + 1; r < n; ++r) {
      double f = M[r][c] / M[c][c];
      for (int j = c; j <= n; ++j) M[r][j] -= f * M[c][j];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = M[i][n];
    for (int j = i + 1; j < n; ++j) s -= M[i][j] * x[j];
    x[i] = s / M[i][i];
  }
  return 1;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10, from the definition in Salmon, Moraes, Dror, Shaw,    */
/* "Parallel random numbers: as easy as 1, 2, 3" (SC'11).               */
/* ------------------------------------------------------------------ */
void or_philox4x32(const unsigned int ctr[4], const unsigned int key[2], unsigned int out[4]) {
  unsigned int c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  unsigned int k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
    unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
    unsigned int hi0 = (unsigned int)(p0 >> 32), lo0 = (unsigned int)p0;
    unsigned int hi1 = (unsigned int)(p1 >> 32), lo1 = (unsigned int)p1;
    unsigned int n0 = hi1 ^ c1 ^ k0;
    unsigned int n1 = lo1;
    unsigned int n2 = hi0 ^ c3 ^ k1;
    unsigned int n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 24-bit uniform in [0, 1): exact in both float and double */
static double u01(unsigned int x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

static void philox_uniforms(unsigned long long seed, int index, int iter, int problem,
                            int stream, double u[4]) {
  unsigned int ctr[4] = {(unsigned int)index, (unsigned int)iter, (unsigned int)problem,
                         (unsigned int)stream};
  unsigned int key[2] = {(unsigned int)(seed & 0xffffffffu), (unsigned int)(seed >> 32)};
  unsigned int out[4];
  or_philox4x32(ctr, key, out);
  for (int i = 0; i < 4; ++i) u[i] = u01(out[i]);
}

/* Uniform free candidates: q_j = q_lo + u (q_hi - q_lo), qd_j uniform in
 * +-vel_frac * qdbar_j(q_j).  Uniforms: streams 0..3 of the candidate's counter. */
void or_sample_uniform(const or_arm* arm, unsigned long long seed, int iter, int problem,
                       int first_index, int n, double vel_frac, double* states) {
  for (int c = 0; c < n; ++c) {
    double u[16];
    for (int s = 0; s < 4; ++s) philox_uniforms(seed, first_index + c, iter, problem, s, u + 4 * s);
    double* st = states + 16 * (size_t)c;
    for (int i = 0; i < 16; ++i) st[i] = 0.0;
    for (int j = 0; j < 7; ++j) {
      double qj = arm->q_lo[j] + u[j] * (arm->q_hi[j] - arm->q_lo[j]);
      double vb = vel_frac * or_taper(arm, j, qj);
      st[j] = qj;
      st[8 + j] = (2.0 * u[7 + j] - 1.0) * vb;
    }
  }
}

/* unit vector pair (e1, e2) completing u to a right-handed frame */
static void complete_basis(const double* u, double* e1, double* e2) {
  double h[3] = {0, 0, 1};
  if (!(fabs(u[2]) < 0.9)) { h[0] = 1; h[1] = 0; h[2] = 0; }
  cross3(h, u, e1);
  double l = norm3(e1);
  for (int k = 0; k < 3; ++k) e1[k] /= l;
  cross3(u, e1, e2);
}

#define OR_IK_ITERS 24
#define OR_IK_LAMBDA 5e-2
#define OR_IK_POS_TOL 1e-4
#define OR_IK_ROT_TOL 1e-3
#define OR_IK_STARTS 4

/* One damped-least-squares IK run on joints 1-6 with q7 fixed.  Start `st`
 * is the box centre shifted by a fixed fraction of each half-range (four
 * postures: centre, the shoulder/elbow/wrist pattern +-(0,.5,0,-.5,0,.5),
 * and (0,-.5,0,-.5,0,-.5)), with joint 1 turned towards the target's
 * azimuth; each iterate is projected onto the joint box.  Returns 1 when the
 * pose residuals are under tolerance and the rotation error is under 90
 * degrees (trace > 1; the cross-product residual also vanishes at a half
 * turn). */
static int ik_solve(const or_arm* arm, double Rg[3][3], const double* pg, double z6, int st,
                    double* q) {
  static const double pattern[2][6] = {{0.0, 0.5, 0.0, -0.5, 0.0, 0.5},
                                       {0.0, -0.5, 0.0, -0.5, 0.0, -0.5}};
  double sgn = st == 0 ? 0.0 : (st == 2 ? -1.0 : 1.0);
  const double* pat = pattern[st == 3 ? 1 : 0];
  for (int j = 0; j < 7; ++j) {
    double c = 0.5 * (arm->q_lo[j] + arm->q_hi[j]);
    double h = 0.5 * (arm->q_hi[j] - arm->q_lo[j]);
    q[j] = j < 6 ? c + sgn * pat[j] * h : c;
  }
  q[6] = arm->q_lo[6] + z6 * (arm->q_hi[6] - arm->q_lo[6]);
  q[0] = fmin(fmax(atan2(pg[1], pg[0]), arm->q_lo[0]), arm->q_hi[0]);
  double ep[3], er[3];
  double R[8][3][3], o[8][3];
  for (int it = 0; it <= OR_IK_ITERS; ++it) {
    or_fk(arm, q, R, o);
    for (int k = 0; k < 3; ++k) ep[k] = pg[k] - o[7][k];
    er[0] = er[1] = er[2] = 0.0;
    for (int col = 0; col < 3; ++col) {
      double rc[3] = {R[7][0][col], R[7][1][col], R[7][2][col]};
      double rg[3] = {Rg[0][col], Rg[1][col], Rg[2][col]};
      double x[3];
      cross3(rc, rg, x);
      for (int k = 0; k < 3; ++k) er[k] += 0.5 * x[k];
    }
    if (it == OR_IK_ITERS) break;
    double J[6][7];
    or_jacobian_point(arm, q, o[7], J);
    double A[6][6];
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) {
        double sacc = 0.0;
        for (int m = 0; m < 6; ++m) sacc += J[i][m] * J[j][m];
        A[i][j] = sacc + (i == j ? OR_IK_LAMBDA * OR_IK_LAMBDA : 0.0);
      }
    double e[6] = {ep[0], ep[1], ep[2], er[0], er[1], er[2]};
    double y[6];
    if (!solve_gepp(6, A, e, y)) return 0;
    for (int m = 0; m < 6; ++m) {
      double dq = 0.0;
      for (int i = 0; i < 6; ++i) dq += J[i][m] * y[i];
      q[m] = fmin(fmax(q[m] + dq, arm->q_lo[m]), arm->q_hi[m]);
    }
  }
  if (!(norm3(ep) < OR_IK_POS_TOL && norm3(er) < OR_IK_ROT_TOL)) return 0;
  double tr = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) tr += Rg[k][i] * R[7][k][i];
  return tr > 1.0;
}

/* Goal chart phi(z) (Def. "Goal chart" and the decoding after it).
 * Readings (the paper fixes the roles of z, not the formulas):
 *  z0 -> T = t_enter + z0 (t_fall - t_enter); contact c = x(T + t_offset)
 *  z1, z2 -> approach direction d in the cone of half-angle acos(a_min) about
 *            -xdot(T): polar angle acos(1 - z1 (1 - a_min)), azimuth 2 pi z2
 *  z8 -> closing speed s = 0.5 + 1.5 z8; blade velocity v_b = s d;
 *        v_rel = v_b - xdot(T); undefined if |v_rel| < v_min
 *  z5, z4 -> cutting direction n_b = v_rel/|v_rel| tilted by z5 acos(a_min)
 *            towards the roll direction 2 pi z4 (so alignment >= a_min)
 *  z3 -> blade axis: spin 2 pi z3 about n_b
 *  z7 -> contact at arclength z7 * blade_len along the edge
 *  z6 -> q7 = q7_lo + z6 (q7_hi - q7_lo)
 *  q_g by damped least squares on joints 1-6 (the paper's closed-form FR3 IK
 *  does not apply to a synthetic arm): up to four starts (ik_solve), 24
 *  iterations each, lambda = 0.05; the first start that converges wins
 *  qd_g = J_p^+ v_b with J_p the 3x7 Jacobian of the contact point's linear
 *  velocity, J_p^+ = J_p^T (J_p J_p^T)^-1: v_ee is a linear velocity, so the
 *  minimum-norm joint velocity that gives the blade v_b at the contact;
 *  undefined if any |qd_g,i| exceeds the taper at q_g.
 * Returns 1 where phi is defined, else 0; `reason` (may be NULL) receives
 * OR_CHART_OK or the first condition that left phi undefined. */
int or_goal_chart(const or_arm* arm, const or_problem* pr, const double* z,
                  double* out_state, double* T_req, double* vrel_out, double* vb_out,
                  int* reason) {
  int why_dummy;
  int* why = reason ? reason : &why_dummy;
  *why = OR_CHART_SPEED;
  double T = pr->t_enter + z[0] * (pr->t_fall - pr->t_enter);
  double tf = T + pr->t_offset;
  double c[3], xd[3];
  for (int k = 0; k < 3; ++k) {
    c[k] = pr->x0[k] + pr->v0[k] * tf + 0.5 * pr->g[k] * tf * tf;
    xd[k] = pr->v0[k] + pr->g[k] * tf;
  }
  *T_req = T;
  double sp = norm3(xd);
  if (!(sp > 0.0)) return 0;
  double u[3] = {-xd[0] / sp, -xd[1] / sp, -xd[2] / sp};
  double e1[3], e2[3];
  complete_basis(u, e1, e2);
  double ct = 1.0 - z[1] * (1.0 - pr->a_min);
  double st = sqrt(fmax(0.0, 1.0 - ct * ct));
  double ph = 2.0 * M_PI * z[2];
  double dvec[3];
  for (int k = 0; k < 3; ++k) dvec[k] = ct * u[k] + st * (cos(ph) * e1[k] + sin(ph) * e2[k]);
  double s = 0.5 + 1.5 * z[8];
  double vb[3], vr[3];
  for (int k = 0; k < 3; ++k) { vb[k] = s * dvec[k]; vr[k] = vb[k] - xd[k]; }
  double vrn = norm3(vr);
  *vrel_out = vrn;
  for (int k = 0; k < 3; ++k) vb_out[k] = vb[k];
  if (!(vrn >= pr->v_min)) return 0;
  double nh[3] = {vr[0] / vrn, vr[1] / vrn, vr[2] / vrn};
  double m1[3], m2[3];
  complete_basis(nh, m1, m2);
  double beta = z[5] * acos(pr->a_min);
  double gam = 2.0 * M_PI * z[4];
  double nb[3];
  for (int k = 0; k < 3; ++k)
    nb[k] = cos(beta) * nh[k] + sin(beta) * (cos(gam) * m1[k] + sin(gam) * m2[k]);
  double k1[3], k2[3];
  complete_basis(nb, k1, k2);
  double psi = 2.0 * M_PI * z[3];
  double bax[3];
  for (int k = 0; k < 3; ++k) bax[k] = cos(psi) * k1[k] + sin(psi) * k2[k];
  double bz[3];
  cross3(bax, nb, bz);
  /* R_g maps (blade_axis, blade_normal, axis x normal) of the EE frame onto
   * (bax, nb, bax x nb) */
  double ea[3] = {arm->blade_axis[0], arm->blade_axis[1], arm->blade_axis[2]};
  double en[3] = {arm->blade_normal[0], arm->blade_normal[1], arm->blade_normal[2]};
  double ez[3];
  cross3(ea, en, ez);
  double Rg[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Rg[i][j] = bax[i] * ea[j] + nb[i] * en[j] + bz[i] * ez[j];
  double pe[3];
  for (int k = 0; k < 3; ++k) pe[k] = arm->blade_base[k] + z[7] * arm->blade_len * arm->blade_axis[k];
  double Rpe[3];
  matvec(Rg, pe, Rpe);
  double pg[3] = {c[0] - Rpe[0], c[1] - Rpe[1], c[2] - Rpe[2]};

  double q[7];
  int found = 0;
  for (int st = 0; st < OR_IK_STARTS && !found; ++st)
    found = ik_solve(arm, Rg, pg, z[6], st, q);
  *why = OR_CHART_IK;
  if (!found) return 0;
  *why = OR_CHART_BOX;
  for (int j = 0; j < 7; ++j)
    if (!(q[j] >= arm->q_lo[j] && q[j] <= arm->q_hi[j])) return 0;
  /* rows 0-2 of the point Jacobian: the contact point's linear velocity */
  double J[6][7];
  or_jacobian_point(arm, q, c, J);
  double A[6][6];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double sacc = 0.0;
      for (int m = 0; m < 7; ++m) sacc += J[i][m] * J[j][m];
      A[i][j] = sacc;
    }
  double y[3];
  *why = OR_CHART_SINGULAR;
  if (!solve_gepp(3, A, vb, y)) return 0;
  double qd[7];
  for (int m = 0; m < 7; ++m) {
    double acc = 0.0;
    for (int i = 0; i < 3; ++i) acc += J[i][m] * y[i];
    qd[m] = acc;
  }
  *why = OR_CHART_TAPER;
  for (int j = 0; j < 7; ++j)
    if (!(fabs(qd[j]) <= or_taper(arm, j, q[j]))) return 0;
  for (int i = 0; i < 16; ++i) out_state[i] = 0.0;
  for (int j = 0; j < 7; ++j) { out_state[j] = q[j]; out_state[8 + j] = qd[j]; }
  *why = OR_CHART_OK;
  return 1;
}

/* Goal candidates: z from Philox streams 8..10 of the candidate's counter. */
void or_sample_goals(const or_arm* arm, const or_problem* pr, unsigned long long seed,
                     int iter, int problem, int first_index, int n, double* states,
                     double* T_req, double* vrel, int* valid, int* reason) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int c = 0; c < n; ++c) {
    double u[12], z[9], vb[3];
    for (int s = 0; s < 3; ++s) philox_uniforms(seed, first_index + c, iter, problem, 8 + s, u + 4 * s);
    for (int i = 0; i < 9; ++i) z[i] = u[i];
    valid[c] = or_goal_chart(arm, pr, z, states + 16 * (size_t)c, &T_req[c], &vrel[c], vb,
                             reason ? reason + c : NULL);
    if (!valid[c])
      for (int i = 0; i < 16; ++i) states[16 * (size_t)c + i] = 0.0;
  }
}

/* Eq. (ballistic) */
static void flight(const or_problem* pr, double t, double* x, double* xd) {
  for (int k = 0; k < 3; ++k) {
    if (x) x[k] = pr->x0[k] + pr->v0[k] * t + 0.5 * pr->g[k] * t * t;
    if (xd) xd[k] = pr->v0[k] + pr->g[k] * t;
  }
}

/* Eq. (objective) with Eq. (terms).  Readings: times T are plan times and the
 * flight (and its uncertainty) is evaluated at T + t_offset; probabilities
 * are clamped to >= 1e-30 before the log; (nu - nu0)_+ = 0 for nu <= nu0. */
static double sigma_at(const or_problem* pr, double t) {
  if (pr->sig_linear) return pr->sig_lin_a + pr->sig_lin_b * t;
  double a = pr->sig_p, b = pr->sig_v * t, c = 0.5 * pr->sig_a * t * t;
  return sqrt(a * a + b * b + c * c);
}

double or_objective(const or_problem* pr, double T, double vrel, double nu) {
  double sg = sigma_at(pr, T + pr->t_offset);
  double p_obj = erf(pr->r_catch / (sg * sqrt(2.0)));
  double xdf[3];
  flight(pr, pr->t_fall + pr->t_offset, NULL, xdf);
  double sig_t = sg / fabs(xdf[2]);
  double p_in = 0.5 * erfc(-((pr->t_fall - T) / sig_t) / sqrt(2.0));
  double log_arm = 0.0;
  if (nu > pr->nu0) log_arm = -pr->lam * (nu - pr->nu0) * T * (1.0 - pr->nu0 / nu);
  if (p_obj < 1e-30) p_obj = 1e-30;
  if (p_in < 1e-30) p_in = 1e-30;
  return pr->w_v * fmin(vrel, pr->v_target) + pr->w_p * log(p_obj) + pr->w_r * log(p_in) +
         pr->w_x * log_arm;
}

/* closest point of segment [a, b] to x */
static void seg_closest(const double* a, const double* b, const double* x, double* p) {
  double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double ax[3] = {x[0] - a[0], x[1] - a[1], x[2] - a[2]};
  double l2 = dot3(ab, ab);
  double u = l2 > 0.0 ? dot3(ax, ab) / l2 : 0.0;
  if (u < 0.0) u = 0.0;
  if (u > 1.0) u = 1.0;
  for (int k = 0; k < 3; ++k) p[k] = a[k] + u * ab[k];
}

/* Eq. (reach) on a G-point grid T_g = t_enter + g (t_fall - t_enter)/(G-1):
 * the first T_g with t_n + |p_n - x(T_g)| / V_tip <= T_g, where p_n is the
 * point of the node's blade edge nearest to x(T_g) (reading). */
int or_reach_time(const or_arm* arm, const or_problem* pr, const double* q, double t_n,
                  int G, double* T_n) {
  double b0[3], b1[3];
  or_blade(arm, q, b0, b1);
  for (int g = 0; g < G; ++g) {
    double T = pr->t_enter + (double)g * (pr->t_fall - pr->t_enter) / (double)(G - 1);
    double x[3], p[3];
    flight(pr, T + pr->t_offset, x, NULL);
    seg_closest(b0, b1, x, p);
    double dd[3] = {p[0] - x[0], p[1] - x[1], p[2] - x[2]};
    if (t_n + norm3(dd) / pr->v_tip <= T) { *T_n = T; return g; }
  }
  *T_n = INFINITY;
  return -1;
}

/* distance between point x and segment [a, b] */
static double point_seg_dist(const double* a, const double* b, const double* x) {
  double p[3];
  seg_closest(a, b, x, p);
  double d[3] = {x[0] - p[0], x[1] - p[1], x[2] - p[2]};
  return norm3(d);
}

/* Clear (Sec. IV-E, collision checking), with the obstacle/arm roles of the
 * stress workload: obstacles are spheres, the arm is one capsule per link
 * (segment between consecutive frame origins 1..7 and then to the
 * end-effector origin, radius link_radius[j]).  Returns the minimum over the
 * S collocation points (both ends included), links and spheres of
 *   |centre - segment| - r_link - r_obs. */
double or_edge_clearance(const or_arm* arm, const float* s0, const float* s1, double T,
                         int S, const float* obs, int n_obs) {
  int n = arm->dof;
  double q0[7], qd0[7], q1[7], qd1[7];
  unpack(s0, n, q0, qd0);
  unpack(s1, n, q1, qd1);
  double best = INFINITY;
  for (int s = 0; s < S; ++s) {
    double t = (double)s * T / (double)(S - 1);
    double q[7] = {0}, qd[7], qdd[7];
    or_cubic(n, q0, qd0, q1, qd1, T, t, q, qd, qdd);
    double R[8][3][3], o[8][3];
    or_fk(arm, q, R, o);
    for (int j = 0; j < 7; ++j) {
      for (int b = 0; b < n_obs; ++b) {
        double cc[3] = {obs[4 * b], obs[4 * b + 1], obs[4 * b + 2]};
        double dist = point_seg_dist(o[j], o[j + 1], cc) - arm->link_radius[j] - (double)obs[4 * b + 3];
        if (dist < best) best = dist;
      }
    }
  }
  return best;
}

/* The tracking controller of Eq. (controller), one control cycle per
 * instance b.  From the measured state (q, qd) it refits the cubic to the
 * rendezvous (q_g, qd_g) over the horizon T and takes its initial
 * acceleration 6 (q_g - q) / T^2 - (4 qd + 2 qd_g) / T, clipped to [l, u];
 * Eq. (torque) gives the command, which is clipped to the torque, power and
 * slew limits.  Readings:
 *   - [l, u] keeps the velocity after one control period dt inside the
 *     taper: l = (-qdbar(q) - qd) / dt, u = (qdbar(q) - qd) / dt;
 *   - torque: each tau_i clamped to [-tau_max_i, tau_max_i];
 *   - power: if |sum_i tau_i qd_i| > W_max the whole vector is scaled by
 *     W_max / |sum| (its direction is kept);
 *   - slew (if tau_prev and rate are given): each tau_i clamped to
 *     tau_prev_i +- rate_i dt, last, so the rate limit always holds;
 *   - flags: bit 0 acceleration clipped, 1 torque, 2 power, 3 slew;
 *     0x80 invalid input (non-finite values, T <= 0): tau and qdd are NaN. */
void or_controller_torque(const or_arm* arm, int B, const float* state, const float* goal,
                          const float* T, const float* tau_prev, double dt, const double* rate,
                          double* tau, double* qdd, unsigned char* flags) {
  int n = arm->dof;
  for (int b = 0; b < B; ++b) {
    const float* sx = state + 16 * (size_t)b;
    const float* sg = goal + 16 * (size_t)b;
    double* tb = tau + 7 * (size_t)b;
    double* ab = qdd + 7 * (size_t)b;
    double Tb = (double)T[b];
    unsigned char f = 0;
    if (!state_finite(sx, n) || !state_finite(sg, n) || !isfinite(Tb) || !(Tb > 0.0)) {
      for (int i = 0; i < 7; ++i) tb[i] = ab[i] = NAN;
      flags[b] = 0x80;
      continue;
    }
    double q[7], qd[7], qg[7], qdg[7];
    unpack(sx, n, q, qd);
    unpack(sg, n, qg, qdg);
    for (int i = 0; i < n; ++i) {
      double a = 6.0 * (qg[i] - q[i]) / (Tb * Tb) - (4.0 * qd[i] + 2.0 * qdg[i]) / Tb;
      double bound = or_taper(arm, i, q[i]);
      double lo = (-bound - qd[i]) / dt, hi = (bound - qd[i]) / dt;
      double c = a < lo ? lo : (a > hi ? hi : a);
      if (c != a) f |= 1;
      ab[i] = c;
    }
    double t7[7];
    or_torque(arm, q, qd, ab, t7);
    for (int i = 0; i < n; ++i) {
      double m = arm->tau_max[i];
      if (t7[i] > m) { t7[i] = m; f |= 2; }
      if (t7[i] < -m) { t7[i] = -m; f |= 2; }
    }
    double pw = 0.0;
    for (int i = 0; i < n; ++i) pw += t7[i] * qd[i];
    if (fabs(pw) > arm->w_max) {
      double sc = arm->w_max / fabs(pw);
      for (int i = 0; i < n; ++i) t7[i] *= sc;
      f |= 4;
    }
    if (tau_prev && rate) {
      const float* tp = tau_prev + 7 * (size_t)b;
      for (int i = 0; i < n; ++i) {
        double lo = (double)tp[i] - rate[i] * dt, hi = (double)tp[i] + rate[i] * dt;
        if (t7[i] < lo) { t7[i] = lo; f |= 8; }
        if (t7[i] > hi) { t7[i] = hi; f |= 8; }
      }
    }
    for (int i = 0; i < 7; ++i) tb[i] = i < n ? t7[i] : 0.0;
    for (int i = n; i < 7; ++i) ab[i] = 0.0;
    flags[b] = f;
  }
}

/* The full-resolution recheck of a plan's edges (Sec. IV-E: the plan sent to
 * the controller is rechecked at full resolution): each edge at its own
 * duration T[e], all three ratios of Def. "Feasibility Check" over S samples
 * and the clearance of or_edge_clearance over S_clear points;
 * ok = rho_tau, rho_P, rho_v <= 1 and (no obstacles or clearance >= margin).
 * Non-finite states or T <= 0: NaN ratios and clearance, ok = 0. */
void or_check_edges(const or_arm* arm, int E, const float* s0, const float* s1, const float* T,
                    int S, int S_clear, const float* obs, int n_obs, double margin, double* rho3,
                    double* clearance, unsigned char* ok) {
  int n = arm->dof;
#pragma omp parallel for schedule(dynamic, 1)
  for (int e = 0; e < E; ++e) {
    const float* a = s0 + 16 * (size_t)e;
    const float* b = s1 + 16 * (size_t)e;
    double* r3 = rho3 + 3 * (size_t)e;
    if (!state_finite(a, n) || !state_finite(b, n) || !isfinite(T[e]) || !(T[e] > 0.0f)) {
      r3[0] = r3[1] = r3[2] = NAN;
      clearance[e] = NAN;
      ok[e] = 0;
      continue;
    }
    or_rho(arm, a, b, (double)T[e], S, r3);
    double c = n_obs > 0 ? or_edge_clearance(arm, a, b, (double)T[e], S_clear, obs, n_obs) : INFINITY;
    clearance[e] = c;
    ok[e] = (r3[0] <= 1.0 && r3[1] <= 1.0 && r3[2] <= 1.0 && (n_obs == 0 || c >= margin)) ? 1 : 0;
  }
}

/* ------------------------------------------------------------------------
 * Sampling densities of Sec. IV-E ("Batched expansion").
 * Goal parameters come from p_theta, a Gaussian mixture over the chart's
 * parameter cube Z = [0, 1]^9 mixed with a uniform component; free states
 * are Gaussian perturbations of points on the joint-space chord from the
 * root to a decoded goal of the same round, mixed with uniform draws.
 * Readings:
 *   - diagonal covariances, at most 4 components; the uniform weight w_u
 *     is fixed, the mixture is refit (or_em in oracle/density.py);
 *   - a Gaussian draw is folded back into Z: the three angle parameters
 *     (z2, z3, z4) wrap modulo 1, the others reflect at 0 and 1;
 *   - normals by Box-Muller from the candidate's own Philox uniforms;
 *   - the integer decisions (uniform component or not, which component,
 *     chord or uniform, which goal) are taken in single precision from the
 *     exactly representable uniforms, as on the GPU;
 *   - chord point: q0 + lambda (q_g - q0) + sigma * half-range * n, clamped
 *     to the joint box; the velocity is drawn as for a uniform candidate.
 * Philox streams of candidate (seed, index, iter, problem): 0-3 uniform free
 * state, 4 chord decisions (choice, goal, lambda), 5-6 chord normals, 8-10
 * chart parameters, 11 mixture decision, 12-14 mixture normals. */
static int z_angle(int i) { return i == 2 || i == 3 || i == 4; }

static double z_fold(int i, double z) {
  if (z_angle(i)) return z - floor(z);
  double t = z - 2.0 * floor(0.5 * z);
  return t <= 1.0 ? t : 2.0 - t;
}

static void box_muller(double ua, double ub, double* n0, double* n1) {
  double r = sqrt(-2.0 * log(1.0 - ua));
  *n0 = r * cos(2.0 * M_PI * ub);
  *n1 = r * sin(2.0 * M_PI * ub);
}

void or_density_z(const or_density* th, unsigned long long seed, int index, int iter, int problem,
                  double* z) {
  double u[12];
  for (int s = 0; s < 3; ++s) philox_uniforms(seed, index, iter, problem, 8 + s, u + 4 * s);
  for (int i = 0; i < 9; ++i) z[i] = u[i];
  if (th == NULL || th->C <= 0) return;
  double us[4];
  philox_uniforms(seed, index, iter, problem, 11, us);
  float sel = (float)us[0];
  if (sel < th->w_u) return;                       /* the uniform component */
  float v = (sel - th->w_u) / (1.0f - th->w_u);
  int m = th->C - 1;
  float acc = 0.0f;
  for (int c = 0; c < th->C; ++c) {
    acc += th->pi[c];
    if (v < acc) { m = c; break; }
  }
  double un[12], nrm[10];
  for (int s = 0; s < 3; ++s) philox_uniforms(seed, index, iter, problem, 12 + s, un + 4 * s);
  for (int k = 0; k < 5; ++k) box_muller(un[2 * k], un[2 * k + 1], &nrm[2 * k], &nrm[2 * k + 1]);
  for (int i = 0; i < 9; ++i)
    z[i] = z_fold(i, (double)th->mu[m][i] + (double)th->sd[m][i] * nrm[i]);
}

void or_sample_goals_density(const or_arm* arm, const or_problem* pr, const or_density* th,
                             unsigned long long seed, int iter, int problem, int first_index,
                             int n, double* states, double* T_req, double* vrel, int* valid,
                             double* zs) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int c = 0; c < n; ++c) {
    double z[9], vb[3];
    or_density_z(th, seed, first_index + c, iter, problem, z);
    if (zs)
      for (int i = 0; i < 9; ++i) zs[9 * (size_t)c + i] = z[i];
    valid[c] = or_goal_chart(arm, pr, z, states + 16 * (size_t)c, &T_req[c], &vrel[c], vb, NULL);
    if (!valid[c])
      for (int i = 0; i < 16; ++i) states[16 * (size_t)c + i] = 0.0;
  }
}

void or_sample_chord(const or_arm* arm, unsigned long long seed, int iter, int problem,
                     int first_index, int n, double vel_frac, const double* q0,
                     const double* goals, int n_goals, float w_chord, double sigma,
                     double* states) {
  for (int c = 0; c < n; ++c) {
    const int index = first_index + c;
    double u[16], uc[4];
    for (int s = 0; s < 4; ++s) philox_uniforms(seed, index, iter, problem, s, u + 4 * s);
    philox_uniforms(seed, index, iter, problem, 4, uc);
    double* st = states + 16 * (size_t)c;
    for (int i = 0; i < 16; ++i) st[i] = 0.0;
    int chord = n_goals > 0 && (float)uc[0] < w_chord;
    int g = 0;
    double nrm[8];
    if (chord) {
      g = (int)floorf((float)uc[1] * (float)n_goals);
      if (g > n_goals - 1) g = n_goals - 1;
      double un[8];
      for (int s = 0; s < 2; ++s) philox_uniforms(seed, index, iter, problem, 5 + s, un + 4 * s);
      for (int k = 0; k < 4; ++k) box_muller(un[2 * k], un[2 * k + 1], &nrm[2 * k], &nrm[2 * k + 1]);
    }
    for (int j = 0; j < 7; ++j) {
      double lo = arm->q_lo[j], hi = arm->q_hi[j], qj;
      if (chord) {
        const double qg = goals[16 * (size_t)g + j];
        qj = q0[j] + uc[2] * (qg - q0[j]) + sigma * 0.5 * (hi - lo) * nrm[j];
        qj = qj < lo ? lo : (qj > hi ? hi : qj);
      } else {
        qj = lo + u[j] * (hi - lo);
      }
      st[j] = qj;
      st[8 + j] = (2.0 * u[7 + j] - 1.0) * vel_frac * or_taper(arm, j, qj);
    }
  }
}
