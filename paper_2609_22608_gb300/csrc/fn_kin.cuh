// Device kinematics and the planner's per-sample math (FP32):
//   forward kinematics / geometric Jacobian (modified DH),
//   Philox4x32-10 (Salmon et al., SC'11) for the samplers,
//   the goal chart phi(z) of Def. "Goal chart" with a damped-least-squares IK,
//   the objective of Eq. (objective) / Eq. (terms),
//   the earliest reach time of Eq. (reach),
//   link-capsule clearance to obstacle spheres (Sec. IV-E, collision checking).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fn_api.h"
#include "fn_arm.cuh"

namespace fn {

// ---------------------------------------------------------------------------
// Philox4x32-10: ten rounds of the Philox S-box with the key bumped by the
// Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// 24-bit uniform in [0, 1), exactly representable in FP32
__device__ __forceinline__ float u01(unsigned x) { return __uint2float_rn(x >> 8) * 5.9604644775390625e-8f; }

__device__ __forceinline__ void philox_u4(unsigned long long seed, int index, int iter,
                                          int problem, int stream, float* u) {
  const uint4 r = philox4x32_10(make_uint4((unsigned)index, (unsigned)iter, (unsigned)problem,
                                           (unsigned)stream),
                                make_uint2((unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32)));
  u[0] = u01(r.x); u[1] = u01(r.y); u[2] = u01(r.z); u[3] = u01(r.w);
}

// ---------------------------------------------------------------------------
// small vector helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cross3(const float* a, const float* b, float* c) {
  const float x = a[1] * b[2] - a[2] * b[1];
  const float y = a[2] * b[0] - a[0] * b[2];
  const float z = a[0] * b[1] - a[1] * b[0];
  c[0] = x; c[1] = y; c[2] = z;
}
__device__ __forceinline__ float dot3(const float* a, const float* b) {
  return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2]));
}
__device__ __forceinline__ float norm3(const float* a) { return sqrtf(dot3(a, a)); }

// ---------------------------------------------------------------------------
// Forward kinematics.  Joint j's frame: R_j = R_{j-1} Rx(alpha_j) Rz(theta_j),
// o_j = o_{j-1} + R_{j-1} p_j.  Calls visit(j, R (row-major 3x3), o) for
// frames 1..7 (j = 0..6) and returns the end-effector frame (frame 7 moved
// flange_d along its z axis).
// ---------------------------------------------------------------------------
template <class Visit>
__device__ __forceinline__ void fk_frames(const ArmK& A, const float* q, float* Ree, float* oee,
                                          Visit&& visit) {
  float R[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
  float o[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    float s, c;
    sincosf(q[j] + A.th0[j], &s, &c);
    const float ca = A.ca[j], sa = A.sa[j];
    // o += R p_j
    const float px = A.px[j], py = A.py[j], pz = A.pz[j];
    float n0 = fmaf(R[0], px, fmaf(R[1], py, R[2] * pz));
    float n1 = fmaf(R[3], px, fmaf(R[4], py, R[5] * pz));
    float n2 = fmaf(R[6], px, fmaf(R[7], py, R[8] * pz));
    o[0] += n0; o[1] += n1; o[2] += n2;
    // R = R Rx(alpha) Rz(theta); Rx(alpha) Rz(theta) = [[c,-s,0],[s ca, c ca,-sa],[s sa, c sa, ca]]
    const float m00 = c, m01 = -s, m02 = 0.f;
    const float m10 = s * ca, m11 = c * ca, m12 = -sa;
    const float m20 = s * sa, m21 = c * sa, m22 = ca;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float a0 = R[3 * r], a1 = R[3 * r + 1], a2 = R[3 * r + 2];
      R[3 * r + 0] = fmaf(a0, m00, fmaf(a1, m10, a2 * m20));
      R[3 * r + 1] = fmaf(a0, m01, fmaf(a1, m11, a2 * m21));
      R[3 * r + 2] = fmaf(a0, m02, fmaf(a1, m12, a2 * m22));
    }
    visit(j, R, o);
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) Ree[i] = R[i];
  oee[0] = fmaf(A.flange_d, R[2], o[0]);
  oee[1] = fmaf(A.flange_d, R[5], o[1]);
  oee[2] = fmaf(A.flange_d, R[8], o[2]);
}

// Joint axes z_j and origins o_j (frames 1..7) with the end-effector pose.
struct Axes {
  float z[7][3], o[7][3];
};

__device__ __forceinline__ void fk_axes(const ArmK& A, const float* q, Axes& ax, float* Ree,
                                        float* oee) {
  fk_frames(A, q, Ree, oee, [&](int j, const float* R, const float* o) {
    ax.z[j][0] = R[2]; ax.z[j][1] = R[5]; ax.z[j][2] = R[8];
    ax.o[j][0] = o[0]; ax.o[j][1] = o[1]; ax.o[j][2] = o[2];
  });
}

// blade edge endpoints in the world frame
__device__ __forceinline__ void blade_world(const ArmK& A, const float* Ree, const float* oee,
                                            float* b0, float* b1) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float w = fmaf(Ree[3 * r], A.bb[0], fmaf(Ree[3 * r + 1], A.bb[1], Ree[3 * r + 2] * A.bb[2]));
    const float a = fmaf(Ree[3 * r], A.bax[0], fmaf(Ree[3 * r + 1], A.bax[1], Ree[3 * r + 2] * A.bax[2]));
    b0[r] = oee[r] + w;
    b1[r] = fmaf(A.blen, a, b0[r]);
  }
}

// closest point of segment [a, b] to x
__device__ __forceinline__ void seg_closest(const float* a, const float* b, const float* x,
                                            float* p) {
  const float ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  const float ax[3] = {x[0] - a[0], x[1] - a[1], x[2] - a[2]};
  const float l2 = dot3(ab, ab);
  float u = l2 > 0.f ? dot3(ax, ab) / l2 : 0.f;
  u = fminf(fmaxf(u, 0.f), 1.f);
  p[0] = fmaf(u, ab[0], a[0]);
  p[1] = fmaf(u, ab[1], a[1]);
  p[2] = fmaf(u, ab[2], a[2]);
}

// hardware reciprocal approximation (rcp.approx, relative error ~2^-23)
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// unit vectors (e1, e2) completing u to a right-handed frame
__device__ __forceinline__ void complete_basis(const float* u, float* e1, float* e2) {
  float h[3] = {0.f, 0.f, 1.f};
  if (!(fabsf(u[2]) < 0.9f)) { h[0] = 1.f; h[2] = 0.f; }
  cross3(h, u, e1);
  const float l = norm3(e1);
  e1[0] /= l; e1[1] /= l; e1[2] /= l;
  cross3(u, e1, e2);
}

#define FN_IK_ITERS 24
#define FN_IK_STARTS 4
#define FN_IK_LAMBDA 5e-2f
#define FN_IK_POS_TOL 1e-4f
#define FN_IK_ROT_TOL 1e-3f

// One damped-least-squares IK run on joints 1-6, q7 fixed: start `st` is the
// box centre shifted by +-(0, .5, 0, -.5, 0, .5) half-ranges (st = 1, 2) or
// by (0, -.5, 0, -.5, 0, -.5) (st = 3), with joint 1 turned towards the
// target's azimuth; iterates are projected onto
// the box; accepted when the position residual < 1e-4 m, the rotation
// residual (half the sum of column cross products) < 1e-3 and the rotation
// error is under 90 degrees (trace > 1).  The damped step
// dq = J^T (J J^T + lambda^2 I)^-1 e is taken in its equal form
// (J^T J + lambda^2 I)^-1 J^T e (J is square here: joints 1-6 against the
// six pose residuals), whose rows belong to the joints; the system is
// solved by Gauss-Jordan elimination without pivoting (symmetric positive
// definite), with the hardware reciprocal of each pivot, and the link
// rotations use the hardware sine/cosine.  Both are a few ulp from the
// rounded values, three orders below the residual tolerances that accept a
// start.
//
// The work of one iteration is spread over a group of 8 lanes (aligned in
// the warp; all 32 lanes must call this): lane s < 7 owns joint s, lane 7
// the flange offset.  The frames are
// the inclusive product scan of the 8 local transforms [Rx(alpha) Rz(theta),
// p] (three shuffle steps), lanes 0..5 form the Jacobian columns and share
// them, lane s < 6 forms row s of J^T J + lambda^2 I and entry s of J^T e,
// the six elimination steps take their pivot row from lane k by shuffles,
// and lane s then updates its own joint.  Returns (uniformly in the group)
// whether the start converged; qs is the lane's own final joint value.
__device__ __forceinline__ bool ik_solve_group(const ArmK& A, const float* Rg, const float* pg,
                                               float q7, int st, float& qs) {
  const int s = threadIdx.x & 7;
  const float sgn = st == 0 ? 0.f : (st == 2 ? -1.f : 1.f);
  // (0, .5, 0, -.5, 0, .5) for starts 1 and 2, (0, -.5, 0, -.5, 0, -.5) for start 3
  const float pat = (s & 1) ? (st == 3 ? -0.5f : (s == 3 ? -0.5f : 0.5f)) : 0.f;
  float qj = 0.f;
  if (s < 6) {
    const float c = 0.5f * (A.q_lo[s] + A.q_hi[s]);
    const float h = 0.5f * (A.q_hi[s] - A.q_lo[s]);
    qj = fmaf(sgn * pat, h, c);
  }
  if (s == 6) qj = q7;
  if (s == 0) qj = fminf(fmaxf(atan2f(pg[1], pg[0]), A.q_lo[0]), A.q_hi[0]);
  const float lo = s < 7 ? A.q_lo[s] : 0.f, hi = s < 7 ? A.q_hi[s] : 0.f;
  float ep[3], er[3], Ree[9], oee[3];
  bool failed = false;
  for (int it = 0; it <= FN_IK_ITERS; ++it) {
    // local transform of this lane's link
    float R[9], o[3];
    if (s < 7) {
      float sn, cs;
      __sincosf(qj + A.th0[s], &sn, &cs);   // |angle| < 2 pi; error ~1e-6, far below the IK tolerances
      const float ca = A.ca[s], sa = A.sa[s];
      R[0] = cs;      R[1] = -sn;     R[2] = 0.f;
      R[3] = sn * ca; R[4] = cs * ca; R[5] = -sa;
      R[6] = sn * sa; R[7] = cs * sa; R[8] = ca;
      o[0] = A.px[s]; o[1] = A.py[s]; o[2] = A.pz[s];
    } else {
      R[0] = 1.f; R[1] = 0.f; R[2] = 0.f;
      R[3] = 0.f; R[4] = 1.f; R[5] = 0.f;
      R[6] = 0.f; R[7] = 0.f; R[8] = 1.f;
      o[0] = 0.f; o[1] = 0.f; o[2] = A.flange_d;
    }
    // inclusive scan: [R, o] <- [Rl, ol] [R, o] = [Rl R, ol + Rl o]
#pragma unroll
    for (int d = 1; d < 8; d <<= 1) {
      float Rl[9], ol[3];
#pragma unroll
      for (int k = 0; k < 9; ++k) Rl[k] = __shfl_up_sync(0xffffffffu, R[k], d, 8);
#pragma unroll
      for (int k = 0; k < 3; ++k) ol[k] = __shfl_up_sync(0xffffffffu, o[k], d, 8);
      if (s >= d) {
        float Rn[9], on[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
#pragma unroll
          for (int c = 0; c < 3; ++c)
            Rn[3 * r + c] = fmaf(Rl[3 * r], R[c], fmaf(Rl[3 * r + 1], R[3 + c], Rl[3 * r + 2] * R[6 + c]));
          on[r] = ol[r] + fmaf(Rl[3 * r], o[0], fmaf(Rl[3 * r + 1], o[1], Rl[3 * r + 2] * o[2]));
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = Rn[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) o[k] = on[k];
      }
    }
    // end-effector pose from lane 7 of the group
#pragma unroll
    for (int k = 0; k < 9; ++k) Ree[k] = __shfl_sync(0xffffffffu, R[k], 7, 8);
#pragma unroll
    for (int k = 0; k < 3; ++k) oee[k] = __shfl_sync(0xffffffffu, o[k], 7, 8);
    ep[0] = pg[0] - oee[0]; ep[1] = pg[1] - oee[1]; ep[2] = pg[2] - oee[2];
    er[0] = er[1] = er[2] = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float rc[3] = {Ree[c], Ree[3 + c], Ree[6 + c]};
      const float rg[3] = {Rg[c], Rg[3 + c], Rg[6 + c]};
      float x[3];
      cross3(rc, rg, x);
      er[0] = fmaf(0.5f, x[0], er[0]); er[1] = fmaf(0.5f, x[1], er[1]); er[2] = fmaf(0.5f, x[2], er[2]);
    }
    if (it == FN_IK_ITERS || failed) break;
    // own Jacobian column c_s (joints 0..5), then everyone's
    float Jc[6];
    {
      const float z[3] = {R[2], R[5], R[8]};
      const float r[3] = {oee[0] - o[0], oee[1] - o[1], oee[2] - o[2]};
      float v[3];
      cross3(z, r, v);
      Jc[0] = v[0]; Jc[1] = v[1]; Jc[2] = v[2]; Jc[3] = z[0]; Jc[4] = z[1]; Jc[5] = z[2];
    }
    float J[6][6];
#pragma unroll
    for (int m = 0; m < 6; ++m)
#pragma unroll
      for (int i = 0; i < 6; ++i) J[i][m] = __shfl_sync(0xffffffffu, Jc[i], m, 8);
    // lane s < 6 owns row s of N = J^T J + lambda^2 I and g_s = c_s . e
    const float e[6] = {ep[0], ep[1], ep[2], er[0], er[1], er[2]};
    float Nr[6], gr = 0.f;
#pragma unroll
    for (int n = 0; n < 6; ++n) {
      float sacc = n == s ? FN_IK_LAMBDA * FN_IK_LAMBDA : 0.f;
#pragma unroll
      for (int i = 0; i < 6; ++i) sacc = fmaf(Jc[i], J[i][n], sacc);
      Nr[n] = sacc;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) gr = fmaf(Jc[i], e[i], gr);
    // Gauss-Jordan on the rows: step k takes pivot row k from lane k and
    // clears column k in every other row (columns below k are no longer
    // read); every lane sees the same pivots, so a non-positive one fails
    // the whole group
    bool pos = true;
    float piv = 1.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float pkk = __shfl_sync(0xffffffffu, Nr[k], k, 8);
      const float pg = __shfl_sync(0xffffffffu, gr, k, 8);
      float pr[6];
#pragma unroll
      for (int j = k + 1; j < 6; ++j) pr[j] = __shfl_sync(0xffffffffu, Nr[j], k, 8);
      pos = pos && pkk > 0.f;
      if (s == k) piv = pkk;
      const float f = s == k ? 0.f : Nr[k] * rcp_approx(pkk);
#pragma unroll
      for (int j = k + 1; j < 6; ++j) Nr[j] = fmaf(-f, pr[j], Nr[j]);
      gr = fmaf(-f, pg, gr);
    }
    if (!pos) {
      failed = true;
      break;
    }
    if (s < 6) qj = fminf(fmaxf(fmaf(gr, rcp_approx(piv), qj), lo), hi);
  }
  qs = qj;
  if (failed || !(norm3(ep) < FN_IK_POS_TOL && norm3(er) < FN_IK_ROT_TOL)) return false;
  float tr = 0.f;
#pragma unroll
  for (int i = 0; i < 9; ++i) tr = fmaf(Rg[i], Ree[i], tr);
  return tr > 1.f;
}

// Eq. (ballistic) at flight time t
__device__ __forceinline__ void flight(const fn_problem_t& P, float t, float* x, float* xd) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (x) x[k] = fmaf(0.5f * P.g[k] * t, t, fmaf(P.v0[k], t, P.x0[k]));
    if (xd) xd[k] = fmaf(P.g[k], t, P.v0[k]);
  }
}

// Goal chart phi(z), decoding part: arrival T, contact c = x(T + t_offset),
// blade velocity v_b, |v_rel| and the end-effector target pose (R_g, p_g).
// Returns false where phi is undefined before the IK (|v_rel| < v_min).
//   z0: T in [t_enter, t_fall];  z1, z2: approach direction in the cone of
//   half-angle acos(a_min) about -xdot (polar acos(1 - z1 (1 - a_min)),
//   azimuth 2 pi z2);  z8: closing speed 0.5 + 1.5 z8 -> v_b;
//   z5, z4: cutting direction = v_rel direction tilted by z5 acos(a_min)
//   towards roll 2 pi z4;  z3: blade-axis spin 2 pi z3 about it;
//   z7: contact at z7 blade_len along the edge;  z6: q7 in its range.
struct ChartPose {
  float T, vrel, q7;
  float c[3], vb[3], Rg[9], pg[3];
};

__device__ __forceinline__ bool chart_pose(const ArmK& A, const fn_problem_t& P, const float* z,
                                           ChartPose& o) {
  o.T = fmaf(z[0], P.t_fall - P.t_enter, P.t_enter);
  float xd[3];
  flight(P, o.T + P.t_offset, o.c, xd);
  const float sp = norm3(xd);
  o.vrel = 0.f;
  if (!(sp > 0.f)) return false;
  const float u[3] = {-xd[0] / sp, -xd[1] / sp, -xd[2] / sp};
  float e1[3], e2[3];
  complete_basis(u, e1, e2);
  const float ct = fmaf(-z[1], 1.f - P.a_min, 1.f);
  const float st = sqrtf(fmaxf(0.f, fmaf(-ct, ct, 1.f)));
  float sph, cph;
  sincospif(2.f * z[2], &sph, &cph);
  float vr[3];
  const float s = fmaf(1.5f, z[8], 0.5f);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float d = fmaf(ct, u[k], st * fmaf(cph, e1[k], sph * e2[k]));
    o.vb[k] = s * d;
    vr[k] = o.vb[k] - xd[k];
  }
  o.vrel = norm3(vr);
  if (!(o.vrel >= P.v_min)) return false;
  const float nh[3] = {vr[0] / o.vrel, vr[1] / o.vrel, vr[2] / o.vrel};
  float m1[3], m2[3];
  complete_basis(nh, m1, m2);
  const float beta = z[5] * acosf(P.a_min);
  float sb, cb, sg, cg;
  sincosf(beta, &sb, &cb);
  sincospif(2.f * z[4], &sg, &cg);
  float nb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) nb[k] = fmaf(cb, nh[k], sb * fmaf(cg, m1[k], sg * m2[k]));
  float k1[3], k2[3];
  complete_basis(nb, k1, k2);
  float sps, cps;
  sincospif(2.f * z[3], &sps, &cps);
  float bax[3], bz[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) bax[k] = fmaf(cps, k1[k], sps * k2[k]);
  cross3(bax, nb, bz);
  const float ea[3] = {A.bax[0], A.bax[1], A.bax[2]};
  const float en[3] = {A.bnm[0], A.bnm[1], A.bnm[2]};
  float ez[3];
  cross3(ea, en, ez);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) o.Rg[3 * i + j] = fmaf(bax[i], ea[j], fmaf(nb[i], en[j], bz[i] * ez[j]));
  float pe[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) pe[k] = fmaf(z[7] * A.blen, A.bax[k], A.bb[k]);
#pragma unroll
  for (int r = 0; r < 3; ++r)
    o.pg[r] = o.c[r] - fmaf(o.Rg[3 * r], pe[0], fmaf(o.Rg[3 * r + 1], pe[1], o.Rg[3 * r + 2] * pe[2]));
  o.q7 = fmaf(z[6], A.q_hi[6] - A.q_lo[6], A.q_lo[6]);
  return true;
}

// why a goal draw is undefined: the first failing condition of phi(z)
enum ChartWhy { CHART_OK = 0, CHART_SPEED = 1, CHART_IK = 2, CHART_BOX = 3, CHART_SINGULAR = 4,
                CHART_TAPER = 5 };

// Goal chart phi(z), velocity part after the IK: the box check, then
// qd_g = J_p^T (J_p J_p^T)^-1 v_b with J_p the 3x7 Jacobian of the contact
// point's linear velocity (v_ee is a linear velocity: the minimum-norm joint
// velocity that moves the blade at v_b at the contact), undefined if any
// |qd_g,j| exceeds the taper.  Returns CHART_OK or the failing condition.
__device__ __forceinline__ int chart_velocity(const ArmK& A, const ChartPose& o, const float* q,
                                              float* qd) {
#pragma unroll
  for (int j = 0; j < 7; ++j)
    if (!(q[j] >= A.q_lo[j] && q[j] <= A.q_hi[j])) return CHART_BOX;
  Axes ax;
  float Ree[9], oee[3];
  fk_axes(A, q, ax, Ree, oee);
  float J[3][7];
#pragma unroll
  for (int m = 0; m < 7; ++m) {
    const float r[3] = {o.c[0] - ax.o[m][0], o.c[1] - ax.o[m][1], o.c[2] - ax.o[m][2]};
    float v[3];
    cross3(ax.z[m], r, v);
    J[0][m] = v[0]; J[1][m] = v[1]; J[2][m] = v[2];
  }
  // M = J_p J_p^T (symmetric positive definite unless J_p loses rank),
  // solved by Cholesky
  float M[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float sacc = 0.f;
#pragma unroll
      for (int m = 0; m < 7; ++m) sacc = fmaf(J[i][m], J[j][m], sacc);
      M[i][j] = sacc;
    }
  const float l00sq = M[0][0];
  if (!(l00sq > 0.f)) return CHART_SINGULAR;
  const float l00 = sqrtf(l00sq);
  const float l10 = M[1][0] / l00, l20 = M[2][0] / l00;
  const float l11sq = fmaf(-l10, l10, M[1][1]);
  if (!(l11sq > 0.f)) return CHART_SINGULAR;
  const float l11 = sqrtf(l11sq);
  const float l21 = fmaf(-l20, l10, M[2][1]) / l11;
  const float l22sq = fmaf(-l21, l21, fmaf(-l20, l20, M[2][2]));
  if (!(l22sq > 0.f)) return CHART_SINGULAR;
  const float l22 = sqrtf(l22sq);
  const float w0 = o.vb[0] / l00;
  const float w1 = fmaf(-l10, w0, o.vb[1]) / l11;
  const float w2 = fmaf(-l21, w1, fmaf(-l20, w0, o.vb[2])) / l22;
  float y[3];
  y[2] = w2 / l22;
  y[1] = fmaf(-l21, y[2], w1) / l11;
  y[0] = fmaf(-l20, y[2], fmaf(-l10, y[1], w0)) / l00;
#pragma unroll
  for (int m = 0; m < 7; ++m) qd[m] = fmaf(J[0][m], y[0], fmaf(J[1][m], y[1], J[2][m] * y[2]));
#pragma unroll
  for (int j = 0; j < 7; ++j)
    if (!(fabsf(qd[j]) <= taper(A, j, q[j]))) return CHART_TAPER;
  return CHART_OK;
}

// phi(z) on a whole warp (all 32 lanes call it): the chart pose on every
// lane, the FN_IK_STARTS starts on 8-lane groups (the lowest start that
// converges wins, the same result as trying them in order), then the
// velocity part on every lane.  Returns CHART_OK or the condition that left
// phi undefined (warp-uniform); q and qd hold the goal state on every lane
// when CHART_OK; o holds T, |v_rel| and the pose.
__device__ __forceinline__ int warp_decode_goal(const ArmK& A, const fn_problem_t& P,
                                                const float* z, ChartPose& o, float* q,
                                                float* qd) {
  const int lane = threadIdx.x & 31, grp = lane >> 3;
  if (!chart_pose(A, P, z, o)) return CHART_SPEED;   // warp-uniform
  float qs;
  static_assert(FN_IK_STARTS <= 4, "one 8-lane group per IK start");
  const bool found = ik_solve_group(A, o.Rg, o.pg, o.q7, grp < FN_IK_STARTS ? grp : 0, qs);
  const unsigned won = __ballot_sync(0xffffffffu, found && (lane & 7) == 0 && grp < FN_IK_STARTS);
  if (!won) return CHART_IK;
  const int winner = __ffs(won) - 1;                 // first lane of the winning group
#pragma unroll
  for (int j = 0; j < 7; ++j) q[j] = __shfl_sync(0xffffffffu, qs, winner + j);
  return chart_velocity(A, o, q, qd);
}

// Eq. (objective) with Eq. (terms); flight quantities at T + t_offset,
// probabilities clamped to >= 1e-30 before the log.
__device__ __forceinline__ float objective(const fn_problem_t& P, float T, float vrel, float nu) {
  const float tf = T + P.t_offset;
  float sg;
  if (P.sig_linear) {
    sg = fmaf(P.sig_lin_b, tf, P.sig_lin_a);
  } else {
    const float b = P.sig_v * tf, c = 0.5f * P.sig_a * tf * tf;
    sg = sqrtf(fmaf(P.sig_p, P.sig_p, fmaf(b, b, c * c)));
  }
  float p_obj = erff(P.r_catch / (sg * 1.41421356237f));
  const float xdz = fabsf(fmaf(P.g[2], P.t_fall + P.t_offset, P.v0[2]));
  const float sig_t = sg / xdz;
  float p_in = normcdff((P.t_fall - T) / sig_t);
  float log_arm = 0.f;
  if (nu > P.nu0) log_arm = -P.lam * (nu - P.nu0) * T * (1.f - P.nu0 / nu);
  p_obj = fmaxf(p_obj, 1e-30f);
  p_in = fmaxf(p_in, 1e-30f);
  return P.w_v * fminf(vrel, P.v_target) + P.w_p * logf(p_obj) + P.w_r * logf(p_in) +
         P.w_x * log_arm;
}

// Eq. (reach) on a G-point grid: first grid index g with
// t_n + |p_n - x(T_g + t_offset)| / V_tip <= T_g, p_n the closest point of the
// node's blade edge; -1 if none.
__device__ __forceinline__ int reach_index(const ArmK& A, const fn_problem_t& P, const float* q,
                                           float t_n, int G) {
  float Ree[9], oee[3], b0[3], b1[3];
  fk_frames(A, q, Ree, oee, [](int, const float*, const float*) {});
  blade_world(A, Ree, oee, b0, b1);
  const float step = (P.t_fall - P.t_enter) / (float)(G - 1);
  for (int g = 0; g < G; ++g) {
    const float T = fmaf((float)g, step, P.t_enter);
    float x[3], p[3];
    flight(P, T + P.t_offset, x, nullptr);
    seg_closest(b0, b1, x, p);
    const float d[3] = {p[0] - x[0], p[1] - x[1], p[2] - x[2]};
    if (t_n + norm3(d) / P.v_tip <= T) return g;
  }
  return -1;
}

// minimum over links and spheres of |centre - capsule axis| - r_link - r_obs
// at configuration q (capsules between consecutive frame origins 1..7 and
// from frame 7 to the end-effector origin)
__device__ __forceinline__ float config_clearance(const ArmK& A, const float* q,
                                                  const fn_problem_t& P) {
  float pts[8][3];
  float Ree[9], oee[3];
  fk_frames(A, q, Ree, oee, [&](int j, const float*, const float* o) {
    pts[j][0] = o[0]; pts[j][1] = o[1]; pts[j][2] = o[2];
  });
  pts[7][0] = oee[0]; pts[7][1] = oee[1]; pts[7][2] = oee[2];
  float best = INFINITY;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    for (int b = 0; b < P.n_obs; ++b) {
      const float cc[3] = {P.obs[b][0], P.obs[b][1], P.obs[b][2]};
      float p[3];
      seg_closest(pts[j], pts[j + 1], cc, p);
      const float d[3] = {cc[0] - p[0], cc[1] - p[1], cc[2] - p[2]};
      best = fminf(best, norm3(d) - A.lrad[j] - P.obs[b][3]);
    }
  }
  return best;
}

}  // namespace fn
