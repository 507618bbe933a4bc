// Device-side robot model and the per-sample dynamics of the edge check.
//
//   cubic edge ............ Def. "Cubic edge", Eq. (cubic)
//   torque ................ Eq. (torque): recursive Newton-Euler (modified DH)
//                           + reflected rotor inertia + Eq. (friction)
//   limit ratios .......... Def. "Feasibility Check", Eq. (rho)
//
// The robot is passed to every kernel by value (`ArmK`), so it lives in the
// kernel-parameter constant bank: every lane of a warp reads the same link
// entry at the same time, which the constant cache serves as a broadcast, and
// fully unrolled link loops turn each read into an immediate operand.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fn_api.h"

namespace fn {

struct ArmK {
  // modified-DH link transforms: R_j = Rx(alpha_j) Rz(theta0_j + q_j),
  // origin of frame j in frame j-1: p_j = (a_j, -sin(alpha_j) d_j, cos(alpha_j) d_j)
  float ca[7], sa[7];
  float px[7], py[7], pz[7];
  float th0[7];
  // inertial parameters (link frame, diagonal inertia about the COM)
  float m[7], cx[7], cy[7], cz[7], Ix[7], Iy[7], Iz[7];
  float arma[7];
  // friction: psi1 / (1 + exp(-psi2 (qd + psi3))) - foff, foff = psi1 sigmoid(psi2 psi3)
  float f1[7], f2[7], f3[7], foff[7];
  // limits
  float inv_tau[7], inv_w;
  float q_lo[7], q_hi[7], qd_max[7], taper2a[7];
  // base acceleration = -gravity (the standard RNEA gravity trick)
  float g0x, g0y, g0z;
  // end effector and blade (end-effector frame), capsule radii
  float flange_d;
  float bb[3], bax[3], bnm[3], blen;
  float lrad[7];
};

// Host-side conversion with validation (fn_api.cu).
bool make_armk(const fn_arm_t* a, ArmK* out);

// ---------------------------------------------------------------------------
// The cubic of Eq. (cubic) in normalised time u = t/T in [0, 1]:
//   sigma(u)     = q0 + b1 u + b2 u^2 + b3 u^3,
//   sigma_dot    = (b1 + 2 b2 u + 3 b3 u^2) / T,
//   sigma_ddot   = (2 b2 + 6 b3 u) / T^2,
//   b1 = qd0 T,  b2 = 3 d1 - d2 T,  b3 = d2 T - 2 d1,
//   d1 = q1 - q0 - qd0 T,  d2 = qd1 - qd0
// (identical to Eq. (cubic) with c2 = b2/T^2, c3 = b3/T^3).  In this form the
// coefficients are O(|q|) at any T, so the short edges whose t-form terms
// (~1e4 rad/s^2 at T = 0.05 s) cancel at mid-edge keep their accuracy.
// ---------------------------------------------------------------------------
struct Cubic {
  float q0[7], b1[7], b2[7], b3[7];
  float iT, iT2;
};

struct EdgeStates {
  float q0[7], qd0[7], q1[7], qd1[7];
};

__device__ __forceinline__ void load_state(const float4* __restrict__ p, float* q, float* qd) {
  float4 a = __ldg(p + 0), b = __ldg(p + 1), c = __ldg(p + 2), d = __ldg(p + 3);
  q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w;
  q[4] = b.x; q[5] = b.y; q[6] = b.z;
  qd[0] = c.x; qd[1] = c.y; qd[2] = c.z; qd[3] = c.w;
  qd[4] = d.x; qd[5] = d.y; qd[6] = d.z;
}

// error-free transformations (Knuth TwoSum, FMA-based TwoProd)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = fmaf(a, b, -p);
}

// Coefficients of one joint.  ACC = true carries d1, d2 and the products as
// unevaluated float pairs, so b2 and b3 come out (nearly) correctly rounded;
// ACC = false is the plain FP32 evaluation used where a decision only needs
// to hold up to the feasibility margin (the end-sample probes).
template <bool ACC>
__device__ __forceinline__ void joint_coef(float q0, float qd0, float q1, float qd1, float T,
                                           float& b1, float& b2, float& b3) {
  if (!ACC) {
    const float d1 = fmaf(-qd0, T, q1 - q0);
    const float d2 = qd1 - qd0;
    b1 = qd0 * T;
    b2 = fmaf(-d2, T, 3.0f * d1);
    b3 = fmaf(d2, T, -2.0f * d1);
    return;
  }
  float dqh, dql, ph, pl, d1h, d1l, d2h, d2l;
  two_sum(q1, -q0, dqh, dql);
  two_prod(qd0, T, ph, pl);
  two_sum(dqh, -ph, d1h, d1l);
  d1l = __fadd_rn(d1l, __fsub_rn(dql, pl));
  two_sum(qd1, -qd0, d2h, d2l);
  float t3h, t3l, mh, ml, b2h, b2l, b3h, b3l;
  two_prod(3.0f, d1h, t3h, t3l);
  t3l = fmaf(3.0f, d1l, t3l);
  two_prod(d2h, T, mh, ml);
  ml = fmaf(d2l, T, ml);
  two_sum(t3h, -mh, b2h, b2l);
  b2 = __fadd_rn(b2h, __fadd_rn(b2l, __fsub_rn(t3l, ml)));
  two_sum(mh, -2.0f * d1h, b3h, b3l);
  b3 = __fadd_rn(b3h, __fadd_rn(b3l, __fsub_rn(ml, 2.0f * d1l)));
  b1 = ph;
}

// coefficients from an edge held in shared memory as two packed states
// (sh[0..6] = q0, sh[8..14] = qd0, sh[16..22] = q1, sh[24..30] = qd1)
template <bool ACC>
__device__ __forceinline__ void cubic_coef_sh(const float* sh, float T, Cubic& c) {
  c.iT = 1.0f / T;
  c.iT2 = c.iT * c.iT;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    c.q0[j] = sh[j];
    joint_coef<ACC>(sh[j], sh[8 + j], sh[16 + j], sh[24 + j], T, c.b1[j], c.b2[j], c.b3[j]);
  }
}

template <bool ACC>
__device__ __forceinline__ void cubic_coef(const EdgeStates& e, float T, Cubic& c) {
  c.iT = 1.0f / T;
  c.iT2 = c.iT * c.iT;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    c.q0[j] = e.q0[j];
    joint_coef<ACC>(e.q0[j], e.qd0[j], e.q1[j], e.qd1[j], T, c.b1[j], c.b2[j], c.b3[j]);
  }
}

// sigma, sigma_dot, sigma_ddot of joint j at normalised time u
__device__ __forceinline__ void cubic_eval(const Cubic& c, int j, float u, float& q, float& v,
                                           float& a) {
  q = fmaf(fmaf(fmaf(c.b3[j], u, c.b2[j]), u, c.b1[j]), u, c.q0[j]);
  v = fmaf(fmaf(3.0f * c.b3[j], u, 2.0f * c.b2[j]), u, c.b1[j]) * c.iT;
  a = fmaf(6.0f * c.b3[j], u, 2.0f * c.b2[j]) * c.iT2;
}

// The same coefficients held in shared memory, one column per lane
// (element (f, lane) at p[32 f]): frees ~30 registers in the hot loop.
#define FN_CUBIC_WORDS 30
struct CubicLane {
  float* p;  // &buf[lane] of a [FN_CUBIC_WORDS][32] per-warp buffer
  __device__ __forceinline__ float q0(int j) const { return p[32 * j]; }
  __device__ __forceinline__ float b1(int j) const { return p[32 * (7 + j)]; }
  __device__ __forceinline__ float b2(int j) const { return p[32 * (14 + j)]; }
  __device__ __forceinline__ float b3(int j) const { return p[32 * (21 + j)]; }
  __device__ __forceinline__ float iT() const { return p[32 * 28]; }
  __device__ __forceinline__ float iT2() const { return p[32 * 29]; }
  __device__ __forceinline__ void store(const Cubic& c) const {
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      p[32 * j] = c.q0[j];
      p[32 * (7 + j)] = c.b1[j];
      p[32 * (14 + j)] = c.b2[j];
      p[32 * (21 + j)] = c.b3[j];
    }
    p[32 * 28] = c.iT;
    p[32 * 29] = c.iT2;
  }
};

__device__ __forceinline__ void cubic_eval(const CubicLane& c, int j, float u, float& q, float& v,
                                           float& a) {
  const float b2 = c.b2(j), b3 = c.b3(j);
  q = fmaf(fmaf(fmaf(b3, u, b2), u, c.b1(j)), u, c.q0(j));
  v = fmaf(fmaf(3.0f * b3, u, 2.0f * b2), u, c.b1(j)) * c.iT();
  a = fmaf(6.0f * b3, u, 2.0f * b2) * c.iT2();
}

// ---------------------------------------------------------------------------
// Elementary functions of the torque evaluation, branch-free and inlined
// once per use (the library versions carry a large-argument path whose code
// is replicated at every call site of the unrolled link loop).
//
// fn_sincos: the hardware sine and cosine (sin.approx / cos.approx); on the
// torque evaluation's angles (a joint value plus its offset, a few radians)
// the absolute error is about 1e-6, an order below the 1e-5 torque tolerance
// (an earlier Cody-Waite reduction with Taylor polynomials, accurate to the
// single-precision rounding, spent a tenth of the scan's instructions).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fn_sincos(float x, float* s, float* c) { __sincosf(x, s, c); }

// exp(x) = 2^(x log2 e) on the hardware base-2 exponential (ex2.approx,
// relative error ~2^-22 on its argument's exact value); the product
// x log2 e adds |x| ulp of relative error, 6e-6 at |x| = 100
__device__ __forceinline__ float fn_exp(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x * 1.44269504088896340736f));
  return y;
}

// 1/x on the hardware reciprocal (rcp.approx, relative error ~2^-23)
__device__ __forceinline__ float fn_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ---------------------------------------------------------------------------
// Eq. (torque) at one sample of the cubic.
//   forward (links 1..7):
//     w_j   = R^T w_{j-1} + qd_j z
//     dw_j  = R^T dw_{j-1} + (R^T w_{j-1}) x qd_j z + qdd_j z
//     dv_j  = R^T (dw_{j-1} x p_j + w_{j-1} x (w_{j-1} x p_j) + dv_{j-1})
//     dvc_j = dw_j x c_j + w_j x (w_j x c_j) + dv_j
//     F_j = m_j dvc_j,   N_j = I_j dw_j + w_j x I_j w_j
//   backward (links 7..1):
//     f_j = R_{j+1} f_{j+1} + F_j
//     n_j = N_j + R_{j+1} n_{j+1} + c_j x F_j + p_{j+1} x R_{j+1} f_{j+1}
//     tau_j = n_j . z + I_m,j qdd_j + tau_f,j(qd_j)
// Each tau_j is handed to `sink(j, tau_j, qd_j)` as soon as the inward pass
// produces it, so no torque array is kept.
// ---------------------------------------------------------------------------
// Link wrenches of the outward pass, kept until the inward pass.  RegWrench
// holds them in registers; LaneWrench in a per-lane column of shared memory
// (42 words x 32 lanes per warp), which frees ~42 registers for occupancy.
struct RegWrench {
  float Fx[7], Fy[7], Fz[7], Nx[7], Ny[7], Nz[7];
  __device__ __forceinline__ void put(int j, float fx, float fy, float fz, float nx, float ny,
                                      float nz) {
    Fx[j] = fx; Fy[j] = fy; Fz[j] = fz; Nx[j] = nx; Ny[j] = ny; Nz[j] = nz;
  }
  __device__ __forceinline__ void get(int j, float& fx, float& fy, float& fz, float& nx,
                                      float& ny, float& nz) const {
    fx = Fx[j]; fy = Fy[j]; fz = Fz[j]; nx = Nx[j]; ny = Ny[j]; nz = Nz[j];
  }
};
#define FN_WRENCH_WORDS 42
struct LaneWrench {
  float* p;  // &buf[lane] of a [FN_WRENCH_WORDS][32] per-warp buffer
  __device__ __forceinline__ void put(int j, float fx, float fy, float fz, float nx, float ny,
                                      float nz) const {
    p[32 * (6 * j + 0)] = fx; p[32 * (6 * j + 1)] = fy; p[32 * (6 * j + 2)] = fz;
    p[32 * (6 * j + 3)] = nx; p[32 * (6 * j + 4)] = ny; p[32 * (6 * j + 5)] = nz;
  }
  __device__ __forceinline__ void get(int j, float& fx, float& fy, float& fz, float& nx,
                                      float& ny, float& nz) const {
    fx = p[32 * (6 * j + 0)]; fy = p[32 * (6 * j + 1)]; fz = p[32 * (6 * j + 2)];
    nx = p[32 * (6 * j + 3)]; ny = p[32 * (6 * j + 4)]; nz = p[32 * (6 * j + 5)];
  }
};

// gs, fs: scale of the gravity and friction terms (1 for Eq. (torque); 0
// gives the mass-matrix-plus-armature product when the velocity is zero)
template <class Coef, class Sink, class Wr = RegWrench>
__device__ __forceinline__ void torque_at(const ArmK& A, const Coef& c, float u, Sink&& sink,
                                          Wr W = Wr(), float gs = 1.f, float fs = 1.f) {
  float qd[7], ex[7];
  float ct[7], st[7];
  float wx = 0.f, wy = 0.f, wz = 0.f;
  float dwx = 0.f, dwy = 0.f, dwz = 0.f;
  float ax = A.g0x * gs, ay = A.g0y * gs, az = A.g0z * gs;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    float q, v, acc;
    cubic_eval(c, j, u, q, v, acc);
    qd[j] = v;
    // armature and friction (logistic; ex2 / rcp: relative errors ~1e-6 on a
    // term of at most psi1 N m, far inside the torque tolerance)
    const float e = fn_exp(-A.f2[j] * (v + A.f3[j]));
    ex[j] = fmaf(A.arma[j], acc, fs * fmaf(A.f1[j], fn_rcp(1.0f + e), -A.foff[j]));
    fn_sincos(q + A.th0[j], &st[j], &ct[j]);
    const float ca = A.ca[j], sa = A.sa[j];
    const float c_ = ct[j], s_ = st[j];
    // u = dw_prev x p + w_prev x (w_prev x p) + dv_prev   (frame j-1)
    const float px = A.px[j], py = A.py[j], pz = A.pz[j];
    float ux, uy, uz;
    if (j == 0) {
      ux = ax; uy = ay; uz = az;  // w_prev = dw_prev = 0 at the base
    } else {
      const float tx = wy * pz - wz * py, ty = wz * px - wx * pz, tz = wx * py - wy * px;
      ux = (dwy * pz - dwz * py) + (wy * tz - wz * ty) + ax;
      uy = (dwz * px - dwx * pz) + (wz * tx - wx * tz) + ay;
      uz = (dwx * py - dwy * px) + (wx * ty - wy * tx) + az;
    }
    // R^T v = Rz(-theta) Rx(-alpha) v
    float r1 = fmaf(ca, uy, sa * uz);
    float r2 = fmaf(-sa, uy, ca * uz);
    ax = fmaf(c_, ux, s_ * r1);
    ay = fmaf(-s_, ux, c_ * r1);
    az = r2;
    float Rwx = 0.f, Rwy = 0.f, Rwz = 0.f, Rdx = 0.f, Rdy = 0.f, Rdz = 0.f;
    if (j > 0) {
      r1 = fmaf(ca, wy, sa * wz);
      r2 = fmaf(-sa, wy, ca * wz);
      Rwx = fmaf(c_, wx, s_ * r1);
      Rwy = fmaf(-s_, wx, c_ * r1);
      Rwz = r2;
      r1 = fmaf(ca, dwy, sa * dwz);
      r2 = fmaf(-sa, dwy, ca * dwz);
      Rdx = fmaf(c_, dwx, s_ * r1);
      Rdy = fmaf(-s_, dwx, c_ * r1);
      Rdz = r2;
    }
    wx = Rwx; wy = Rwy; wz = Rwz + v;
    dwx = fmaf(Rwy, v, Rdx);
    dwy = fmaf(-Rwx, v, Rdy);
    dwz = Rdz + acc;
    // COM acceleration and link wrench
    const float cx = A.cx[j], cy = A.cy[j], cz = A.cz[j];
    const float wcx = wy * cz - wz * cy, wcy = wz * cx - wx * cz, wcz = wx * cy - wy * cx;
    const float vcx = (dwy * cz - dwz * cy) + (wy * wcz - wz * wcy) + ax;
    const float vcy = (dwz * cx - dwx * cz) + (wz * wcx - wx * wcz) + ay;
    const float vcz = (dwx * cy - dwy * cx) + (wx * wcy - wy * wcx) + az;
    const float m = A.m[j];
    const float Iwx = A.Ix[j] * wx, Iwy = A.Iy[j] * wy, Iwz = A.Iz[j] * wz;
    W.put(j, m * vcx, m * vcy, m * vcz, fmaf(A.Ix[j], dwx, wy * Iwz - wz * Iwy),
          fmaf(A.Iy[j], dwy, wz * Iwx - wx * Iwz), fmaf(A.Iz[j], dwz, wx * Iwy - wy * Iwx));
  }
  float fx = 0.f, fy = 0.f, fz = 0.f, nx = 0.f, ny = 0.f, nz = 0.f;
#pragma unroll
  for (int j = 6; j >= 0; --j) {
    float Rfx = 0.f, Rfy = 0.f, Rfz = 0.f, Rnx = 0.f, Rny = 0.f, Rnz = 0.f;
    float pRx = 0.f, pRy = 0.f, pRz = 0.f;
    if (j < 6) {
      // R_{j+1} v = Rx(alpha_{j+1}) Rz(theta_{j+1}) v
      const float ca = A.ca[j + 1], sa = A.sa[j + 1], c_ = ct[j + 1], s_ = st[j + 1];
      float u0 = fmaf(c_, fx, -s_ * fy), u1 = fmaf(s_, fx, c_ * fy), u2 = fz;
      Rfx = u0; Rfy = fmaf(ca, u1, -sa * u2); Rfz = fmaf(sa, u1, ca * u2);
      u0 = fmaf(c_, nx, -s_ * ny); u1 = fmaf(s_, nx, c_ * ny); u2 = nz;
      Rnx = u0; Rny = fmaf(ca, u1, -sa * u2); Rnz = fmaf(sa, u1, ca * u2);
      const float px = A.px[j + 1], py = A.py[j + 1], pz = A.pz[j + 1];
      pRx = py * Rfz - pz * Rfy; pRy = pz * Rfx - px * Rfz; pRz = px * Rfy - py * Rfx;
    }
    const float cx = A.cx[j], cy = A.cy[j], cz = A.cz[j];
    float Fx, Fy, Fz, Nx, Ny, Nz;
    W.get(j, Fx, Fy, Fz, Nx, Ny, Nz);
    const float cFx = cy * Fz - cz * Fy, cFy = cz * Fx - cx * Fz, cFz = cx * Fy - cy * Fx;
    fx = Fx + Rfx; fy = Fy + Rfy; fz = Fz + Rfz;
    nx = Nx + Rnx + cFx + pRx;
    ny = Ny + Rny + cFy + pRy;
    nz = Nz + Rnz + cFz + pRz;
    sink(j, nz + ex[j], qd[j]);
  }
}

// ---------------------------------------------------------------------------
// Eq. (torque) with the link loops rolled: the same recursion and the same
// arithmetic per link as torque_at, one copy of the link body instead of
// seven, for the warp-per-edge kernels whose state machine around the torque
// evaluation does not fit the instruction cache next to seven unrolled
// links.  The per-link constants come from a shared-memory table (LinkTab,
// warp-uniform addresses: broadcast loads); the outward pass leaves, per
// link, the wrench, cos / sin of the joint angle, the joint velocity and the
// armature-plus-friction term in the lane's column of a LaneLink buffer for
// the inward pass.  The base link is evaluated with the general formulas on
// zero velocities (exactly the base case's values).
// ---------------------------------------------------------------------------
#define FN_LINK_F4 5   // float4 per link in the table
struct LinkTab {
  const float4* p;     // [7][FN_LINK_F4] in shared memory
  // (ca, sa, px, py) (pz, th0, m, cx) (cy, cz, Ix, Iy) (Iz, arma, f1, f2) (f3, foff, inv_tau, 0)
};

// fill the table (thread 0 of the block; the caller synchronises)
__device__ __forceinline__ void fill_links(const ArmK& A, float4* t) {
  if (threadIdx.x != 0) return;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    t[FN_LINK_F4 * j + 0] = make_float4(A.ca[j], A.sa[j], A.px[j], A.py[j]);
    t[FN_LINK_F4 * j + 1] = make_float4(A.pz[j], A.th0[j], A.m[j], A.cx[j]);
    t[FN_LINK_F4 * j + 2] = make_float4(A.cy[j], A.cz[j], A.Ix[j], A.Iy[j]);
    t[FN_LINK_F4 * j + 3] = make_float4(A.Iz[j], A.arma[j], A.f1[j], A.f2[j]);
    t[FN_LINK_F4 * j + 4] = make_float4(A.f3[j], A.foff[j], A.inv_tau[j], 0.f);
  }
}

#define FN_LINK_WORDS 70   // 10 per link: F (3), N (3), cos, sin, qd, armature + friction
struct LaneLink {
  float* p;  // &buf[lane] of a [FN_LINK_WORDS][32] per-warp buffer
  __device__ __forceinline__ void put(int j, int k, float v) const { p[32 * (10 * j + k)] = v; }
  __device__ __forceinline__ float get(int j, int k) const { return p[32 * (10 * j + k)]; }
};

// sink(j, tau_j, qd_j, 1 / tau_max_j) in the inward order j = 6..0
template <class Coef, class Sink>
__device__ __forceinline__ void torque_at_rolled(const ArmK& A, LinkTab L, const Coef& c, float u,
                                                 Sink&& sink, LaneLink W, float gs = 1.f,
                                                 float fs = 1.f) {
  float wx = 0.f, wy = 0.f, wz = 0.f;
  float dwx = 0.f, dwy = 0.f, dwz = 0.f;
  float ax = A.g0x * gs, ay = A.g0y * gs, az = A.g0z * gs;
#pragma unroll 1
  for (int j = 0; j < 7; ++j) {
    const float4 l0 = L.p[FN_LINK_F4 * j + 0], l1 = L.p[FN_LINK_F4 * j + 1];
    const float4 l2 = L.p[FN_LINK_F4 * j + 2], l3 = L.p[FN_LINK_F4 * j + 3];
    const float4 l4 = L.p[FN_LINK_F4 * j + 4];
    const float ca = l0.x, sa = l0.y, px = l0.z, py = l0.w, pz = l1.x;
    float q, v, acc;
    cubic_eval(c, j, u, q, v, acc);
    const float e = fn_exp(-l3.w * (v + l4.x));
    W.put(j, 9, fmaf(l3.y, acc, fs * fmaf(l3.z, fn_rcp(1.0f + e), -l4.y)));
    W.put(j, 8, v);
    float s_, c_;
    fn_sincos(q + l1.y, &s_, &c_);
    W.put(j, 6, c_);
    W.put(j, 7, s_);
    // u = dw_prev x p + w_prev x (w_prev x p) + dv_prev   (frame j-1)
    const float tx = wy * pz - wz * py, ty = wz * px - wx * pz, tz = wx * py - wy * px;
    const float ux = (dwy * pz - dwz * py) + (wy * tz - wz * ty) + ax;
    const float uy = (dwz * px - dwx * pz) + (wz * tx - wx * tz) + ay;
    const float uz = (dwx * py - dwy * px) + (wx * ty - wy * tx) + az;
    // R^T v = Rz(-theta) Rx(-alpha) v
    float r1 = fmaf(ca, uy, sa * uz);
    float r2 = fmaf(-sa, uy, ca * uz);
    ax = fmaf(c_, ux, s_ * r1);
    ay = fmaf(-s_, ux, c_ * r1);
    az = r2;
    r1 = fmaf(ca, wy, sa * wz);
    r2 = fmaf(-sa, wy, ca * wz);
    const float Rwx = fmaf(c_, wx, s_ * r1), Rwy = fmaf(-s_, wx, c_ * r1), Rwz = r2;
    r1 = fmaf(ca, dwy, sa * dwz);
    r2 = fmaf(-sa, dwy, ca * dwz);
    const float Rdx = fmaf(c_, dwx, s_ * r1), Rdy = fmaf(-s_, dwx, c_ * r1), Rdz = r2;
    wx = Rwx; wy = Rwy; wz = Rwz + v;
    dwx = fmaf(Rwy, v, Rdx);
    dwy = fmaf(-Rwx, v, Rdy);
    dwz = Rdz + acc;
    // COM acceleration and link wrench
    const float cx = l1.w, cy = l2.x, cz = l2.y;
    const float wcx = wy * cz - wz * cy, wcy = wz * cx - wx * cz, wcz = wx * cy - wy * cx;
    const float vcx = (dwy * cz - dwz * cy) + (wy * wcz - wz * wcy) + ax;
    const float vcy = (dwz * cx - dwx * cz) + (wz * wcx - wx * wcz) + ay;
    const float vcz = (dwx * cy - dwy * cx) + (wx * wcy - wy * wcx) + az;
    const float m = l1.z, Ix = l2.z, Iy = l2.w, Iz = l3.x;
    const float Iwx = Ix * wx, Iwy = Iy * wy, Iwz = Iz * wz;
    W.put(j, 0, m * vcx);
    W.put(j, 1, m * vcy);
    W.put(j, 2, m * vcz);
    W.put(j, 3, fmaf(Ix, dwx, wy * Iwz - wz * Iwy));
    W.put(j, 4, fmaf(Iy, dwy, wz * Iwx - wx * Iwz));
    W.put(j, 5, fmaf(Iz, dwz, wx * Iwy - wy * Iwx));
  }
  float fx = 0.f, fy = 0.f, fz = 0.f, nx = 0.f, ny = 0.f, nz = 0.f;
#pragma unroll 1
  for (int j = 6; j >= 0; --j) {
    // R_{j+1} (f, n) and p_{j+1} x R_{j+1} f; zero for the last link (f = n = 0)
    const int jc = j < 6 ? j + 1 : 6;
    const float4 k0 = L.p[FN_LINK_F4 * jc + 0], k1 = L.p[FN_LINK_F4 * jc + 1];
    const float ca = k0.x, sa = k0.y, c_ = W.get(jc, 6), s_ = W.get(jc, 7);
    float u0 = fmaf(c_, fx, -s_ * fy), u1 = fmaf(s_, fx, c_ * fy), u2 = fz;
    const float Rfx = u0, Rfy = fmaf(ca, u1, -sa * u2), Rfz = fmaf(sa, u1, ca * u2);
    u0 = fmaf(c_, nx, -s_ * ny); u1 = fmaf(s_, nx, c_ * ny); u2 = nz;
    const float Rnx = u0, Rny = fmaf(ca, u1, -sa * u2), Rnz = fmaf(sa, u1, ca * u2);
    const float px = k0.z, py = k0.w, pz = k1.x;
    const float pRx = py * Rfz - pz * Rfy, pRy = pz * Rfx - px * Rfz, pRz = px * Rfy - py * Rfx;
    const float4 m1 = L.p[FN_LINK_F4 * j + 1], m2 = L.p[FN_LINK_F4 * j + 2];
    const float cx = m1.w, cy = m2.x, cz = m2.y;
    const float Fx = W.get(j, 0), Fy = W.get(j, 1), Fz = W.get(j, 2);
    const float Nx = W.get(j, 3), Ny = W.get(j, 4), Nz = W.get(j, 5);
    const float cFx = cy * Fz - cz * Fy, cFy = cz * Fx - cx * Fz, cFz = cx * Fy - cy * Fx;
    fx = Fx + Rfx; fy = Fy + Rfy; fz = Fz + Rfz;
    nx = Nx + Rnx + cFx + pRx;
    ny = Ny + Rny + cFy + pRy;
    nz = Nz + Rnz + cFz + pRz;
    sink(j, nz + W.get(j, 9), W.get(j, 8), L.p[FN_LINK_F4 * j + 4].z);
  }
}

// ---------------------------------------------------------------------------
// Eq. (torque) at two samples of the same cubic per lane, u = (u.x, u.y):
// torque_at_rolled's recursion with every floating-point step done on both
// samples at once by the paired FP32 instructions (fma / add / mul .f32x2;
// each half rounds like the scalar instruction).  Per-link constants come
// from LinkTab2, whose entries hold each constant twice, (x, x, y, y), so a
// pair is one load; the outward pass leaves its per-link state in a
// LaneLink2 column of float2, the coefficients come from a CubicLane2 column
// of duplicated pairs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// a x b - the pair form of the scalar cross products (a_y b_z - a_z b_y, ...)
__device__ __forceinline__ void cross2(float2 ax, float2 ay, float2 az, float2 bx, float2 by,
                                       float2 bz, float2& cx, float2& cy, float2& cz) {
  cx = fma2(ay, bz, neg2(mul2(az, by)));
  cy = fma2(az, bx, neg2(mul2(ax, bz)));
  cz = fma2(ax, by, neg2(mul2(ay, bx)));
}

#define FN_LINK2_F4 10   // float4 per link in the paired table
struct LinkTab2 {
  const float4* p;       // [7][FN_LINK2_F4] in shared memory
  // (ca ca sa sa) (px px py py) (pz pz th0 th0) (m m cx cx) (cy cy cz cz)
  // (Ix Ix Iy Iy) (Iz Iz arma arma) (f1 f1 f2 f2) (f3 f3 foff foff) (inv_tau 0 0 0)
};

// fill the paired table (thread 0 of the block; the caller synchronises)
__device__ __forceinline__ void fill_links2(const ArmK& A, float4* t) {
  if (threadIdx.x != 0) return;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    float4* e = t + FN_LINK2_F4 * j;
    e[0] = make_float4(A.ca[j], A.ca[j], A.sa[j], A.sa[j]);
    e[1] = make_float4(A.px[j], A.px[j], A.py[j], A.py[j]);
    e[2] = make_float4(A.pz[j], A.pz[j], A.th0[j], A.th0[j]);
    e[3] = make_float4(A.m[j], A.m[j], A.cx[j], A.cx[j]);
    e[4] = make_float4(A.cy[j], A.cy[j], A.cz[j], A.cz[j]);
    e[5] = make_float4(A.Ix[j], A.Ix[j], A.Iy[j], A.Iy[j]);
    e[6] = make_float4(A.Iz[j], A.Iz[j], A.arma[j], A.arma[j]);
    e[7] = make_float4(A.f1[j], A.f1[j], A.f2[j], A.f2[j]);
    e[8] = make_float4(A.f3[j], A.f3[j], A.foff[j], A.foff[j]);
    e[9] = make_float4(A.inv_tau[j], 0.f, 0.f, 0.f);
  }
}

// Per-link record of the outward pass, kept until the inward pass: F (3),
// N (3), cos, sin, qd, armature + friction, as pairs (10 float2).
#define FN_REC2 10
// LaneLink2 keeps the records in the lane's column of a shared-memory buffer
// ([FN_LINK2_WORDS / 2][32] float2 per warp).
#define FN_LINK2_WORDS 140
struct LaneLink2 {
  float2* p;  // &buf[lane]
  __device__ __forceinline__ void store(int j, const float2 (&r)[FN_REC2]) const {
#pragma unroll
    for (int k = 0; k < FN_REC2; ++k) p[32 * (FN_REC2 * j + k)] = r[k];
  }
  __device__ __forceinline__ void stored() const {}
  __device__ __forceinline__ void load(int j, float2 (&r)[FN_REC2]) const {
#pragma unroll
    for (int k = 0; k < FN_REC2; ++k) r[k] = p[32 * (FN_REC2 * j + k)];
  }
};

// the cubic's coefficients, each stored twice (one float2 per word)
#define FN_CUBIC2_WORDS 60
struct CubicLane2 {
  float2* p;  // &buf[lane] of a [FN_CUBIC_WORDS][32] float2 per-warp buffer
  __device__ __forceinline__ float2 q0(int j) const { return p[32 * j]; }
  __device__ __forceinline__ float2 b1(int j) const { return p[32 * (7 + j)]; }
  __device__ __forceinline__ float2 b2(int j) const { return p[32 * (14 + j)]; }
  __device__ __forceinline__ float2 b3(int j) const { return p[32 * (21 + j)]; }
  __device__ __forceinline__ float2 iT() const { return p[32 * 28]; }
  __device__ __forceinline__ float2 iT2() const { return p[32 * 29]; }
  __device__ __forceinline__ void store(const Cubic& c) const { store2(c, c); }
  // different cubics in the two halves (x: cx, y: cy)
  __device__ __forceinline__ void store2(const Cubic& cx, const Cubic& cy) const {
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      p[32 * j] = make_float2(cx.q0[j], cy.q0[j]);
      p[32 * (7 + j)] = make_float2(cx.b1[j], cy.b1[j]);
      p[32 * (14 + j)] = make_float2(cx.b2[j], cy.b2[j]);
      p[32 * (21 + j)] = make_float2(cx.b3[j], cy.b3[j]);
    }
    p[32 * 28] = make_float2(cx.iT, cy.iT);
    p[32 * 29] = make_float2(cx.iT2, cy.iT2);
  }
};

// sink(j, tau_j, qd_j, 1 / tau_max_j) in the inward order j = 6..0, tau_j and
// qd_j as pairs; gs, fs: per-half gravity and friction scales.  Stash:
// store(j, rec) / stored() / load(j, rec) (LaneLink2, or a tensor-memory
// column block); every lane of the warp must call this.
template <class Sink, class Stash>
__device__ __forceinline__ void torque_at_pair(const ArmK& A, LinkTab2 L, CubicLane2 c, float2 u,
                                               Sink&& sink, Stash W, float2 gs = {1.f, 1.f},
                                               float2 fs2 = {1.f, 1.f}) {
  float2 wx = dup2(0.f), wy = dup2(0.f), wz = dup2(0.f);
  float2 dwx = dup2(0.f), dwy = dup2(0.f), dwz = dup2(0.f);
  float2 ax = mul2(dup2(A.g0x), gs), ay = mul2(dup2(A.g0y), gs), az = mul2(dup2(A.g0z), gs);
  const float2 iT = c.iT(), iT2 = c.iT2();
#pragma unroll 1
  for (int j = 0; j < 7; ++j) {
    const float4* t = L.p + FN_LINK2_F4 * j;
    const float4 t0 = t[0], t1 = t[1], t2 = t[2], t3 = t[3], t4 = t[4];
    const float4 t5 = t[5], t6 = t[6], t7 = t[7], t8 = t[8];
    const float2 ca = lo2(t0), sa = hi2(t0), px = lo2(t1), py = hi2(t1), pz = lo2(t2);
    float2 rec[FN_REC2];
    // sigma, sigma_dot, sigma_ddot at both samples
    const float2 b1 = c.b1(j), b2 = c.b2(j), b3 = c.b3(j), tb2 = add2(b2, b2);
    const float2 q = fma2(fma2(fma2(b3, u, b2), u, b1), u, c.q0(j));
    const float2 v = mul2(fma2(fma2(mul2(dup2(3.0f), b3), u, tb2), u, b1), iT);
    const float2 acc = mul2(fma2(mul2(dup2(6.0f), b3), u, tb2), iT2);
    // armature and friction
    const float2 x = mul2(neg2(hi2(t7)), add2(v, lo2(t8)));
    const float2 xe = mul2(x, dup2(1.44269504088896340736f));
    float ex, ey;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ex) : "f"(xe.x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ey) : "f"(xe.y));
    const float2 rc = make_float2(fn_rcp(1.0f + ex), fn_rcp(1.0f + ey));
    rec[9] = fma2(hi2(t6), acc, mul2(fs2, fma2(lo2(t7), rc, neg2(hi2(t8)))));
    rec[8] = v;
    float2 s_, c_;
    {
      const float2 th = add2(q, hi2(t2));
      fn_sincos(th.x, &s_.x, &c_.x);
      fn_sincos(th.y, &s_.y, &c_.y);
    }
    rec[6] = c_;
    rec[7] = s_;
    // u = dw_prev x p + w_prev x (w_prev x p) + dv_prev   (frame j-1)
    float2 tx, ty, tz, gx, gy, gz, hx, hy, hz;
    cross2(wx, wy, wz, px, py, pz, tx, ty, tz);
    cross2(dwx, dwy, dwz, px, py, pz, gx, gy, gz);
    cross2(wx, wy, wz, tx, ty, tz, hx, hy, hz);
    const float2 ux = add2(add2(gx, hx), ax);
    const float2 uy = add2(add2(gy, hy), ay);
    const float2 uz = add2(add2(gz, hz), az);
    // R^T v = Rz(-theta) Rx(-alpha) v
    const float2 ns = neg2(s_), nsa = neg2(sa);
    float2 r1 = fma2(ca, uy, mul2(sa, uz));
    float2 r2 = fma2(nsa, uy, mul2(ca, uz));
    ax = fma2(c_, ux, mul2(s_, r1));
    ay = fma2(ns, ux, mul2(c_, r1));
    az = r2;
    r1 = fma2(ca, wy, mul2(sa, wz));
    r2 = fma2(nsa, wy, mul2(ca, wz));
    const float2 Rwx = fma2(c_, wx, mul2(s_, r1)), Rwy = fma2(ns, wx, mul2(c_, r1)), Rwz = r2;
    r1 = fma2(ca, dwy, mul2(sa, dwz));
    r2 = fma2(nsa, dwy, mul2(ca, dwz));
    const float2 Rdx = fma2(c_, dwx, mul2(s_, r1)), Rdy = fma2(ns, dwx, mul2(c_, r1)), Rdz = r2;
    wx = Rwx; wy = Rwy; wz = add2(Rwz, v);
    dwx = fma2(Rwy, v, Rdx);
    dwy = fma2(neg2(Rwx), v, Rdy);
    dwz = add2(Rdz, acc);
    // COM acceleration and link wrench
    const float2 cx = hi2(t3), cy = lo2(t4), cz = hi2(t4);
    float2 wcx, wcy, wcz, dcx, dcy, dcz, ex2_, ey2_, ez2_;
    cross2(wx, wy, wz, cx, cy, cz, wcx, wcy, wcz);
    cross2(dwx, dwy, dwz, cx, cy, cz, dcx, dcy, dcz);
    cross2(wx, wy, wz, wcx, wcy, wcz, ex2_, ey2_, ez2_);
    const float2 m = lo2(t3), Ix = lo2(t5), Iy = hi2(t5), Iz = lo2(t6);
    rec[0] = mul2(m, add2(add2(dcx, ex2_), ax));
    rec[1] = mul2(m, add2(add2(dcy, ey2_), ay));
    rec[2] = mul2(m, add2(add2(dcz, ez2_), az));
    const float2 Iwx = mul2(Ix, wx), Iwy = mul2(Iy, wy), Iwz = mul2(Iz, wz);
    float2 kx, ky, kz;
    cross2(wx, wy, wz, Iwx, Iwy, Iwz, kx, ky, kz);
    rec[3] = fma2(Ix, dwx, kx);
    rec[4] = fma2(Iy, dwy, ky);
    rec[5] = fma2(Iz, dwz, kz);
    W.store(j, rec);
  }
  W.stored();
  float2 fx = dup2(0.f), fy = dup2(0.f), fz = dup2(0.f);
  float2 nx = dup2(0.f), ny = dup2(0.f), nz = dup2(0.f);
  float2 cn = dup2(1.f), sn = dup2(0.f);   // cos, sin of joint j + 1 (any value for j = 6)
#pragma unroll 1
  for (int j = 6; j >= 0; --j) {
    float2 rec[FN_REC2];
    W.load(j, rec);
    // R_{j+1} (f, n) and p_{j+1} x R_{j+1} f; zero for the last link (f = n = 0)
    const int jc = j < 6 ? j + 1 : 6;
    const float4* t = L.p + FN_LINK2_F4 * jc;
    const float4 k0 = t[0], k1 = t[1], k2 = t[2];
    const float2 ca = lo2(k0), sa = hi2(k0), nsa = neg2(sa), ns = neg2(sn);
    float2 u0 = fma2(cn, fx, mul2(ns, fy)), u1 = fma2(sn, fx, mul2(cn, fy)), u2 = fz;
    const float2 Rfx = u0, Rfy = fma2(ca, u1, mul2(nsa, u2)), Rfz = fma2(sa, u1, mul2(ca, u2));
    u0 = fma2(cn, nx, mul2(ns, ny)); u1 = fma2(sn, nx, mul2(cn, ny)); u2 = nz;
    const float2 Rnx = u0, Rny = fma2(ca, u1, mul2(nsa, u2)), Rnz = fma2(sa, u1, mul2(ca, u2));
    float2 pRx, pRy, pRz;
    cross2(lo2(k1), hi2(k1), lo2(k2), Rfx, Rfy, Rfz, pRx, pRy, pRz);
    const float4* m = L.p + FN_LINK2_F4 * j;
    const float4 m3 = m[3], m4 = m[4];
    float2 cFx, cFy, cFz;
    cross2(hi2(m3), lo2(m4), hi2(m4), rec[0], rec[1], rec[2], cFx, cFy, cFz);
    fx = add2(rec[0], Rfx); fy = add2(rec[1], Rfy); fz = add2(rec[2], Rfz);
    nx = add2(add2(add2(rec[3], Rnx), cFx), pRx);
    ny = add2(add2(add2(rec[4], Rny), cFy), pRy);
    nz = add2(add2(add2(rec[5], Rnz), cFz), pRz);
    cn = rec[6];
    sn = rec[7];
    sink(j, add2(nz, rec[9]), rec[8], m[9].x);
  }
}

// one configuration (q, qd, qdd) handed to torque_at as its "sample"
struct PointCoef {
  float q[7], qd[7], qdd[7];
};

__device__ __forceinline__ void cubic_eval(const PointCoef& c, int j, float, float& q, float& v,
                                           float& a) {
  q = c.q[j];
  v = c.qd[j];
  a = c.qdd[j];
}

// Eq. (torque) at an end of the cubic as a function of the duration T.  At
// u = 0 and u = 1 the position and velocity are the edge's end state,
// whatever T; only the acceleration depends on T, and it is
//   u = 0:  qdd = 6 (q1 - q0) / T^2 - (4 qd0 + 2 qd1) / T,
//   u = 1:  qdd = -6 (q1 - q0) / T^2 + (4 qd1 + 2 qd0) / T.
// Eq. (torque) is affine in qdd (mass matrix plus armature times qdd, plus
// the velocity, gravity and friction terms at the end state), so
//   tau(T) = alpha / T^2 + beta / T + gamma
// with alpha = (M(q) + I_m) a and beta = (M(q) + I_m) b for the two vectors
// above, and gamma = tau(q, qd, 0).  One part per call: part 0 writes gamma
// to out[14..20] and the end velocity to out[21..27]; parts 1 and 2 write
// alpha to out[0..6] and beta to out[7..13], evaluated with the gravity and
// friction terms scaled to zero, so that the torque of (q, 0, x) is
// (M(q) + I_m) x.
__device__ __forceinline__ void end_torque_part(const ArmK& A, const float* q0, const float* qd0,
                                                const float* q1, const float* qd1, int end,
                                                int part, float* out) {
  PointCoef pc;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    const float d = q1[j] - q0[j];
    const float a = end ? -6.0f * d : 6.0f * d;
    const float b = end ? fmaf(4.0f, qd1[j], 2.0f * qd0[j]) : -fmaf(4.0f, qd0[j], 2.0f * qd1[j]);
    pc.q[j] = end ? q1[j] : q0[j];
    pc.qd[j] = part == 0 ? (end ? qd1[j] : qd0[j]) : 0.f;
    pc.qdd[j] = part == 0 ? 0.f : (part == 1 ? a : b);
  }
  const int o = part == 0 ? 14 : 7 * (part - 1);
  const float on = part == 0 ? 1.f : 0.f;
  torque_at(A, pc, 0.f, [&](int j, float t, float) { out[o + j] = t; }, RegWrench(), on, on);
  if (part == 0)
#pragma unroll
    for (int j = 0; j < 7; ++j) out[21 + j] = pc.qd[j];
}

// ratios of one sample at normalised time u: rho_tau(s) and rho_P(s)
template <class Coef, class Wr = RegWrench>
__device__ __forceinline__ void sample_ratios(const ArmK& A, const Coef& c, float u, float& rt,
                                              float& rp, Wr W = Wr()) {
  float r = 0.f, pw = 0.f;
  torque_at(
      A, c, u,
      [&](int j, float tau, float v) {
        r = fmaxf(r, fabsf(tau) * A.inv_tau[j]);
        pw = fmaf(tau, v, pw);
      },
      W);
  rt = r;
  rp = fabsf(pw) * A.inv_w;
}

// position-dependent velocity bound qdbar_j(q)
__device__ __forceinline__ float taper(const ArmK& A, int j, float q) {
  float m = fminf(q - A.q_lo[j], A.q_hi[j] - q);
  m = fmaxf(m, 0.f);
  return fminf(A.qd_max[j], sqrtf(A.taper2a[j] * m));
}

// rho_v contribution of joint j: exact extremum of the quadratic velocity
// (b1 + 2 b2 u + 3 b3 u^2)/T over u in [0, 1] (ends and the stationary point
// u* = -b2/(3 b3)), each compared with the taper at the joint's position at
// that same time.
__device__ __forceinline__ float rho_v_joint(const ArmK& A, const Cubic& c, int j) {
  float best = 0.f;
  float cand[3] = {0.f, 1.f, -1.f};
  if (c.b3[j] != 0.f) {
    const float us = -c.b2[j] / (3.0f * c.b3[j]);
    if (us > 0.f && us < 1.f) cand[2] = us;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float u = cand[i];
    if (u < 0.f) continue;
    float pos, vel, acc;
    cubic_eval(c, j, u, pos, vel, acc);
    const float b = taper(A, j, pos);
    float r;
    if (b > 0.f) r = fabsf(vel) / b;
    else r = (vel != 0.f) ? INFINITY : 0.f;
    best = fmaxf(best, r);
  }
  return best;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

}  // namespace fn
