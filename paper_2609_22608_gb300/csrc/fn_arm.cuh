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
// Cubic coefficients of one edge at duration T:
//   sigma(t) = q0 + qd0 t + c2 t^2 + c3 t^3
//   c2 = 3 d1/T^2 - d2/T,  c3 = d2/T^2 - 2 d1/T^3,
//   d1 = q1 - q0 - qd0 T,  d2 = qd1 - qd0.
// ---------------------------------------------------------------------------
struct Cubic {
  float q0[7], qd0[7], c2[7], c3[7];
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

__device__ __forceinline__ bool edge_finite(const EdgeStates& e) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 7; ++j)
    ok = ok && isfinite(e.q0[j]) && isfinite(e.qd0[j]) && isfinite(e.q1[j]) && isfinite(e.qd1[j]);
  return ok;
}

// coefficients from an edge held in shared memory as two packed states
// (sh[0..6] = q0, sh[8..14] = qd0, sh[16..22] = q1, sh[24..30] = qd1)
__device__ __forceinline__ void cubic_coef_sh(const float* sh, float T, Cubic& c) {
  const float iT = 1.0f / T;
  const float iT2 = iT * iT;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    const float q0 = sh[j], qd0 = sh[8 + j], q1 = sh[16 + j], qd1 = sh[24 + j];
    const float d1 = fmaf(-qd0, T, q1 - q0);
    const float d2 = qd1 - qd0;
    c.q0[j] = q0;
    c.qd0[j] = qd0;
    c.c2[j] = fmaf(3.0f * d1, iT2, -d2 * iT);
    c.c3[j] = fmaf(-2.0f * d1, iT2 * iT, d2 * iT2);
  }
}

__device__ __forceinline__ void cubic_coef(const EdgeStates& e, float T, Cubic& c) {
  const float iT = 1.0f / T;
  const float iT2 = iT * iT;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    const float d1 = fmaf(-e.qd0[j], T, e.q1[j] - e.q0[j]);
    const float d2 = e.qd1[j] - e.qd0[j];
    c.q0[j] = e.q0[j];
    c.qd0[j] = e.qd0[j];
    c.c2[j] = fmaf(3.0f * d1, iT2, -d2 * iT);
    c.c3[j] = fmaf(-2.0f * d1, iT2 * iT, d2 * iT2);
  }
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
template <class Sink>
__device__ __forceinline__ void torque_at(const ArmK& A, const Cubic& c, float t, Sink&& sink) {
  float qd[7], ex[7];
  float ct[7], st[7];
  float Fx[7], Fy[7], Fz[7], Nx[7], Ny[7], Nz[7];
  float wx = 0.f, wy = 0.f, wz = 0.f;
  float dwx = 0.f, dwy = 0.f, dwz = 0.f;
  float ax = A.g0x, ay = A.g0y, az = A.g0z;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    const float q = fmaf(fmaf(fmaf(c.c3[j], t, c.c2[j]), t, c.qd0[j]), t, c.q0[j]);
    const float v = fmaf(fmaf(3.0f * c.c3[j], t, 2.0f * c.c2[j]), t, c.qd0[j]);
    const float acc = fmaf(6.0f * c.c3[j], t, 2.0f * c.c2[j]);
    qd[j] = v;
    // armature and friction (logistic with an IEEE division)
    const float e = expf(-A.f2[j] * (v + A.f3[j]));
    ex[j] = fmaf(A.arma[j], acc, A.f1[j] / (1.0f + e) - A.foff[j]);
    sincosf(q + A.th0[j], &st[j], &ct[j]);
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
    Fx[j] = m * vcx; Fy[j] = m * vcy; Fz[j] = m * vcz;
    const float Iwx = A.Ix[j] * wx, Iwy = A.Iy[j] * wy, Iwz = A.Iz[j] * wz;
    Nx[j] = fmaf(A.Ix[j], dwx, wy * Iwz - wz * Iwy);
    Ny[j] = fmaf(A.Iy[j], dwy, wz * Iwx - wx * Iwz);
    Nz[j] = fmaf(A.Iz[j], dwz, wx * Iwy - wy * Iwx);
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
    const float cFx = cy * Fz[j] - cz * Fy[j], cFy = cz * Fx[j] - cx * Fz[j],
                cFz = cx * Fy[j] - cy * Fx[j];
    fx = Fx[j] + Rfx; fy = Fy[j] + Rfy; fz = Fz[j] + Rfz;
    nx = Nx[j] + Rnx + cFx + pRx;
    ny = Ny[j] + Rny + cFy + pRy;
    nz = Nz[j] + Rnz + cFz + pRz;
    sink(j, nz + ex[j], qd[j]);
  }
}

// ratios of one sample: rho_tau(s) and rho_P(s)
__device__ __forceinline__ void sample_ratios(const ArmK& A, const Cubic& c, float t, float& rt,
                                              float& rp) {
  float r = 0.f, pw = 0.f;
  torque_at(A, c, t, [&](int j, float tau, float v) {
    r = fmaxf(r, fabsf(tau) * A.inv_tau[j]);
    pw = fmaf(tau, v, pw);
  });
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
// qd(t) = qd0 + 2 c2 t + 3 c3 t^2 over [0, T] (ends and stationary point),
// each compared with the taper at the joint's position at that time.
__device__ __forceinline__ float rho_v_joint(const ArmK& A, const Cubic& c, int j, float T) {
  float best = 0.f;
  float cand[3] = {0.f, T, -1.f};
  if (c.c3[j] != 0.f) {
    const float ts = -c.c2[j] / (3.0f * c.c3[j]);
    if (ts > 0.f && ts < T) cand[2] = ts;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float t = cand[i];
    if (t < 0.f) continue;
    const float pos = fmaf(fmaf(fmaf(c.c3[j], t, c.c2[j]), t, c.qd0[j]), t, c.q0[j]);
    const float vel = fmaf(fmaf(3.0f * c.c3[j], t, 2.0f * c.c2[j]), t, c.qd0[j]);
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
