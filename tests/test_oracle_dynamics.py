"""Pins of the oracle's Eq. (torque) against physics that does not use RNEA.

* Lagrange's equations, tau = d/dt dL/dqd - dL/dq, with L built from forward
  kinematics written here with 4x4 homogeneous transforms (modified DH) and
  differentiated numerically in FP64 -- on 1-, 2-, 3-link chains and the full
  7-link arm.
* The single-link pendulum closed form.
* Static torques equal the gradient of the potential energy.
* Eq. (friction): tau_f(0) = 0 (stated beside the equation), its saturation
  limits, its midpoint, and monotonicity.
* Eq. (torque) adds exactly I_m qdd + tau_f(qd) to the rigid-body part.
"""
import math

import numpy as np
import pytest

from paper_2609_22608_gb300 import synth


def _dh(alpha, a, theta, d):
    ca, sa, ct, st = math.cos(alpha), math.sin(alpha), math.cos(theta), math.sin(theta)
    Rx = np.array([[1, 0, 0, 0], [0, ca, -sa, 0], [0, sa, ca, 0], [0, 0, 0, 1.0]])
    Tx = np.eye(4); Tx[0, 3] = a
    Rz = np.array([[ct, -st, 0, 0], [st, ct, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1.0]])
    Tz = np.eye(4); Tz[2, 3] = d
    return Rx @ Tx @ Rz @ Tz


def _frames(arm, q):
    n = arm["dof"]
    T = np.eye(4)
    out = []
    for j in range(n):
        T = T @ _dh(float(arm["dh_alpha"][j]), float(arm["dh_a"][j]),
                    float(q[j] + arm["dh_theta0"][j]), float(arm["dh_d"][j]))
        out.append(T.copy())
    return out


def _lagrangian(arm, q, qd):
    """L = KE - PE with link velocities from the geometric Jacobian of the
    homogeneous-transform FK (no recursion shared with RNEA)."""
    n = arm["dof"]
    Fs = _frames(arm, q)
    g = arm["gravity"].astype(np.float64)
    ke = pe = 0.0
    for i in range(n):
        R = Fs[i][:3, :3]
        pc = Fs[i][:3, 3] + R @ arm["com"][i].astype(np.float64)
        v = np.zeros(3)
        w = np.zeros(3)
        for j in range(i + 1):
            z = Fs[j][:3, 2]
            o = Fs[j][:3, 3]
            v += np.cross(z, pc - o) * qd[j]
            w += z * qd[j]
        m = float(arm["mass"][i])
        Iw = R @ np.diag(arm["inertia"][i].astype(np.float64)) @ R.T
        ke += 0.5 * m * v @ v + 0.5 * w @ Iw @ w
        pe += -m * g @ pc
    return ke - pe


def _lagrange_tau(arm, q, qd, qdd):
    n = arm["dof"]
    h = 1e-5

    def dL_dqd(qq, vv):
        out = np.zeros(n)
        for i in range(n):
            e = np.zeros(n); e[i] = 1.0
            # KE is quadratic in qd: the central difference is exact up to rounding
            out[i] = (_lagrangian(arm, qq, vv + e) - _lagrangian(arm, qq, vv - e)) / 2.0
        return out

    def dL_dq(qq, vv):
        out = np.zeros(n)
        for i in range(n):
            e = np.zeros(n); e[i] = h
            out[i] = (_lagrangian(arm, qq + e, vv) - _lagrangian(arm, qq - e, vv)) / (2 * h)
        return out

    ht = 1e-4
    # d/dt along q(t) = q + qd t + qdd t^2 / 2 (fourth-order central difference)
    def p_at(t):
        return dL_dqd(q + qd * t + 0.5 * qdd * t * t, qd + qdd * t)
    ddt = (-p_at(2 * ht) + 8 * p_at(ht) - 8 * p_at(-ht) + p_at(-2 * ht)) / (12 * ht)
    return ddt - dL_dq(q, qd)


@pytest.mark.parametrize("dof", [1, 2, 3, 7])
def test_rnea_matches_lagrange(orc, arm, dof):
    a = synth.arm_with_dof(arm, dof)
    rng = np.random.default_rng(dof)
    for _ in range(4):
        q = rng.uniform(-2, 2, 7)
        qd = rng.uniform(-2, 2, 7)
        qdd = rng.uniform(-5, 5, 7)
        tau = orc.rnea(a, q, qd, qdd)
        ref = _lagrange_tau(a, q[:dof], qd[:dof], qdd[:dof])
        scale = max(np.abs(ref).max(), 1.0)
        assert np.abs(tau - ref).max() <= 1e-6 * scale, (tau, ref)


def test_rnea_lagrange_catches_planted_mistake(orc, arm):
    """The Lagrange pin is sharp enough to see a dropped Coriolis-size term."""
    a = synth.arm_with_dof(arm, 3)
    q = np.array([0.3, -0.7, 1.1, 0, 0, 0, 0])
    qd = np.array([1.5, -1.2, 2.0, 0, 0, 0, 0])
    qdd = np.zeros(7)
    tau = orc.rnea(a, q, qd, qdd)
    ref = _lagrange_tau(a, q[:3], qd[:3], qdd[:3])
    # removing the velocity-dependent part changes the answer by far more than
    # the test tolerance
    tau_static = orc.rnea(a, q, np.zeros(7), qdd)
    assert np.abs(tau - ref).max() < 1e-6 * max(1, np.abs(ref).max())
    assert np.abs(tau_static - ref).max() > 1e-3


def _pendulum_arm(arm, m=2.0, r=0.3, izz=0.05):
    a = synth.arm_with_dof(arm, 1)
    # float64 copies: the closed form below uses exact pi/2 and g
    a = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in a.items()}
    a["dh_alpha"][0] = -math.pi / 2  # horizontal axis
    a["dh_a"] = a["dh_a"].copy(); a["dh_a"][0] = 0.0
    a["dh_d"] = a["dh_d"].copy(); a["dh_d"][0] = 0.0
    a["dh_theta0"] = a["dh_theta0"].copy(); a["dh_theta0"][0] = 0.0
    a["mass"] = a["mass"].copy(); a["mass"][0] = m
    a["com"] = a["com"].copy(); a["com"][0] = [r, 0.0, 0.0]
    a["inertia"] = a["inertia"].copy(); a["inertia"][0] = [0.01, 0.02, izz]
    return a


def test_pendulum_closed_form(orc, arm):
    """alpha_0 = -pi/2 makes joint 1 horizontal: the COM height is -r sin q,
    so tau = (I_zz + m r^2) qdd - m g r cos q for any velocity."""
    m, r, izz, g = 2.0, 0.3, 0.05, 9.81
    a = _pendulum_arm(arm, m, r, izz)
    a["gravity"] = np.array([0, 0, -g])
    for q, qd, qdd in [(0.0, 0.0, 0.0), (0.4, 1.3, -2.0), (-1.2, -3.0, 5.0), (2.5, 0.1, 0.7)]:
        tau = orc.rnea(a, [q] + [0] * 6, [qd] + [0] * 6, [qdd] + [0] * 6)[0]
        expect = (izz + m * r * r) * qdd - m * g * r * math.cos(q)
        assert tau == pytest.approx(expect, rel=1e-12, abs=1e-12)


def test_static_torque_is_potential_gradient(orc, arm):
    rng = np.random.default_rng(3)
    h = 1e-6
    for _ in range(5):
        q = rng.uniform(-2, 2, 7)
        tau = orc.rnea(arm, q, np.zeros(7), np.zeros(7))
        grad = np.zeros(7)
        for i in range(7):
            e = np.zeros(7); e[i] = h
            grad[i] = (-_lagrangian(arm, q + e, np.zeros(7)) + _lagrangian(arm, q - e, np.zeros(7))) / (2 * h)
        assert np.allclose(tau, grad, rtol=1e-7, atol=1e-7)


def test_friction_properties(orc):
    for psi in ([0.5, 10.0, 0.1], [0.3, 50.0, -0.05], [0.05, 5.0, 0.0]):
        p1, p2, p3 = psi
        s0 = 1.0 / (1.0 + math.exp(-p2 * p3))
        assert orc.friction(psi, 0.0) == pytest.approx(0.0, abs=1e-15)   # tau_f(0) = 0
        assert orc.friction(psi, 1e3) == pytest.approx(p1 - p1 * s0, abs=1e-12)
        assert orc.friction(psi, -1e3) == pytest.approx(-p1 * s0, abs=1e-12)
        assert orc.friction(psi, -p3) == pytest.approx(p1 / 2 - p1 * s0, abs=1e-12)
        xs = np.linspace(-3, 3, 301)
        vals = np.array([orc.friction(psi, x) for x in xs])
        assert np.all(np.diff(vals) >= 0)


def test_torque_adds_armature_and_friction(orc, arm):
    rng = np.random.default_rng(5)
    q, qd, qdd = rng.uniform(-1, 1, 7), rng.uniform(-2, 2, 7), rng.uniform(-4, 4, 7)
    full = orc.torque(arm, q, qd, qdd)
    rigid = orc.rnea(arm, q, qd, qdd)
    extra = np.array([arm["armature"][j] * qdd[j] + orc.friction(arm["fric"][j], qd[j]) for j in range(7)])
    assert np.allclose(full - rigid, extra, rtol=1e-12, atol=1e-12)
    # armature enters only the diagonal: d tau_i / d qdd_j changes by I_m,i on i == j
    for j in range(7):
        e = np.zeros(7); e[j] = 1.0
        d_full = orc.torque(arm, q, qd, qdd + e) - full
        d_rigid = orc.rnea(arm, q, qd, qdd + e) - rigid
        diff = d_full - d_rigid
        expect = np.zeros(7); expect[j] = arm["armature"][j]
        assert np.allclose(diff, expect, atol=1e-12)


def test_end_sample_torque_is_affine_in_inverse_duration(orc, arm):
    """At the ends of the cubic (t = 0 and t = T) the position and velocity
    are the edge's end states for every T, and Eq. (torque) there is
    alpha / T^2 + beta / T + gamma: alpha and beta the torque increments of
    the accelerations +-6 (q1 - q0) and -(4 qd0 + 2 qd1) or (4 qd1 + 2 qd0)
    at zero velocity, gamma the torque at the end state with zero
    acceleration.  The probe of the edge pipeline checks durations from
    this split."""
    rng = np.random.default_rng(17)
    s0, s1 = synth.random_edges(arm, 6, 23)
    for e in range(6):
        q0, qd0 = s0[e, :7].astype(np.float64), s0[e, 8:15].astype(np.float64)
        q1, qd1 = s1[e, :7].astype(np.float64), s1[e, 8:15].astype(np.float64)
        d = q1 - q0
        for end, (q, qd, a, b) in enumerate([(q0, qd0, 6 * d, -(4 * qd0 + 2 * qd1)),
                                             (q1, qd1, -6 * d, 4 * qd1 + 2 * qd0)]):
            z = np.zeros(7)
            g0 = orc.torque(arm, q, z, z)
            alpha = orc.torque(arm, q, z, a) - g0
            beta = orc.torque(arm, q, z, b) - g0
            gamma = orc.torque(arm, q, qd, z)
            for T in rng.uniform(0.05, 1.5, 4):
                pos, vel, acc = orc.cubic(q0, qd0, q1, qd1, T, end * T)
                assert np.allclose(pos, q, rtol=0, atol=1e-12)
                assert np.allclose(vel, qd, rtol=0, atol=1e-12)
                tau = orc.torque(arm, pos, vel, acc)
                split = alpha / T ** 2 + beta / T + gamma
                assert np.allclose(split, tau, rtol=1e-10, atol=1e-9 * np.abs(tau).max())


def test_end_sample_split_does_not_cancel_near_decisions(orc, arm):
    """Near a probe decision (the largest end-sample torque ratio within
    [0.5, 2]), the three terms of alpha / T^2 + beta / T + gamma add up to
    at most a few torque limits, so the single-precision rounding of the
    split (relative ~1e-7 per term and operation) moves a ratio by far less
    than the 1e-4 margin within which decisions may differ."""
    grid = synth.duration_grid(128)
    s0, s1 = synth.random_edges(arm, 120, 5)
    tm = np.asarray(arm["tau_max"], np.float64)
    worst, near = 0.0, 0
    for e in range(s0.shape[0]):
        q0, qd0 = s0[e, :7].astype(np.float64), s0[e, 8:15].astype(np.float64)
        q1, qd1 = s1[e, :7].astype(np.float64), s1[e, 8:15].astype(np.float64)
        d = q1 - q0
        z = np.zeros(7)
        for q, qd, a, b in [(q0, qd0, 6 * d, -(4 * qd0 + 2 * qd1)),
                            (q1, qd1, -6 * d, 4 * qd1 + 2 * qd0)]:
            g0 = orc.torque(arm, q, z, z)
            alpha = orc.torque(arm, q, z, a) - g0
            beta = orc.torque(arm, q, z, b) - g0
            gamma = orc.torque(arm, q, qd, z)
            for T in grid:
                ratio = np.abs(alpha / T ** 2 + beta / T + gamma) / tm
                if 0.5 <= ratio.max() <= 2.0:
                    near += 1
                    amp = (np.abs(alpha) / T ** 2 + np.abs(beta) / T + np.abs(gamma)) / tm
                    worst = max(worst, float(amp.max()))
    assert near > 1000
    assert worst < 20.0          # x ~1e-6 relative rounding << 1e-4
