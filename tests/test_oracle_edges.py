"""Pins of the oracle's cubic edge, feasibility ratios and duration scan.

* Def. "Cubic edge": boundary conditions in closed form; sigma_ddot(0) equals
  the controller law of Eq. (controller) (the same cubic refitted from the
  measured state), sigma_ddot is linear in t, derivatives match differences.
* Def. "Feasibility Check" on a one-link, gravity-free rest-to-rest edge:
  rho_tau = 6 I |dq| / (T^2 tau_max), peak speed 1.5 |dq| / T, and the power
  samples at t_s = s T/(S-1) in closed form (pins the sample placement).
* Def. "Minimum feasible time": the scan's k* equals the closed-form
  first index with T_k >= sqrt(6 I |dq| / tau_max); on random 7-DOF edges
  every index below k* is infeasible and k* is feasible; caps and invalid
  inputs follow the documented codes.
"""
import math

import numpy as np
import pytest

from paper_2609_22608_gb300 import synth


def test_cubic_boundary_conditions(orc):
    rng = np.random.default_rng(0)
    for _ in range(20):
        q0, qd0, q1, qd1 = rng.uniform(-2, 2, (4, 7))
        T = rng.uniform(0.05, 2.0)
        s, sd, _ = orc.cubic(q0, qd0, q1, qd1, T, 0.0)
        assert np.allclose(s, q0, atol=1e-12) and np.allclose(sd, qd0, atol=1e-12)
        s, sd, _ = orc.cubic(q0, qd0, q1, qd1, T, T)
        assert np.allclose(s, q1, atol=1e-11) and np.allclose(sd, qd1, atol=1e-10)


def test_cubic_start_acceleration_is_controller_law(orc):
    """Eq. (controller) refits the cubic from (q, qd) to (q_g, qd_g, T); its
    acceleration at the start is 6(q_g - q)/T^2 - (4 qd + 2 qd_g)/T."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        q, qd, qg, qdg = rng.uniform(-2, 2, (4, 7))
        T = rng.uniform(0.05, 2.0)
        _, _, sdd = orc.cubic(q, qd, qg, qdg, T, 0.0)
        law = 6 * (qg - q) / T**2 - (4 * qd + 2 * qdg) / T
        assert np.allclose(sdd, law, rtol=1e-12, atol=1e-9)


def test_cubic_derivatives(orc):
    rng = np.random.default_rng(2)
    q0, qd0, q1, qd1 = rng.uniform(-2, 2, (4, 7))
    T = 0.7
    h = 1e-6
    for t in (0.0 + 2 * h, 0.2, 0.5, T - 2 * h):
        s_p, sd_p, sdd_p = orc.cubic(q0, qd0, q1, qd1, T, t + h)
        s_m, sd_m, sdd_m = orc.cubic(q0, qd0, q1, qd1, T, t - h)
        s, sd, sdd = orc.cubic(q0, qd0, q1, qd1, T, t)
        assert np.allclose((s_p - s_m) / (2 * h), sd, atol=1e-6)
        assert np.allclose((sd_p - sd_m) / (2 * h), sdd, atol=1e-5)
    # acceleration is linear in t
    a = [orc.cubic(q0, qd0, q1, qd1, T, t)[2] for t in (0.0, 0.3, 0.6)]
    assert np.allclose(a[1] - a[0], a[2] - a[1], atol=1e-9)


def one_link_arm(arm, izz=0.04, m=1.5, c=(0.2, 0.1, 0.0), arma=0.1, tau_max=20.0):
    """7-DOF arm whose joints 2-7 carry no mass: joint 1 is a vertical axis
    (no gravity torque), no friction, wide joint box."""
    a = {k: (v.astype(np.float64).copy() if isinstance(v, np.ndarray) else v) for k, v in arm.items()}
    a["dh_alpha"][0] = 0.0
    a["mass"][:] = 0.0
    a["inertia"][:] = 0.0
    a["com"][:] = 0.0
    a["armature"][:] = 0.0
    a["fric"][:, 0] = 0.0
    a["mass"][0] = m
    a["com"][0] = c
    a["inertia"][0] = [0.01, 0.02, izz]
    a["armature"][0] = arma
    a["tau_max"][:] = 1.0
    a["tau_max"][0] = tau_max
    a["w_max"] = 1e9
    a["q_lo"][:] = -50.0
    a["q_hi"][:] = 50.0
    a["qd_max"][:] = 1e3
    a["qd_taper_a"][:] = 1e6  # the taper never binds inside the box
    a = {k: (v.astype(np.float32) if isinstance(v, np.ndarray) else v) for k, v in a.items()}
    a["w_max"] = np.float32(1e9)
    return a


def _itot(a):
    m = float(a["mass"][0]); c = a["com"][0].astype(np.float64)
    return float(a["inertia"][0][2]) + m * (c[0] ** 2 + c[1] ** 2) + float(a["armature"][0])


def _rest_edge(dq, q0=0.3):
    s0 = np.zeros((1, 16), np.float32)
    s1 = np.zeros((1, 16), np.float32)
    s0[0, 0] = q0
    s1[0, 0] = q0 + dq
    return s0, s1


def test_rest_to_rest_rho_closed_form(orc, arm):
    a = one_link_arm(arm)
    I = _itot(a)
    for dq in (0.5, -1.3, 2.0):
        s0, s1 = _rest_edge(dq)
        dq32 = float(s1[0, 0]) - float(s0[0, 0])
        for T in (0.3, 0.8, 1.7):
            r = orc.rho_batch(a, s0, s1, [T], 16)[0]
            assert r[0] == pytest.approx(6 * I * abs(dq32) / (T * T * float(a["tau_max"][0])), rel=1e-10)
            assert r[2] == pytest.approx(1.5 * abs(dq32) / T / float(a["qd_max"][0]), rel=1e-10)


@pytest.mark.parametrize("S,fmax", [(2, 0.0), (3, 0.0), (4, 2.0 / 27.0), (5, 3.0 / 32.0)])
def test_power_sample_placement(orc, arm, S, fmax):
    """P(t) = I qdd qd = 36 I dq^2 / T^3 (1-2u) u (1-u) with u = t/T; with
    samples u_s = s/(S-1) the maximum of |(1-2u)u(1-u)| is 0 (S=2,3),
    2/27 (S=4, u=1/3) and 3/32 (S=5, u=1/4)."""
    a = one_link_arm(arm)
    a["w_max"] = np.float32(1.0)
    I = _itot(a)
    s0, s1 = _rest_edge(1.0)
    dq32 = float(s1[0, 0]) - float(s0[0, 0])
    T = 0.9
    r = orc.rho_batch(a, s0, s1, [T], S)[0]
    assert r[1] == pytest.approx(36 * I * dq32**2 / T**3 * fmax, rel=1e-9, abs=1e-12)


def test_scan_matches_closed_form_min_time(orc, arm):
    a = one_link_arm(arm)
    I = _itot(a)
    Tg = synth.duration_grid(64)
    rng = np.random.default_rng(7)
    dqs = rng.uniform(-3, 3, 40)
    s0 = np.zeros((40, 16), np.float32)
    s1 = np.zeros((40, 16), np.float32)
    s1[:, 0] = dqs
    res = orc.time_edges(a, s0, s1, Tg, 32)
    for e in range(40):
        dq = float(s1[e, 0])
        Tstar = math.sqrt(6 * I * abs(dq) / float(a["tau_max"][0]))
        ks = [k for k in range(64) if float(Tg[k]) >= Tstar]
        expect = ks[0] if ks else -1
        # stay clear of the boundary so rounding cannot decide it
        if expect > 0:
            assert abs(float(Tg[expect]) / Tstar - 1) > 1e-9
        assert res["k_star"][e] == expect
        if expect >= 0:
            assert res["T_star"][e] == Tg[expect]
            assert res["ok"][e] == 1


def test_scan_first_feasible_invariant(orc, arm):
    s0, s1 = synth.random_edges(arm, 48, 3)
    Tg = synth.duration_grid(32)
    S = 16
    res = orc.time_edges(arm, s0, s1, Tg, S)
    for k in range(32):
        r = orc.rho_batch(arm, s0, s1, np.full(48, float(Tg[k])), S)
        feas = (r[:, 0] <= 1) & (r[:, 1] <= 1)
        ks = res["k_star"]
        assert np.all(~feas[(ks > k) | (ks == -1)])      # everything before k* fails
        hit = ks == k
        assert np.all(feas[hit])                           # k* itself passes
        if hit.any():
            assert np.allclose(res["rho3"][hit], r[hit])
            assert np.all(res["ok"][hit] == (r[hit, 2] <= 1))


def test_scan_cap_and_invalid(orc, arm):
    s0, s1 = synth.random_edges(arm, 16, 4)
    Tg = synth.duration_grid(32)
    free = orc.time_edges(arm, s0, s1, Tg, 16)
    cap = np.full(16, 0.8, np.float32)
    capped = orc.time_edges(arm, s0, s1, Tg, 16, T_cap=cap)
    for e in range(16):
        k = free["k_star"][e]
        if k >= 0 and Tg[k] <= 0.8:
            assert capped["k_star"][e] == k
        else:
            assert capped["k_star"][e] == -1 and np.isinf(capped["T_star"][e])
    bad0 = s0.copy(); bad0[3, 2] = np.nan
    r = orc.time_edges(arm, bad0, s1, Tg, 16)
    assert r["k_star"][3] == -2 and r["ok"][3] == 0
    Tf = np.full(16, 0.5, np.float32); Tf[5] = 0.0; Tf[6] = -1.0; Tf[7] = np.inf
    r = orc.time_edges(arm, s0, s1, Tg, 16, mode=1, T_fixed=Tf)
    assert list(r["k_star"][5:8]) == [-2, -2, -2]
    ok_fixed = (r["rho3"][:, 0] <= 1) & (r["rho3"][:, 1] <= 1) & (r["rho3"][:, 2] <= 1)
    good = np.ones(16, bool); good[5:8] = False
    assert np.all(r["ok"][good] == ok_fixed[good])


def test_rho_v_exact_extremum(orc, arm):
    """Away from the joint limits the taper is the constant qd_max, so rho_v
    must equal the dense-sampled max |sigma_dot| / qd_max."""
    a = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in arm.items()}
    a["q_lo"] = np.full(7, -100, np.float32)
    a["q_hi"] = np.full(7, 100, np.float32)
    s0, s1 = synth.random_edges(arm, 20, 9)
    for e in range(20):
        for T in (0.1, 0.6, 1.9):
            r = orc.rho_batch(a, s0[e:e + 1], s1[e:e + 1], [T], 4)[0]
            ts = np.linspace(0, T, 200001)
            best = 0.0
            for j in range(7):
                q0, qd0, q1, qd1 = (float(s0[e, j]), float(s0[e, 8 + j]), float(s1[e, j]), float(s1[e, 8 + j]))
                d1 = q1 - q0 - qd0 * T; d2 = qd1 - qd0
                v = qd0 + 2 * (3 * d1 / T**2 - d2 / T) * ts + 3 * (d2 / T**2 - 2 * d1 / T**3) * ts**2
                best = max(best, np.abs(v).max() / float(a["qd_max"][j]))
            assert r[2] >= best * (1 - 1e-12)
            assert r[2] == pytest.approx(best, rel=1e-7)
