"""Pins of the oracle's tracking controller (Eq. controller) and of the
full-resolution recheck of a plan's edges (Sec. IV-E).

* Unclipped, the controller's acceleration is the initial acceleration of the
  cubic refitted from the measured state to the rendezvous (Def. "Cubic
  edge" at t = 0), and its command is Eq. (torque) there.
* One link turning about a vertical axis, no friction: tau_1 = I qdd_des in
  closed form, the other joints carry nothing.
* The acceleration box keeps the velocity inside the taper after one control
  period; the torque, power and slew clips leave the command on their bound
  (power: same direction); invalid inputs give NaN and flag 0x80.
* Recheck: a parked edge (equal states at rest) needs only the static torque
  at every sample (rho_tau = max |g(q)| / tau_max, rho_P = rho_v = 0) and its
  clearance is that of the one configuration.
"""
import numpy as np
import pytest

from paper_2609_22608_gb300 import synth
from tests.test_oracle_edges import _itot, one_link_arm


def _states(arm, B, seed, speed=0.3):
    rng = np.random.default_rng(seed)
    lo, hi = np.asarray(arm["q_lo"], np.float64), np.asarray(arm["q_hi"], np.float64)
    st = np.zeros((B, 16), np.float32)
    c, h = 0.5 * (lo + hi), 0.5 * (hi - lo)
    st[:, :7] = c + rng.uniform(-0.5, 0.5, (B, 7)) * h
    st[:, 8:15] = rng.uniform(-speed, speed, (B, 7)) * np.asarray(arm["qd_max"], np.float64)
    return st


def _relaxed(arm):
    a = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in arm.items()}
    a["tau_max"] = np.full(7, 1e6, np.float32)
    a["w_max"] = np.float32(1e9)
    return a


def test_unclipped_is_refitted_cubic_and_torque(orc, arm):
    a = _relaxed(arm)
    B = 24
    x, g = _states(a, B, 1), _states(a, B, 2)
    T = np.random.default_rng(3).uniform(0.3, 1.5, B).astype(np.float32)
    out = orc.controller_torque(a, x, g, T, 1e-3)
    assert np.all(out["flags"] == 0)
    for b in range(B):
        q0, qd0 = x[b, :7].astype(np.float64), x[b, 8:15].astype(np.float64)
        q1, qd1 = g[b, :7].astype(np.float64), g[b, 8:15].astype(np.float64)
        _, _, sdd = orc.cubic(q0, qd0, q1, qd1, float(T[b]), 0.0)
        assert np.allclose(out["qdd"][b], sdd, rtol=1e-12, atol=1e-9)
        tau = orc.torque(a, q0, qd0, sdd)
        assert np.allclose(out["tau"][b], tau, rtol=1e-12, atol=1e-9)


def test_one_link_closed_form(orc, arm):
    a = _relaxed(one_link_arm(arm))
    I = _itot(a)
    rng = np.random.default_rng(5)
    B = 16
    x = np.zeros((B, 16), np.float32)
    g = np.zeros((B, 16), np.float32)
    x[:, 0] = rng.uniform(-0.5, 0.5, B)
    x[:, 8] = rng.uniform(-0.5, 0.5, B)
    g[:, 0] = rng.uniform(-0.5, 0.5, B)
    g[:, 8] = rng.uniform(-0.5, 0.5, B)
    T = rng.uniform(0.4, 1.2, B).astype(np.float32)
    out = orc.controller_torque(a, x, g, T, 1e-3)
    q, qd, qg, qdg = (x[:, 0].astype(np.float64), x[:, 8].astype(np.float64),
                      g[:, 0].astype(np.float64), g[:, 8].astype(np.float64))
    Td = T.astype(np.float64)
    acc = 6 * (qg - q) / Td**2 - (4 * qd + 2 * qdg) / Td
    assert np.allclose(out["qdd"][:, 0], acc, rtol=1e-12)
    assert np.allclose(out["tau"][:, 0], I * acc, rtol=1e-9, atol=1e-12)
    assert np.allclose(out["tau"][:, 1:], 0.0, atol=1e-12)


def test_acceleration_box_tapers_velocity(orc, arm):
    a = _relaxed(arm)
    dt = 1e-3
    x = _states(a, 8, 7, speed=0.0)
    g = _states(a, 8, 8, speed=0.0)
    hi = np.asarray(a["q_hi"], np.float64)
    # joint 2 next to its upper limit and moving toward it, rendezvous beyond it
    x[:, 1] = (hi[1] - 1e-4).astype(np.float32)
    x[:, 9] = 0.5
    g[:, 1] = hi[1]
    g[:, 9] = 1.0
    T = np.full(8, 0.2, np.float32)
    out = orc.controller_torque(a, x, g, T, dt)
    qb = float(x[0, 1])
    bound = min(float(a["qd_max"][1]), np.sqrt(2 * float(a["qd_taper_a"][1]) * max(0.0, float(hi[1]) - qb)))
    # the clipped acceleration brings the velocity exactly onto the taper
    assert np.allclose(0.5 + out["qdd"][:, 1] * dt, bound, rtol=1e-9, atol=1e-12)
    assert np.all(out["flags"] & 1)


def test_torque_power_and_slew_clips(orc, arm):
    B = 32
    x, g = _states(arm, B, 11, speed=0.8), _states(arm, B, 12, speed=0.8)
    T = np.full(B, 0.08, np.float32)           # fast: large torques
    tight = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in arm.items()}
    tight["w_max"] = np.float32(1e9)
    out = orc.controller_torque(tight, x, g, T, 1e-3)
    tmax = np.asarray(tight["tau_max"], np.float64)
    assert np.all(np.abs(out["tau"]) <= tmax + 1e-12)
    assert np.any(out["flags"] & 2)
    raw = orc.controller_torque(_relaxed(arm), x, g, T, 1e-3)
    clipped = np.abs(raw["tau"]) > tmax
    assert np.allclose(np.abs(out["tau"][clipped]), np.broadcast_to(tmax, out["tau"].shape)[clipped])
    assert np.allclose(out["tau"][~clipped], raw["tau"][~clipped], rtol=1e-12, atol=1e-12)
    # power: the torque-clipped command scaled onto W_max, direction kept
    low = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in tight.items()}
    low["w_max"] = np.float32(5.0)
    pw = orc.controller_torque(low, x, g, T, 1e-3)
    qd = x[:, 8:15].astype(np.float64)
    P = np.sum(pw["tau"] * qd, axis=1)
    scaled = (pw["flags"] & 4) != 0
    assert scaled.any()
    assert np.allclose(np.abs(P[scaled]), 5.0, rtol=1e-9)
    Pin = np.sum(out["tau"] * qd, axis=1)
    ratio = pw["tau"][scaled] / out["tau"][scaled]
    assert np.allclose(ratio, (5.0 / np.abs(Pin[scaled]))[:, None], rtol=1e-9)
    # slew: within rate * dt of the previous command, on the bound where clipped
    prev = np.zeros((B, 7), np.float32)
    rate = np.full(7, 1000.0)
    sl = orc.controller_torque(low, x, g, T, 1e-3, tau_prev=prev, rate=rate)
    assert np.all(np.abs(sl["tau"]) <= 1.0 + 1e-12)
    hit = (sl["flags"] & 8) != 0
    assert hit.any()
    moved = np.abs(pw["tau"]) > 1.0
    assert np.allclose(np.abs(sl["tau"][moved]), 1.0)


def test_controller_invalid_inputs(orc, arm):
    x, g = _states(arm, 4, 21), _states(arm, 4, 22)
    x[1, 3] = np.nan
    g[2, 10] = np.inf
    T = np.array([0.5, 0.5, 0.5, 0.0], np.float32)
    out = orc.controller_torque(arm, x, g, T, 1e-3)
    assert out["flags"][0] != 0x80
    assert np.all(out["flags"][1:] == 0x80)
    assert np.all(np.isnan(out["tau"][1:]))


def test_recheck_parked_edge(orc, arm):
    rng = np.random.default_rng(31)
    E = 12
    x = _states(arm, E, 31, speed=0.0)
    T = rng.uniform(0.1, 1.0, E).astype(np.float32)
    obs = np.array([[0.5, 0.1, 0.4, 0.1], [0.3, -0.4, 0.6, 0.08]], np.float32)
    res = orc.check_edges(arm, x, x, T, 64, 16, obs, 0.02)
    tmax = np.asarray(arm["tau_max"], np.float64)
    for e in range(E):
        q = x[e, :7].astype(np.float64)
        tg = orc.torque(arm, q, np.zeros(7), np.zeros(7))
        assert res["rho3"][e, 0] == pytest.approx(np.max(np.abs(tg) / tmax), rel=1e-12)
        assert res["rho3"][e, 1] == 0.0 and res["rho3"][e, 2] == 0.0
        one = orc.edge_clearance(arm, x[e], x[e], 1.0, 2, obs)
        assert res["clearance"][e] == pytest.approx(one, rel=1e-12)
        expect = res["rho3"][e, 0] <= 1 and one >= 0.02
        assert res["ok"][e] == int(expect)
    none = orc.check_edges(arm, x, x, T, 64, 16, np.zeros((0, 4), np.float32), 0.02)
    assert np.all(np.isinf(none["clearance"]))


def test_recheck_invalid_and_resolution(orc, arm):
    s0, s1 = synth.random_edges(arm, 16, 41)
    T = np.full(16, 0.8, np.float32)
    T[3] = -1.0
    s0[5, 2] = np.nan
    res = orc.check_edges(arm, s0, s1, T, 256, 64, np.zeros((0, 4), np.float32), 0.02)
    assert np.isnan(res["rho3"][3]).all() and np.isnan(res["rho3"][5]).all()
    assert res["ok"][3] == 0 and res["ok"][5] == 0
    # a finer resolution samples a superset of points when (S-1) divides (S'-1)
    coarse = orc.check_edges(arm, s0, s1, T, 64, 16, np.zeros((0, 4), np.float32), 0.02)
    fine = orc.check_edges(arm, s0, s1, T, 253, 16, np.zeros((0, 4), np.float32), 0.02)
    good = np.isfinite(coarse["rho3"][:, 0])
    assert np.all(fine["rho3"][good, :2] >= coarse["rho3"][good, :2] - 1e-12)
