"""Pins of the oracle's gradient refinement of a rendezvous node
(oracle/refine.py; the reading is in its module docstring):

* the objective's dependence on the arrival time T: central differences of
  the oracle's Eq. (objective) against the derivative written out from
  Eq. (terms) in closed form;
* the step rule on a known concave objective (a quadratic in z with a
  known maximiser, the angle coordinates measured around the circle): the
  iterates approach the maximiser and the objective never decreases;
* a node whose neighbourhood is undefined is left unchanged;
* on a real rendezvous node of an oracle round (a goal reached from an
  approach node), the refined node's J is at least the original's and the
  node still passes the exact check; refinement improves it here.
"""
import math

import numpy as np
import pytest

import oracle.plan as OP
import oracle.refine as R
from paper_2609_22608_gb300 import synth

F32 = np.float32


def _dJ_dT(pr, T, vrel, nu):
    """d/dT of Eq. (objective) at fixed v_rel and nu, from Eq. (terms)."""
    sp, sv, sa = pr["sig_p"], pr["sig_v"], pr["sig_a"]
    s = math.sqrt(sp * sp + (sv * T) ** 2 + (0.5 * sa * T * T) ** 2)
    ds = (sv * sv * T + 0.5 * sa * sa * T ** 3) / s
    a = pr["r_catch"] / math.sqrt(2.0)
    x = a / s
    dlog_obj = (2.0 / math.sqrt(math.pi)) * math.exp(-x * x) * (-a * ds / (s * s)) / math.erf(x)
    xdz = abs(pr["v0"][2] + pr["g"][2] * pr["t_fall"])
    u = (pr["t_fall"] - T) * xdz / s
    du = -xdz / s - (pr["t_fall"] - T) * xdz * ds / (s * s)
    phi = math.exp(-0.5 * u * u) / math.sqrt(2 * math.pi)
    Phi = 0.5 * math.erfc(-u / math.sqrt(2.0))
    dlog_in = phi / Phi * du
    dlog_arm = -pr["lam"] * max(nu - pr["nu0"], 0.0) * (1.0 - pr["nu0"] / nu) if nu > 0 else 0.0
    return pr["w_p"] * dlog_obj + pr["w_r"] * dlog_in + pr["w_x"] * dlog_arm


@pytest.mark.parametrize("nu", [0.5, 0.97])
def test_objective_time_derivative_closed_form(orc, arm, nu):
    pr = synth.make_problem(synth.random_toss(arm, 0, reach=None))
    for T in (0.25, 0.45, 0.7):
        h = 1e-5
        fd = (orc.objective(pr, T + h, 5.0, nu) - orc.objective(pr, T - h, 5.0, nu)) / (2 * h)
        assert fd == pytest.approx(_dJ_dT(pr, T, 5.0, nu), rel=1e-5, abs=1e-6)


def _circ(z, zs):
    d = np.array(z, np.float64) - zs
    for i in R.ANGLE:
        d[i] = (d[i] + 0.5) % 1.0 - 0.5
    return d


def test_step_rule_climbs_a_known_objective():
    zs = np.array([0.4, 0.5, 0.97, 0.3, 0.6, 0.5, 0.5, 0.2, 0.7])
    f = lambda z: -float(np.sum(_circ(z, zs) ** 2))          # noqa: E731
    z0 = np.array([0.45, 0.47, 0.02, 0.32, 0.57, 0.53, 0.48, 0.24, 0.66])  # z2 across the wrap
    seen = []
    F = lambda z: seen.append(f(z)) or seen[-1]               # noqa: E731
    z, Fz, acc = R.refine(F, f, z0)
    assert acc >= 2
    assert np.linalg.norm(_circ(z, zs)) < 0.2 * np.linalg.norm(_circ(z0, zs))
    assert Fz == pytest.approx(f(z)) and Fz >= f(z0)


def test_undefined_neighbourhood_is_left_alone():
    z0 = np.full(9, 0.5)
    f = lambda z: 0.0 if np.array_equal(z, z0) else -np.inf   # noqa: E731
    z, Fz, acc = R.refine(f, f, z0)
    assert acc == 0 and np.array_equal(z, z0) and Fz == 0.0


def test_refine_real_rendezvous_node(orc, arm):
    toss = synth.random_toss(arm, 11)
    root = synth.random_states(arm, 1, 5011)[0]
    pr = synth.make_problem(toss, root=root)
    # uniform draws (no mixture component) with their chart parameters z
    st, Tq, vr, valid, Z = orc.sample_goals_density(arm, pr, dict(C=0, w_u=0.25), 111, 0, 0, 0, 256)
    zs = [Z[c] for c in np.nonzero(valid)[0][:6]]
    assert zs
    S = 32
    improved = 0
    for c, z0 in zip(np.nonzero(valid)[0][:6], zs):
        ok, g, Treq, vrel, vb = orc.goal_chart(arm, pr, z0)
        assert ok and np.allclose(g, st[c])
        # an approach node 0.1 s earlier on the goal's own velocity, at t = T_req - 0.1
        appr = g.astype(np.float64).copy()
        appr[:7] -= 0.1 * appr[8:15]
        t_par = float(F32(Treq - 0.1))
        out = R.refine_node(arm, pr, z0, appr.astype(F32), t_par, 0.0, S)
        J0, feas0, _ = R.node_eval(arm, pr, z0, appr.astype(F32), t_par, 0.0, S)
        if not feas0:
            continue
        assert out["feasible"]
        assert out["J"] >= J0
        improved += out["J"] > J0 + 1e-6
    assert improved >= 1
