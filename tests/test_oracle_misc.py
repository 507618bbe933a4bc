"""Pins of the oracle's Philox generator, kNN, forward kinematics, goal
chart, objective, arrival-time pruning and clearance."""
import math
import os
from statistics import NormalDist

import numpy as np
import pytest

from paper_2609_22608_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(orc):
    for ctr, key, out in _kat():
        assert list(orc.philox4x32(ctr, key)) == out


def test_paper_constants(arm):
    vals = {}
    for line in open(os.path.join(GOLD, "paper_constants.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, v = line.split()[:2]
        vals[name] = float(v)
    pr = synth.make_problem(synth.random_toss(arm, 0))
    for k in ("a_min", "v_min", "w_v", "v_target", "w_p", "w_r", "w_x", "r_catch", "nu0", "lam",
              "sig_p", "sig_v", "sig_a"):
        assert pr[k] == pytest.approx(vals[k], rel=1e-6), k
    assert float(arm["w_max"]) == vals["w_max"]
    assert float(arm["blade_len"]) == pytest.approx(vals["blade_len"], rel=1e-6)


def _np_knn(tree, queries, k, w, first=1):
    """Independent brute force: numpy distances, lexicographic (d2, index) order."""
    t = tree[first:].astype(np.float64)
    q = queries.astype(np.float64)
    d = ((q[:, None, 0:7] - t[None, :, 0:7]) ** 2).sum(-1) + w * ((q[:, None, 8:15] - t[None, :, 8:15]) ** 2).sum(-1)
    idx = np.arange(first, tree.shape[0])
    out_i = np.zeros((q.shape[0], k), np.int64)
    out_d = np.zeros((q.shape[0], k))
    for b in range(q.shape[0]):
        order = np.lexsort((idx, d[b]))[:k]
        out_i[b] = idx[order]
        out_d[b] = d[b][order]
    return out_i, out_d


def test_knn_brute_force(orc, arm):
    tree = synth.random_states(arm, 300, 1)
    qs = synth.random_states(arm, 40, 2)
    # plant exact ties: duplicate nodes must come back in index order
    tree[200] = tree[17]
    qs[5] = tree[17]
    idx, d2 = orc.knn(tree, qs, 8, 0.1)
    ri, rd = _np_knn(tree, qs, 8, 0.1)
    assert np.array_equal(idx, ri)
    assert np.allclose(d2, rd, rtol=1e-12)
    assert idx[5, 0] == 17 and idx[5, 1] == 200 and d2[5, 0] == 0.0
    # fewer candidates than k: padded with -1 / inf, root excluded
    idx, d2 = orc.knn(tree[:4], qs[:2], 6, 0.1)
    assert np.all(idx[:, 3:] == -1) and np.all(np.isinf(d2[:, 3:]))
    assert not np.any(idx == 0)


def _fk4(arm, q):
    from tests.test_oracle_dynamics import _frames
    return _frames(arm, q)


def test_fk_matches_homogeneous_transforms(orc, arm):
    rng = np.random.default_rng(4)
    for _ in range(5):
        q = rng.uniform(-2, 2, 7)
        R, o = orc.fk(arm, q)
        F = _fk4(arm, q)
        for j in range(7):
            assert np.allclose(R[j], F[j][:3, :3], atol=1e-12)
            assert np.allclose(o[j], F[j][:3, 3], atol=1e-12)
        assert np.allclose(o[7], F[6][:3, 3] + float(arm["flange_d"]) * F[6][:3, 2], atol=1e-12)
        # geometric Jacobian of a point = derivative of that point under FK
        p = o[7] + np.array([0.05, -0.02, 0.1])
        J = orc.jacobian_point(arm, q, p)
        h = 1e-7
        for j in range(7):
            e = np.zeros(7); e[j] = h
            Rp, op = orc.fk(arm, q + e)
            Rm, om = orc.fk(arm, q - e)
            # the point moves rigidly with the end-effector frame
            loc = R[7].T @ (p - o[7])
            dp = ((op[7] + Rp[7] @ loc) - (om[7] + Rm[7] @ loc)) / (2 * h)
            assert np.allclose(J[0:3, j], dp, atol=1e-6)


def _tosses(arm, n=6, reach=synth.REACH):
    return [synth.make_problem(synth.random_toss(arm, s, reach=reach)) for s in range(n)]


def test_goal_chart_samples_lie_on_manifold(orc, arm):
    """Def. 2 / Def. 3: every decoded sample intercepts x(T) with the blade,
    with alignment >= a_min and relative speed >= v_min (up to the IK
    residual), inside the joint box and under the velocity taper."""
    n_acc = 0
    for pr in _tosses(arm):
        st, Tq, vr, valid = orc.sample_goals(arm, pr, 31, 0, 0, 0, 2048)
        g = np.asarray(pr["g"])
        for c in np.nonzero(valid)[0]:
            n_acc += 1
            q, qd, T = st[c, :7], st[c, 8:15], Tq[c]
            assert pr["t_enter"] <= T <= pr["t_fall"]
            x = pr["x0"] + pr["v0"] * T + 0.5 * g * T * T
            xd = pr["v0"] + g * T
            b0, b1 = orc.blade(arm, q)
            u = np.clip((x - b0) @ (b1 - b0) / ((b1 - b0) @ (b1 - b0)), 0, 1)
            assert np.linalg.norm(b0 + u * (b1 - b0) - x) < 6e-4
            J = orc.jacobian_point(arm, q, x)
            v6 = J @ qd
            # minimum-norm joint velocity for the contact point's linear
            # velocity: qd lies in the row space of the 3x7 point Jacobian
            # (orthogonal to its null space, from an SVD)
            Jp = J[:3]
            null = np.linalg.svd(Jp)[2][3:]
            assert np.abs(null @ qd).max() < 1e-9 * max(1.0, np.abs(qd).max())
            vrel = v6[:3] - xd
            assert np.linalg.norm(vrel) >= pr["v_min"] - 1e-9
            assert np.linalg.norm(vrel) == pytest.approx(vr[c], rel=1e-9)
            R, _ = orc.fk(arm, q)
            nb = R[7] @ arm["blade_normal"].astype(np.float64)
            a = nb @ vrel / np.linalg.norm(vrel)
            assert a >= pr["a_min"] - 2e-3
            assert np.all(q >= arm["q_lo"]) and np.all(q <= arm["q_hi"])
            assert all(abs(qd[j]) <= orc.taper(arm, j, q[j]) for j in range(7))
    assert n_acc >= 20


def test_goal_chart_reason_codes(orc, arm):
    """Every draw is either defined (then it also decodes) or carries the
    condition that left phi undefined; raising v_min turns every draw into
    a speed rejection, and a zero taper (joint boxes of width zero keep the
    IK from converging or the velocity under its bound) leaves none
    defined."""
    pr = _tosses(arm, 1)[0]
    st, Tq, vr, valid, why = orc.sample_goals(arm, pr, 31, 0, 0, 0, 512, reasons=True)
    assert np.array_equal(valid == 1, why == 0)
    assert set(np.unique(why)) <= set(range(len(orc.CHART_REASONS)))
    slow = dict(pr)
    slow["v_min"] = 1e3
    _, _, _, valid, why = orc.sample_goals(arm, slow, 31, 0, 0, 0, 256, reasons=True)
    assert not valid.any() and np.all(why == orc.CHART_REASONS.index("speed"))
    tight = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in arm.items()}
    tight["qd_taper_a"] = np.zeros(7, np.float32)
    _, _, _, valid, why = orc.sample_goals(tight, pr, 31, 0, 0, 0, 256, reasons=True)
    assert not valid.any()
    assert np.all((why == orc.CHART_REASONS.index("ik")) | (why == orc.CHART_REASONS.index("taper")))


def test_goal_chart_rejects_slow_contacts(orc, arm):
    pr = _tosses(arm, 1)[0]
    pr = dict(pr)
    pr["v_min"] = 1e3
    _, _, _, valid = orc.sample_goals(arm, pr, 31, 0, 0, 0, 256)
    assert not valid.any()


def test_uniform_sampler_box_and_taper(orc, arm):
    st = orc.sample_uniform(arm, 5, 0, 0, 0, 4096, 0.5)
    q, qd = st[:, :7], st[:, 8:15]
    assert np.all(q >= arm["q_lo"]) and np.all(q < arm["q_hi"])
    for j in range(7):
        tap = np.array([orc.taper(arm, j, x) for x in q[:, j]])
        assert np.all(np.abs(qd[:, j]) <= 0.5 * tap + 1e-12)
        # uniform in the box: each decile holds ~10%
        u = (q[:, j] - arm["q_lo"][j]) / (arm["q_hi"][j] - arm["q_lo"][j])
        h = np.histogram(u, bins=10, range=(0, 1))[0]
        assert h.min() > 330 and h.max() < 490


def _J_ref(pr, T, vrel, nu):
    sg = math.sqrt(pr["sig_p"] ** 2 + (pr["sig_v"] * T) ** 2 + (0.5 * pr["sig_a"] * T * T) ** 2)
    p_obj = math.erf(pr["r_catch"] / (sg * math.sqrt(2)))
    xdz = abs(pr["v0"][2] + pr["g"][2] * pr["t_fall"])
    p_in = NormalDist().cdf((pr["t_fall"] - T) / (sg / xdz))
    arm_t = -pr["lam"] * max(nu - pr["nu0"], 0) * T * (1 - pr["nu0"] / nu) if nu > 0 else 0.0
    return pr["w_v"] * min(vrel, pr["v_target"]) + pr["w_p"] * math.log(p_obj) + pr["w_r"] * math.log(p_in) + pr["w_x"] * arm_t


def test_objective_values_and_special_cases(orc, arm):
    pr = _tosses(arm, 1, reach=None)[0]      # window [0.2, 0.9] s: T = 0.9 at its end
    for T in (0.2, 0.5, 0.9):
        for vrel, nu in ((4.0, 0.5), (12.0, 0.95), (6.0, 1.0)):
            assert orc.objective(pr, T, vrel, nu) == pytest.approx(_J_ref(pr, T, vrel, nu), rel=1e-12, abs=1e-12)
    # clipping at v_target, no penalty below nu0, Phi(0) = 1/2 at t_fall
    assert orc.objective(pr, 0.5, 20.0, 0.2) == orc.objective(pr, 0.5, 9.0, 0.2)
    assert orc.objective(pr, 0.5, 5.0, 0.3) == orc.objective(pr, 0.5, 5.0, 0.85)
    base = orc.objective(pr, 0.5, 5.0, 0.0)
    nu0, lam = pr["nu0"], pr["lam"]
    assert orc.objective(pr, 0.5, 5.0, 1.0) - base == pytest.approx(-lam * (1 - nu0) * 0.5 * (1 - nu0), rel=1e-9)
    jt = orc.objective(pr, pr["t_fall"], 5.0, 0.0)
    sg = math.sqrt(pr["sig_p"] ** 2 + (pr["sig_v"] * pr["t_fall"]) ** 2)
    expect = pr["w_v"] * 5.0 + 8 * math.log(math.erf(pr["r_catch"] / (sg * math.sqrt(2)))) + 8 * math.log(0.5)
    assert jt == pytest.approx(expect, rel=1e-9)
    # the score prefers earlier arrivals when everything else is equal
    assert orc.objective(pr, 0.3, 5.0, 0.0) > orc.objective(pr, 0.8, 5.0, 0.0)


def test_reach_time_brute_force(orc, arm):
    pr = _tosses(arm, 2)[1]
    rng = np.random.default_rng(8)
    g = np.asarray(pr["g"])
    for _ in range(30):
        q = rng.uniform(arm["q_lo"], arm["q_hi"])
        t_n = rng.uniform(0.0, 0.6)
        gi, Tn = orc.reach_time(arm, pr, q, t_n, 256)
        b0, b1 = orc.blade(arm, q)
        Ts = pr["t_enter"] + np.arange(256) * (pr["t_fall"] - pr["t_enter"]) / 255
        ok = []
        for T in Ts:
            x = pr["x0"] + pr["v0"] * T + 0.5 * g * T * T
            u = np.clip((x - b0) @ (b1 - b0) / ((b1 - b0) @ (b1 - b0)), 0, 1)
            ok.append(t_n + np.linalg.norm(b0 + u * (b1 - b0) - x) / pr["v_tip"] <= T)
        ok = np.array(ok)
        if ok.any():
            assert gi == int(np.argmax(ok)) and Tn == pytest.approx(Ts[gi], rel=1e-12)
        else:
            assert gi == -1 and math.isinf(Tn)


def test_clearance_brute_force(orc, arm):
    rng = np.random.default_rng(9)
    obs = synth.obstacles(5, 3)
    for _ in range(5):
        s0, s1 = synth.random_edges(arm, 1, int(rng.integers(1000)))
        T, S = 0.7, 9
        c = orc.edge_clearance(arm, s0[0], s1[0], T, S, obs)
        best = np.inf
        for s in range(S):
            t = s * T / (S - 1)
            q, _, _ = orc.cubic(s0[0, :7], s0[0, 8:15], s1[0, :7], s1[0, 8:15], T, t)
            F = _fk4(arm, q)
            pts = [F[j][:3, 3] for j in range(7)] + [F[6][:3, 3] + float(arm["flange_d"]) * F[6][:3, 2]]
            for j in range(7):
                a, b = pts[j], pts[j + 1]
                for ob in obs.astype(np.float64):
                    ab = b - a
                    u = 0.0 if ab @ ab == 0 else np.clip((ob[:3] - a) @ ab / (ab @ ab), 0, 1)
                    dist = np.linalg.norm(a + u * ab - ob[:3]) - float(arm["link_radius"][j]) - ob[3]
                    best = min(best, dist)
        assert c == pytest.approx(best, abs=1e-12)
