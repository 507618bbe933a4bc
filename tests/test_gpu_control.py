"""Parity of the controller (fn_controller_torque), the full-resolution
recheck (fn_check_edges_full) and the incumbent path
(fn_planner_incumbent_path) with the FP64 oracle, through the C ABI.

Rules: torques within 3e-5 of max(|tau_ref|_inf, 1 N m) (the FP32 torque
bar plus the acceleration's rounding); accelerations within 1e-5 of
max(|qdd_ref|, 1); clip flags equal except where the clipped quantity sits
within 1e-4 (relative) of its bound in the oracle.  Recheck ratios by the
edge-timing rule (tests/parity.py), clearances within 2e-5 m, ok equal
except where a ratio or the clearance sits within 1e-4 of its bound.
"""
import numpy as np
import pytest
import torch

from paper_2609_22608_gb300 import synth
from tests.parity import rho_matches
from tests.test_oracle_control import _states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ops():
    from paper_2609_22608_gb300 import ops as o
    return o


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _ctrl_inputs(arm, B, seed):
    rng = np.random.default_rng(seed)
    x = _states(arm, B, seed, speed=0.6)
    g = _states(arm, B, seed + 1, speed=0.6)
    T = rng.uniform(0.05, 1.5, B).astype(np.float32)
    # a quarter next to a joint limit, moving toward it
    hi = np.asarray(arm["q_hi"], np.float64)
    near = rng.random(B) < 0.25
    j = rng.integers(0, 7, B)
    x[near, j[near]] = (hi[j[near]] - rng.uniform(1e-5, 1e-2, near.sum())).astype(np.float32)
    x[near, 8 + j[near]] = 0.4
    prev = rng.uniform(-20, 20, (B, 7)).astype(np.float32)
    return x, g, T, prev


def _near_bounds(orc, arm, x, g, T, dt, prev, rate):
    """Instances whose clip decisions sit within 1e-4 of a bound (oracle)."""
    big = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in arm.items()}
    big["tau_max"] = np.full(7, 1e9, np.float32)
    big["w_max"] = np.float32(1e12)
    raw = orc.controller_torque(big, x, g, T, dt)
    tmax = np.asarray(arm["tau_max"], np.float64)
    near = np.any(np.abs(np.abs(raw["tau"]) - tmax) <= 1e-4 * tmax, axis=1)
    tc = np.clip(raw["tau"], -tmax, tmax)
    P = np.abs(np.sum(tc * x[:, 8:15].astype(np.float64), axis=1))
    near |= np.abs(P - float(arm["w_max"])) <= 1e-4 * float(arm["w_max"])
    if prev is not None:
        ref = orc.controller_torque(arm, x, g, T, dt)
        d = np.abs(ref["tau"] - prev.astype(np.float64)) - np.asarray(rate) * dt
        near |= np.any(np.abs(d) <= 1e-4 * np.maximum(np.abs(ref["tau"]), 1.0), axis=1)
    # acceleration box: the unclipped acceleration against the taper bounds
    free = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in big.items()}
    unb = orc.controller_torque(free, x, g, T, 1e-12)        # a box too wide to clip
    qd = x[:, 8:15].astype(np.float64)
    for b in range(x.shape[0]):
        for j in range(7):
            q = float(x[b, j])
            lo_, hi_ = float(arm["q_lo"][j]), float(arm["q_hi"][j])
            bound = min(float(arm["qd_max"][j]),
                        np.sqrt(2 * float(arm["qd_taper_a"][j]) * max(0.0, min(q - lo_, hi_ - q))))
            a = unb["qdd"][b, j]
            for edge in ((-bound - qd[b, j]) / dt, (bound - qd[b, j]) / dt):
                if abs(a - edge) <= 1e-4 * max(abs(edge), 1.0):
                    near[b] = True
    return near


@pytest.mark.parametrize("B,slew", [(1, False), (37, True), (1000, False), (1000, True)])
def test_controller_parity(ops, orc, arm, B, slew):
    x, g, T, prev = _ctrl_inputs(arm, B, 100 + B)
    dt = 1e-3
    rate = np.full(7, 1000.0, np.float32)
    out = ops.controller_torque(arm, dev(x), dev(g), dev(T), dt,
                                tau_prev=dev(prev) if slew else None,
                                tau_rate_max=rate if slew else None)
    ref = orc.controller_torque(arm, x, g, T, dt, tau_prev=prev if slew else None,
                                rate=rate.astype(np.float64) if slew else None)
    tau = out["tau"].cpu().numpy().astype(np.float64)
    qdd = out["qdd"].cpu().numpy().astype(np.float64)
    flags = out["flags"].cpu().numpy()
    scale = np.maximum(np.abs(ref["tau"]).max(axis=1), 1.0)
    err = np.abs(tau - ref["tau"]).max(axis=1) / scale
    assert np.all(err <= 3e-5), (np.argmax(err), err.max())
    aerr = np.abs(qdd - ref["qdd"]) / np.maximum(np.abs(ref["qdd"]), 1.0)
    assert np.all(aerr <= 1e-5), aerr.max()
    diff = flags != ref["flags"]
    if diff.any():
        near = _near_bounds(orc, arm, x, g, T, dt, prev if slew else None, rate)
        assert np.all(near[diff]), np.flatnonzero(diff & ~near)[:5]
    assert np.any(ref["flags"] & 1) or B < 37
    tmax = np.asarray(arm["tau_max"], np.float64)
    if not slew:
        assert np.all(np.abs(tau) <= tmax * (1 + 1e-6))


def test_controller_invalid_and_args(ops, arm):
    x, g, T, prev = _ctrl_inputs(arm, 8, 7)
    x[2, 4] = np.nan
    T[5] = 0.0
    out = ops.controller_torque(arm, dev(x), dev(g), dev(T))
    f = out["flags"].cpu().numpy()
    assert f[2] == 0x80 and f[5] == 0x80
    assert np.isnan(out["tau"].cpu().numpy()[[2, 5]]).all()
    from paper_2609_22608_gb300._lib import FnError
    with pytest.raises(FnError):
        ops.controller_torque(arm, dev(x), dev(g), dev(T), dt=0.0)
    with pytest.raises(FnError):                 # slew without a rate
        ops.controller_torque(arm, dev(x), dev(g), dev(T), tau_prev=dev(prev))
    empty = torch.empty(0, 16, device="cuda")
    ops.controller_torque(arm, empty, empty, torch.empty(0, device="cuda"))


def test_controller_full_size_sampled(ops, orc, arm):
    B = 65536
    x, g, T, prev = _ctrl_inputs(arm, B, 5)
    out = ops.controller_torque(arm, dev(x), dev(g), dev(T), 1e-3)
    idx = np.random.default_rng(5).choice(B, 256, replace=False)
    ref = orc.controller_torque(arm, x[idx], g[idx], T[idx], 1e-3)
    tau = out["tau"].cpu().numpy()[idx].astype(np.float64)
    scale = np.maximum(np.abs(ref["tau"]).max(axis=1), 1.0)
    assert np.all(np.abs(tau - ref["tau"]).max(axis=1) / scale <= 3e-5)


def _check_recheck(orc, arm, s0, s1, T, S, S_clear, obs, margin, res):
    ref = orc.check_edges(arm, s0, s1, T, S, S_clear, obs, margin)
    rho = res["rho3"].cpu().numpy()
    cl = res["clearance"].cpu().numpy().astype(np.float64)
    ok = res["ok"].cpu().numpy()
    fin = np.isfinite(ref["rho3"][:, 0])
    assert np.array_equal(np.isnan(rho[:, 0]), ~fin)
    i = np.flatnonzero(fin)
    bad = rho_matches(orc, arm, s0[i], s1[i], T[i].astype(np.float64), S, rho[i], ref["rho3"][i])
    assert not bad, bad[:3]
    if len(obs):
        assert np.allclose(cl[i], ref["clearance"][i], rtol=0, atol=2e-5)
    near = np.any(np.abs(ref["rho3"][i] - 1) <= 1e-4, axis=1)
    if len(obs):
        near |= np.abs(ref["clearance"][i] - margin) <= 1e-4
    same = ok[i] == ref["ok"][i]
    assert np.all(same | near)
    return ref


@pytest.mark.parametrize("E,S,S_clear", [(1, 256, 64), (45, 256, 64), (300, 64, 16), (129, 33, 7)])
def test_check_edges_parity(ops, orc, arm, E, S, S_clear):
    s0, s1 = synth.random_edges(arm, E, 300 + E)
    rng = np.random.default_rng(E)
    T = rng.uniform(0.3, 2.0, E).astype(np.float32)
    obs = synth.obstacles(5, 3).astype(np.float32)
    res = ops.check_edges_full(arm, dev(s0), dev(s1), dev(T), S, S_clear, obs, 0.02)
    _check_recheck(orc, arm, s0, s1, T, S, S_clear, obs, 0.02, res)
    res = ops.check_edges_full(arm, dev(s0), dev(s1), dev(T), S, S_clear, None, 0.02)
    assert torch.isinf(res["clearance"]).all()


def test_check_edges_device_count_and_invalid(ops, orc, arm):
    s0, s1 = synth.random_edges(arm, 16, 9)
    T = np.full(16, 0.9, np.float32)
    T[1] = np.nan
    s1[2, 0] = np.inf
    n = torch.tensor([5], dtype=torch.int32, device="cuda")
    out = dict(rho3=torch.full((16, 3), -7.0, device="cuda"),
               clearance=torch.full((16,), -7.0, device="cuda"),
               ok=torch.full((16,), 9, dtype=torch.uint8, device="cuda"))
    ops.check_edges_full(arm, dev(s0), dev(s1), dev(T), 64, 8, None, 0.02, E_dev=n, out=out)
    rho = out["rho3"].cpu().numpy()
    assert np.all(rho[5:] == -7.0) and np.all(out["ok"].cpu().numpy()[5:] == 9)
    assert np.isnan(rho[1]).all() and np.isnan(rho[2]).all()
    assert np.all(np.isfinite(rho[[0, 3, 4]]))


def test_incumbent_path_and_recheck(orc, arm):
    """The goal-attach round of the planner tests (approach nodes loaded
    delta seconds before each decoded goal): the incumbent's path is root ->
    approach node (a loaded edge, no duration) -> rendezvous node."""
    from paper_2609_22608_gb300 import planner as P
    from tests.test_gpu_planner import K_GRID, S_COLL, make_case
    case = make_case(arm, orc, 40, N=150, n_free=32)
    states, t, parent = case["tree"]
    G = case["n_goal"]
    g = case["cand"][:G].astype(np.float64)
    appr = g.copy()
    appr[:, :7] = g[:, :7] - 0.05 * g[:, 8:15]
    states = np.concatenate([states, appr.astype(np.float32)])
    t = np.concatenate([t, (case["T_req"] - np.float32(0.05)).astype(np.float32)])
    parent = np.concatenate([parent, np.zeros(G, parent.dtype)])
    N, B = states.shape[0], case["cand"].shape[0]
    obs = synth.obstacles(5, 3).astype(np.float32)
    pl = P.Planner(arm, P=1, n_cap=N + B + 8, b_max=B, k=5, K=K_GRID, S=S_COLL, S_clear=8)
    prob = P.problem_struct(case["pr"], B, G, root=case["root"])
    pl.reset([prob])
    pl.load_tree(0, states, t, parent)
    pl.set_candidates(0, case["cand"], G, case["T_req"], case["v_rel"])
    out = pl.iterate([prob], 0, P.FN_PLAN_EXTERNAL)[0]
    assert out["incumbent"] > 0
    path = pl.recheck_incumbent(arm, 0, S=256, S_clear=64, obs=obs, margin=0.02, max_edges=8)
    torch.cuda.synchronize()
    L = int(path["n_edges"].item())
    tree = pl.get_tree(0)
    short = pl.incumbent_path(0, max_edges=1)          # too short: counted, not written
    torch.cuda.synchronize()
    assert int(short["n_edges"].item()) == L and torch.isnan(short["T"]).all()
    pl.close()
    nodes = [out["incumbent"]]
    while nodes[-1] != 0:
        nodes.append(int(tree["parent"][nodes[-1]]))
    nodes = nodes[::-1]
    assert L == len(nodes) - 1 == 2
    assert path["nodes"][:L + 1].cpu().numpy().tolist() == nodes
    s0 = path["s0"][:L].cpu().numpy()
    s1 = path["s1"][:L].cpu().numpy()
    T = path["T"][:L].cpu().numpy()
    assert np.array_equal(s0, tree["states"][nodes[:-1]])
    assert np.array_equal(s1, tree["states"][nodes[1:]])
    assert np.isnan(T[0])                               # the loaded approach edge
    dt = float(tree["t"][nodes[2]]) - float(tree["t"][nodes[1]])
    assert T[1] == pytest.approx(dt, rel=1e-5, abs=1e-6)
    res = {k: path[k][:L] for k in ("rho3", "clearance", "ok")}
    ref = _check_recheck(orc, arm, s0, s1, T, 256, 64, obs, 0.02, res)
    assert ref["ok"][0] == 0 and np.isfinite(ref["rho3"][1]).all()
