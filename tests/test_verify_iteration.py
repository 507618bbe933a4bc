"""Pins of the per-edge verifier of a planner iteration (tests/parity.py,
verify_iteration), which the GPU tests and the benchmark apply to every edge
of an iteration: fed the oracle's own round in the layout the planner's
readbacks use, it reports no mismatch; each planted mistake on the "device"
side (a wrong grid index, a flipped verdict, a wrong parent list, a wrong
attach, a wrong score) is counted."""
import numpy as np
import pytest

import oracle.plan as OP
from paper_2609_22608_gb300 import synth
from tests.parity import verify_iteration

F32 = np.float32
K_GRID, S_COLL, K_PAR, W_VEL = 64, 16, 5, 0.1


@pytest.fixture(scope="module")
def rnd(orc, arm):
    toss = synth.random_toss(arm, 3)
    root = synth.random_states(arm, 1, 5003)[0]
    pr = synth.make_problem(toss, root=root)
    states, parent, t = synth.random_tree(arm, 150, 3, root=root, t_max=pr["t_fall"])
    G = 24
    st, Tq, vr, valid = orc.sample_goals(arm, pr, 103, 0, 0, 0, G)
    rng = np.random.default_rng(3)
    free = np.repeat(np.asarray(root, F32)[None], 40, axis=0)
    free[:, :7] += rng.uniform(-0.3, 0.3, (40, 7)).astype(F32)
    free[:, 8:15] = rng.uniform(-0.2, 0.2, (40, 7)).astype(F32)
    free[:, 7] = free[:, 15] = 0.0
    # the planner's slot layout: G goal draws (decoded or not), then free
    cand = dict(states=np.concatenate([st.astype(F32), free]),
                T_req=np.concatenate([Tq.astype(F32), np.full(40, np.nan, F32)]),
                v_rel=np.concatenate([vr.astype(F32), np.full(40, np.nan, F32)]),
                valid=np.concatenate([valid.astype(np.uint8), np.ones(40, np.uint8)]))
    grid = synth.duration_grid(K_GRID)
    vi = np.nonzero(cand["valid"])[0]
    n_goal_valid = int(valid.sum())
    tree = OP.Tree(states, t, parent)
    inc0 = dict(id=-1, J=-np.inf, t_best=float(F32(pr["t_fall"])))
    out, inc, det = OP.plan_round(arm, pr, tree, cand["states"][vi], n_goal_valid,
                                  cand["T_req"][vi[:n_goal_valid]], cand["v_rel"][vi[:n_goal_valid]],
                                  inc0, K_PAR, grid, S_COLL)
    B = cand["states"].shape[0]
    nn = np.full((B, K_PAR - 1), -1, np.int32)
    nn[vi] = det["parents"][:, 1:]
    # per-edge results in the planner's layout (k* from the oracle's own scan)
    ks = np.full((B, K_PAR), -1, np.int32)
    T = np.full((B, K_PAR), np.nan, F32)
    rv = np.full((B, K_PAR), np.nan, F32)
    ok = np.zeros((B, K_PAR), np.uint8)
    for r, b in enumerate(vi):
        for j in range(K_PAR):
            T[b, j] = det["T"][r, j]
            rv[b, j] = det["rv"][r, j]
            ok[b, j] = det["ok"][r, j]
            if r < n_goal_valid:
                p = det["parents"][r, j]
                e = orc.time_edges(arm, states[p][None], cand["states"][b][None], grid, S_COLL,
                                   mode=1, T_fixed=np.array([T[b, j]], F32))
                ks[b, j] = 0 if e["k_star"][0] == 0 else -1
            else:
                hit = np.nonzero(grid == T[b, j])[0]
                ks[b, j] = hit[0] if len(hit) else -1
    gtree = dict(states=out.states, t=out.t, parent=out.parent, J=out.J.astype(F32),
                 nu=out.nu.astype(F32), n=out.n)
    return dict(arm=arm, pr=pr, tree=dict(states=states, t=t, parent=parent), cand=cand, G=G,
                nn=nn, edges=dict(k_star=ks, T=T, rho_v=rv, ok=ok), gtree=gtree, grid=grid,
                inc=dict(incumbent=inc["id"]), t_best=inc0["t_best"], added=out.n - tree.n)


def _run(orc, c, **over):
    a = dict(c)
    a.update(over)
    return verify_iteration(orc, a["arm"], a["pr"], a["tree"], a["t_best"], a["cand"], a["G"],
                            a["nn"], a["edges"], a["gtree"], a["grid"], S_COLL, K_PAR, W_VEL,
                            inc_gpu=a["inc"])


def _copy_edges(e):
    return {k: v.copy() for k, v in e.items()}


def test_oracle_round_verifies_clean(orc, rnd):
    r = _run(orc, rnd)
    assert r["edge_mismatches"] == 0 and r["parent_mismatches"] == 0
    assert r["attach_mismatches"] == 0 and r["incumbent_ok"]
    assert r["edges_formed"] == r["valid_candidates"] * K_PAR
    assert rnd["added"] > 0 and r["nodes_added"] == rnd["added"]


def test_planted_grid_index_is_caught(orc, rnd):
    e = _copy_edges(rnd["edges"])
    b, j = [(b, j) for b in range(rnd["G"], e["k_star"].shape[0]) for j in range(K_PAR)
            if e["k_star"][b, j] >= 0][0]
    e["k_star"][b, j] += 7
    e["T"][b, j] = rnd["grid"][e["k_star"][b, j]]
    assert _run(orc, rnd, edges=e)["edge_mismatches"] >= 1


def test_planted_goal_verdict_is_caught(orc, rnd):
    e = _copy_edges(rnd["edges"])
    gb = [b for b in range(rnd["G"]) if rnd["cand"]["valid"][b]]
    e["ok"][gb[0], 0] ^= 1
    r = _run(orc, rnd, edges=e)
    assert r["edge_mismatches"] >= 1


def test_planted_parent_is_caught(orc, rnd):
    nn = rnd["nn"].copy()
    b = rnd["G"] + 1
    nn[b, 0] = rnd["tree"]["states"].shape[0] - 1 if nn[b, 0] != rnd["tree"]["states"].shape[0] - 1 else 1
    assert _run(orc, rnd, nn=nn)["parent_mismatches"] >= 1


def test_planted_attach_and_score_are_caught(orc, rnd):
    n0 = rnd["tree"]["states"].shape[0]
    g = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in rnd["gtree"].items()}
    g["t"][n0] = np.nextafter(g["t"][n0], F32(np.inf))
    assert _run(orc, rnd, gtree=g)["attach_mismatches"] >= 1
    goal_nodes = [i for i in range(n0, g["n"]) if np.isfinite(rnd["gtree"]["J"][i])]
    if goal_nodes:
        g = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in rnd["gtree"].items()}
        g["J"][goal_nodes[0]] += 0.5
        assert _run(orc, rnd, gtree=g)["attach_mismatches"] >= 1
