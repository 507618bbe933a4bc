"""Parity of the planner (fn_plan_iteration and friends) with one round of
Algorithm 1 on the FP64 oracle (oracle/plan.py), through the C ABI.

Candidates are drawn on the host by the oracle's own samplers and given to
both sides (FN_PLAN_EXTERNAL), so the comparison covers parents, edge timing,
clearance, attach, scoring, the incumbent and pruning.  A candidate may end
up differently only where one of its edges sits within the 1e-4 limit margin
in the oracle (the edge-timing parity rule)."""
import numpy as np
import pytest

import oracle.plan as OP
from paper_2609_22608_gb300 import synth
from tests.parity import compare_round

pytestmark = pytest.mark.gpu

K_GRID, S_COLL = 32, 16


@pytest.fixture(scope="module")
def P():
    from paper_2609_22608_gb300 import planner as pl
    return pl


def make_case(arm, orc, seed, N=300, n_goal_draw=512, n_free=96, obstacles=None):
    toss = synth.random_toss(arm, seed)
    root = synth.random_states(arm, 1, 5000 + seed)[0]
    pr = synth.make_problem(toss, root=root)
    states, parent, t = synth.random_tree(arm, N, seed, root=root)
    st, Tq, vr, valid = orc.sample_goals(arm, pr, 100 + seed, 0, 0, 0, n_goal_draw)
    gi = np.nonzero(valid)[0]
    goal = st[gi].astype(np.float32)
    free = orc.sample_uniform(arm, 200 + seed, 0, 0, 0, n_free, 0.5).astype(np.float32)
    cand = np.concatenate([goal, free])
    T_req = Tq[gi].astype(np.float32)
    v_rel = vr[gi].astype(np.float32)
    return dict(pr=pr, root=root, tree=(states, t, parent), cand=cand, n_goal=len(gi),
                T_req=T_req, v_rel=v_rel, obstacles=obstacles)


def run_pair(P, orc, arm, case, k=5, prune=False, obstacles=None, bm=None, sched=None):
    grid = synth.duration_grid(K_GRID)
    states, t, parent = case["tree"]
    N = states.shape[0]
    B = case["cand"].shape[0]
    pl = P.Planner(arm, P=1, n_cap=N + B + 8, b_max=bm or B, k=k, K=K_GRID, S=S_COLL, S_clear=8)
    if sched is not None:
        pl.set_schedule(sched)
    prob = P.problem_struct(case["pr"], B, case["n_goal"], root=case["root"], obstacles=obstacles)
    pl.reset([prob])
    pl.load_tree(0, states, t, parent)
    pl.set_candidates(0, case["cand"], case["n_goal"], case["T_req"], case["v_rel"])
    flags = P.FN_PLAN_EXTERNAL | (P.FN_PLAN_PRUNE if prune else 0)
    out = pl.iterate([prob], 0, flags)[0]
    gtree = pl.get_tree(0)
    pl.close()
    tree = OP.Tree(states, t, parent)
    inc = dict(id=-1, J=-np.inf, t_best=float(np.float32(case["pr"]["t_fall"])))
    rtree, rinc, det = OP.plan_round(arm, case["pr"], tree, case["cand"], case["n_goal"],
                                     case["T_req"], case["v_rel"], inc, k, grid, S_COLL,
                                     S_clear=8, obstacles=obstacles, prune=False)
    return out, gtree, rtree, rinc, det, grid


@pytest.mark.parametrize("seed,bm,sched", [(0, None, None), (1, None, None), (0, 4096, None),
                                           (1, 4096, None), (0, None, 3), (1, None, 3),
                                           (2, None, 0)])
def test_plan_round_parity(P, orc, arm, seed, bm, sched):
    """One round of Algorithm 1's body against the oracle.  bm = 4096: a
    planner for large batches, whose attach runs over many blocks; sched: the
    edge phase's schedule (3: one warp per edge on the paired core, 0: the
    packed stages at the largest register budget)."""
    case = make_case(arm, orc, seed)
    assert case["n_goal"] >= 3
    out, gtree, rtree, rinc, det, grid = run_pair(P, orc, arm, case, bm=bm, sched=sched)
    N = case["tree"][0].shape[0]
    bad = compare_round(orc, arm, case, gtree, rtree, det, N, grid)
    assert not bad, f"candidates attached differently without a near-margin edge: {bad[:5]}"
    assert gtree["n"] - N == out["n_added"]
    assert abs((gtree["n"] - N) - (rtree.n - N)) <= 2
    # incumbent
    if rinc["id"] >= 0:
        assert out["incumbent"] >= 0
        assert out["J"] == pytest.approx(rinc["J"], rel=1e-4, abs=1e-4)
        assert out["t_best"] == pytest.approx(rinc["t_best"], rel=1e-6)
        seg = OP.first_segment(rtree, rinc)
        assert np.array_equal(out["q_g"], seg[0][:7])
    else:
        assert out["incumbent"] == -1
    # tree invariants: parents precede children, time-to-come adds up, J only on goals
    par = gtree["parent"]
    assert par[0] == -1 and np.all(par[1:] < np.arange(1, gtree["n"]))


@pytest.mark.parametrize("seed,delta", [(0, 0.05), (1, 0.1)])
def test_plan_round_goal_attach(P, orc, arm, seed, delta):
    """Goal edges that succeed: the tree holds, for each decoded goal, an
    approach node delta seconds earlier on the goal's velocity line
    (q_g - delta qd_g, qd_g).  The rendezvous nodes, their scores and the
    incumbent (Eq. (objective), the t_best update and the first segment)
    must match the oracle's round."""
    case = make_case(arm, orc, 40 + seed, N=150, n_free=32)
    states, t, parent = case["tree"]
    G = case["n_goal"]
    g = case["cand"][:G].astype(np.float64)
    appr = g.copy()
    appr[:, :7] = g[:, :7] - delta * g[:, 8:15]
    appr = appr.astype(np.float32)
    t_app = (case["T_req"] - np.float32(delta)).astype(np.float32)
    case["tree"] = (np.concatenate([states, appr]), np.concatenate([t, t_app]),
                    np.concatenate([parent, np.zeros(G, parent.dtype)]))
    out, gtree, rtree, rinc, det, grid = run_pair(P, orc, arm, case)
    N = case["tree"][0].shape[0]
    assert rinc["id"] >= 0, "the oracle attached no goal: the case does not exercise the incumbent"
    bad = compare_round(orc, arm, case, gtree, rtree, det, N, grid)
    assert not bad, f"candidates attached differently without a near-margin edge: {bad[:5]}"
    assert out["incumbent"] >= 0
    assert out["J"] == pytest.approx(rinc["J"], rel=1e-4, abs=1e-4)
    assert out["t_best"] == pytest.approx(rinc["t_best"], rel=1e-6)
    seg = OP.first_segment(rtree, rinc)
    assert np.array_equal(out["q_g"], seg[0][:7])
    # scores: rendezvous nodes carry finite J, the others NaN
    Jg = gtree["J"][N:gtree["n"]]
    assert np.sum(np.isfinite(Jg)) >= 1


@pytest.mark.parametrize("trained", [False, True])
def test_surrogate_round_matches_plain_round(P, orc, arm, trained):
    """Free edges routed through the surrogate's window pass attach the same
    candidates as the plain pass (uncertified windows are rescanned exactly;
    a certified window can differ only where the limits are not monotone in
    T), with obstacles so that the clearance of the routed edges is checked
    against each edge's own problem."""
    from paper_2609_22608_gb300 import surrogate as SG
    import torch
    obs = synth.obstacles(5, 3)
    case = make_case(arm, orc, 50, N=400, n_free=200)
    grid = synth.duration_grid(K_GRID)
    mlp = SG.MLP(max_batch=4096, seed=3)
    if trained:
        a, b = synth.random_edges(arm, 8192, 51)
        da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        lab = SG.label_edges(arm, da, db, grid, S_COLL)
        SG.train(mlp, arm, da, db, lab, grid, epochs=3, batch=2048, lr=2e-3)
    states, t, parent = case["tree"]
    N, B = states.shape[0], case["cand"].shape[0]
    trees = []
    for use in (False, True):
        pl = P.Planner(arm, P=1, n_cap=N + B + 8, b_max=B, k=5, K=K_GRID, S=S_COLL, S_clear=8)
        if use:
            pl.set_surrogate(mlp, 8)
        # a generous t_best so that most free edges have admissible durations
        pr = dict(case["pr"])
        prob = P.problem_struct(pr, B, case["n_goal"], root=case["root"], obstacles=obs)
        pl.reset([prob])
        pl.load_tree(0, states, t, parent)
        pl.set_candidates(0, case["cand"], case["n_goal"], case["T_req"], case["v_rel"])
        out = pl.iterate([prob], 0, P.FN_PLAN_EXTERNAL)[0]
        trees.append((pl.get_tree(0), out))
        pl.close()
    (g0, o0), (g1, o1) = trees
    k0 = {g0["states"][i].tobytes() for i in range(N, g0["n"])}
    k1 = {g1["states"][i].tobytes() for i in range(N, g1["n"])}
    assert len(k0 ^ k1) <= max(2, 0.02 * B), (len(k0), len(k1), len(k0 ^ k1))
    assert o0["incumbent"] == o1["incumbent"] or abs(o0["J"] - o1["J"]) < 1e-4
    mlp.close()


@pytest.mark.parametrize("sched", [None, 3])
def test_plan_round_with_obstacles(P, orc, arm, sched):
    obs = synth.obstacles(5, 3)
    case = make_case(arm, orc, 2, N=200, n_free=64)
    out, gtree, rtree, rinc, det, grid = run_pair(P, orc, arm, case, obstacles=obs, sched=sched)
    N = case["tree"][0].shape[0]
    bad = compare_round(orc, arm, case, gtree, rtree, det, N, grid)
    assert not bad


@pytest.mark.parametrize("chain", [0, 150])
def test_plan_prune_parity(P, orc, arm, chain):
    """Eq. (reach) pruning against the oracle's prune_tree.  chain = 150: the
    first 150 nodes form one path, longer than the multi-block prune's parent
    walk, so the single-block prune takes the problem.  In both, every kept
    node keeps its chart parameters."""
    case = make_case(arm, orc, 3, N=400)
    grid = synth.duration_grid(K_GRID)
    states, t, parent = case["tree"]
    if chain:
        t, parent = t.copy(), parent.copy()
        for i in range(1, chain):
            parent[i] = i - 1
            t[i] = np.float32(t[i - 1] + 0.003)
        for i in range(chain, len(t)):   # keep t increasing along every parent link
            t[i] = max(t[i], np.float32(t[parent[i]] + 0.003))
    N, B = states.shape[0], case["cand"].shape[0]
    pl = P.Planner(arm, P=1, n_cap=N + B + 8, b_max=B, k=5, K=K_GRID, S=S_COLL)
    prob = P.problem_struct(case["pr"], B, case["n_goal"], root=case["root"])
    pl.reset([prob])
    pl.load_tree(0, states, t, parent)
    pl.set_candidates(0, case["cand"], case["n_goal"], case["T_req"], case["v_rel"])
    pl.iterate([prob], 0, P.FN_PLAN_EXTERNAL)
    before = pl.get_tree(0)
    z_before = pl.get_node_params(0, before["n"])
    # prune the tree as it stands: an iteration with no candidates and the prune flag
    prob0 = P.problem_struct(case["pr"], 0, 0, root=case["root"])
    out = pl.iterate([prob0], 1, P.FN_PLAN_EXTERNAL | P.FN_PLAN_PRUNE)[0]
    after = pl.get_tree(0)
    z_after = pl.get_node_params(0, after["n"])
    pl.close()
    tree = OP.Tree(before["states"], before["t"], before["parent"], before["J"], before["nu"])
    inc = dict(id=out["incumbent"], J=out["J"], t_best=out["t_best"])
    # the incumbent before pruning: the node whose J equals the reported score
    if out["incumbent"] >= 0:
        ids = np.nonzero(np.isclose(before["J"], out["J"], rtol=0, atol=0))[0]
        inc["id"] = int(ids[0])
    else:
        inc["id"] = -1
    rt, rinc, alive = OP.prune_tree(arm, case["pr"], tree, inc, 256)
    # compare kept sets by state; disagreements only near the T_n <= t_best boundary
    g_keys = {after["states"][i].tobytes() for i in range(after["n"])}
    r_keys = {rt.states[i].tobytes() for i in range(rt.n)}
    diff = g_keys ^ r_keys
    for key in diff:
        i = next(j for j in range(tree.n) if tree.states[j].tobytes() == key)
        g, Tn = orc.reach_time(arm, case["pr"], tree.states[i, :7].astype(float), float(tree.t[i]))
        assert g >= 0 and abs(Tn - inc["t_best"]) < 5e-3, (i, g, Tn, inc["t_best"])
    assert len(diff) <= max(2, 0.01 * tree.n)
    # the kept nodes moved with their parents, times and chart parameters
    old = {before["states"][i].tobytes(): i for i in range(before["n"])}
    for j in range(after["n"]):
        i = old[after["states"][j].tobytes()]
        assert after["t"][j] == before["t"][i]
        pj, pi = after["parent"][j], before["parent"][i]
        if pi >= 0:
            assert np.array_equal(after["states"][pj], before["states"][pi])
        assert np.array_equal(z_after[j], z_before[i], equal_nan=True)
    if out["incumbent"] >= 0:
        assert np.array_equal(after["states"][out["incumbent"]], before["states"][inc["id"]])


@pytest.mark.parametrize("N,B,k,bm,cap", [(300, 97, 5, None, None), (4097, 64, 8, None, None),
                                          (13001, 150, 8, None, None), (9000, 40, 17, None, None),
                                          (300, 97, 5, 8192, None), (4097, 300, 8, 8192, None),
                                          (13001, 150, 8, 8192, None), (9000, 70, 17, 8192, None),
                                          (300, 97, 5, None, 40000), (4097, 300, 8, None, 40000),
                                          (13001, 150, 8, None, 40000), (9000, 70, 17, None, 40000)])
def test_parents_match_brute_force(P, orc, arm, N, B, k, bm, cap):
    """The planner's parent lists equal the oracle's brute-force kNN over the
    non-root nodes (one split of the tree and several, k-1 = 4, 7, 16),
    up to swaps among near-equal exact distances.  bm = 8192: a planner sized
    for 8192 candidates (a larger persistent grid share per query, more
    splits merged); cap = 40000: a planner for large trees, whose free
    queries take the tiled search (eight queries per CTA, ragged groups)."""
    from tests.parity import knn_mismatches
    toss = synth.random_toss(arm, 21)
    root = synth.random_states(arm, 1, 77)[0]
    pr = synth.make_problem(toss, root=root)
    states, parent, t = synth.random_tree(arm, N, 31, root=root)
    cand = synth.random_states(arm, B, 32)
    w_vel = 0.1
    pl = P.Planner(arm, P=1, n_cap=cap or N + B + 8, b_max=bm or B, k=k, K=16, S=8, w_vel=w_vel)
    prob = P.problem_struct(pr, B, 0, root=root)
    pl.reset([prob])
    pl.load_tree(0, states, t, parent)
    pl.set_candidates(0, cand, 0, np.zeros(B, np.float32), np.zeros(B, np.float32))
    pl.iterate([prob], 0, P.FN_PLAN_EXTERNAL)
    nn = pl.get_parents(0, B)
    pl.close()
    idx, d = orc.knn(states, cand, k - 1, float(np.float32(w_vel)), first=1)
    s64, c64 = states.astype(np.float64), cand.astype(np.float64)

    def exact(b, i):
        if i < 0:
            return np.inf
        dq = s64[i, 0:7] - c64[b, 0:7]
        dv = s64[i, 8:15] - c64[b, 8:15]
        return float(dq @ dq + np.float32(w_vel) * (dv @ dv))
    dg = np.array([[exact(b, i) for i in nn[b]] for b in range(B)])
    assert np.all(nn >= 1) and np.all(nn < N)
    assert np.all(np.diff(dg, axis=1) >= -1e-6 * dg[:, 1:])
    assert not knn_mismatches(nn, dg, idx, d)


def test_sampler_uniform_matches_oracle(P, orc, arm):
    """Free candidates: same Philox counters, same formula -> equal to FP32
    rounding."""
    toss = synth.random_toss(arm, 4)
    pr = synth.make_problem(toss, root=synth.random_states(arm, 1, 9)[0])
    B, G = 600, 0
    pl = P.Planner(arm, P=1, n_cap=64, b_max=B, k=1, K=8, S=8)
    prob = P.problem_struct(pr, B, G, seed=1234)
    pl.reset([prob])
    pl.iterate([prob], 3, 0)
    c = pl.get_candidates(0, B)
    pl.close()
    ref = orc.sample_uniform(arm, 1234, 3, 0, 0, B, 0.5)
    q, qr = c["states"][:, :7].astype(np.float64), ref[:, :7]
    assert np.allclose(q, qr, rtol=0, atol=1e-6)
    # qd = (2u - 1) vel_frac qdbar(q): the sqrt taper is ill-conditioned next to
    # a limit, so compare against the oracle's taper evaluated at the GPU's q
    for j in range(7):
        tr = np.array([orc.taper(arm, j, x) for x in qr[:, j]])
        tg = np.array([orc.taper(arm, j, x) for x in q[:, j]])
        s = np.where(tr > 0, ref[:, 8 + j] / np.where(tr > 0, 0.5 * tr, 1), 0)   # 2u - 1
        expect = s * 0.5 * tg
        assert np.allclose(c["states"][:, 8 + j], expect, rtol=0, atol=1e-5 * float(arm["qd_max"][j]))


def test_sampler_single_parent_odd_batch(P, orc, arm):
    """k = 1 (root only, no parent search) with a batch that is not a
    multiple of the sampler's block: the sampling launch has spare warps and
    no tree-mirror work; the iteration must still complete, with the same
    uniform draws as the oracle."""
    toss = synth.random_toss(arm, 6)
    pr = synth.make_problem(toss, root=synth.random_states(arm, 1, 11)[0])
    B = 601
    pl = P.Planner(arm, P=1, n_cap=64, b_max=B, k=1, K=8, S=8)
    prob = P.problem_struct(pr, B, 3, seed=99)
    pl.reset([prob])
    out = pl.iterate([prob], 1, 0)[0]
    c = pl.get_candidates(0, B)
    pl.close()
    ref = orc.sample_uniform(arm, 99, 1, 0, 3, B - 3, 0.5)
    assert np.allclose(c["states"][3:, :7].astype(np.float64), ref[:, :7], rtol=0, atol=1e-6)
    assert out["n_nodes"] >= 1


def test_sampler_goal_chart_on_manifold(P, orc, arm):
    """Goal candidates decoded on the GPU satisfy Def. 2 (checked in FP64)
    and agree with the oracle's decoding where both accept."""
    toss = synth.random_toss(arm, 5)
    pr = synth.make_problem(toss, root=synth.random_states(arm, 1, 10)[0])
    B = 4096
    pl = P.Planner(arm, P=1, n_cap=64, b_max=B, k=1, K=8, S=8)
    prob = P.problem_struct(pr, B, B, seed=77)
    pl.reset([prob])
    pl.iterate([prob], 2, 0)
    c = pl.get_candidates(0, B)
    pl.close()
    st, Tq, vr, valid = orc.sample_goals(arm, pr, 77, 2, 0, 0, B)
    gv = c["valid"] == 1
    assert gv.sum() >= 20
    # acceptance agrees on all but a few near-tolerance samples
    assert np.mean(gv != (valid == 1)) < 0.01
    both = gv & (valid == 1)
    assert np.allclose(c["T_req"][both], Tq[both], rtol=1e-6)
    assert np.abs(c["states"][both, :7] - st[both, :7]).max() < 2e-3
    g = np.asarray(pr["g"])
    for i in np.nonzero(gv)[0]:
        q, qd, T = c["states"][i, :7].astype(float), c["states"][i, 8:15].astype(float), float(c["T_req"][i])
        x = pr["x0"] + pr["v0"] * T + 0.5 * g * T * T
        xd = pr["v0"] + g * T
        b0, b1 = orc.blade(arm, q)
        u = np.clip((x - b0) @ (b1 - b0) / ((b1 - b0) @ (b1 - b0)), 0, 1)
        assert np.linalg.norm(b0 + u * (b1 - b0) - x) < 1e-3
        v6 = orc.jacobian_point(arm, q, x) @ qd
        vrel = v6[:3] - xd
        assert np.linalg.norm(vrel) >= pr["v_min"] - 1e-3
        R, _ = orc.fk(arm, q)
        nb = R[7] @ arm["blade_normal"].astype(float)
        assert nb @ vrel / np.linalg.norm(vrel) >= pr["a_min"] - 3e-3
        assert np.all(q >= arm["q_lo"] - 1e-6) and np.all(q <= arm["q_hi"] + 1e-6)


@pytest.mark.parametrize("chord", [False, True])
def test_graph_replay_matches_iteration(P, orc, arm, chord):
    """A captured iteration (two branches: the goal branch on a side stream)
    computes what the same iteration computes launch by launch in one stream;
    with chord states the fork comes after the goal chart."""
    import torch
    case = make_case(arm, orc, 6, N=500)
    states, t, parent = case["tree"]
    N = states.shape[0]
    B = 512
    flags = P.FN_PLAN_CHORD if chord else 0
    res = []
    for mode in ("iterate", "graph", "async"):
        pl = P.Planner(arm, P=2, n_cap=N + 4 * B, b_max=B, k=8, K=64, S=32)
        if chord:
            pl.set_sampler(w_chord=0.6, chord_sigma=0.15)
        probs = [P.problem_struct(case["pr"], B, B // 2, root=case["root"], seed=11 + i)
                 for i in range(2)]
        pl.reset(probs)
        for p in range(2):
            pl.load_tree(p, states, t, parent)
        s = torch.cuda.Stream()
        outs = []
        if mode == "graph":
            pl.capture(flags, stream=s)
            for it in range(3):
                outs.append(pl.replay(probs, it, stream=s))
        elif mode == "async":
            from paper_2609_22608_gb300._lib import FnError
            with pytest.raises(FnError):
                pl.result()                              # nothing launched yet
            pl.capture(flags, stream=s)
            pl.replay_async(probs, 0, stream=s)
            outs.append(pl.result())
            pl.replay_async(probs, 1, stream=s)          # back to back: the second call
            pl.replay_async(probs, 2, stream=s)          # waits for the first's staging
            outs.append(None)
            outs.append(pl.result())
        else:
            for it in range(3):
                outs.append(pl.iterate(probs, it, flags, stream=s))
        res.append((outs, [pl.get_tree(p) for p in range(2)]))
        pl.close()
    (o1, t1) = res[0]
    for o2, t2 in res[1:]:
        for a, b in zip(o1, o2):
            if b is None:
                continue
            for x, y in zip(a, b):
                assert x["n_nodes"] == y["n_nodes"] and x["incumbent"] == y["incumbent"]
                assert x["J"] == y["J"] or (np.isnan(x["J"]) and np.isnan(y["J"]))
        for x, y in zip(t1, t2):
            assert np.array_equal(x["states"], y["states"])
            assert np.array_equal(x["parent"], y["parent"])


def test_batched_uneven_problems(P, orc, arm):
    """Three problems of different tree and batch sizes in one planner match
    three single-problem rounds on the oracle."""
    cases = [make_case(arm, orc, 10 + i, N=n, n_free=nf) for i, (n, nf) in
             enumerate([(50, 40), (700, 150), (260, 8)])]
    grid = synth.duration_grid(K_GRID)
    Bmax = max(c["cand"].shape[0] for c in cases)
    Nmax = max(c["tree"][0].shape[0] for c in cases)
    pl = P.Planner(arm, P=3, n_cap=Nmax + Bmax + 8, b_max=Bmax, k=5, K=K_GRID, S=S_COLL)
    probs = [P.problem_struct(c["pr"], c["cand"].shape[0], c["n_goal"], root=c["root"]) for c in cases]
    pl.reset(probs)
    for p, c in enumerate(cases):
        pl.load_tree(p, *c["tree"])
        pl.set_candidates(p, c["cand"], c["n_goal"], c["T_req"], c["v_rel"])
    outs = pl.iterate(probs, 0, P.FN_PLAN_EXTERNAL)
    for p, c in enumerate(cases):
        g = pl.get_tree(p)
        st, t, par = c["tree"]
        inc = dict(id=-1, J=-np.inf, t_best=float(np.float32(c["pr"]["t_fall"])))
        rtree, rinc, det = OP.plan_round(arm, c["pr"], OP.Tree(st, t, par), c["cand"], c["n_goal"],
                                         c["T_req"], c["v_rel"], inc, 5, grid, S_COLL)
        assert not compare_round(orc, arm, c, g, rtree, det, st.shape[0], grid)
        if rinc["id"] >= 0:
            assert outs[p]["J"] == pytest.approx(rinc["J"], rel=1e-4, abs=1e-4)
    pl.close()


def test_autotune_keeps_results(P, orc, arm):
    """Every schedule variant computes the same iteration."""
    case = make_case(arm, orc, 8, N=600)
    states, t, parent = case["tree"]
    B = 256
    trees = []
    for tune in (False, True):
        pl = P.Planner(arm, P=1, n_cap=states.shape[0] + B + 8, b_max=B, k=8, K=64, S=32)
        prob = P.problem_struct(case["pr"], B, B // 2, root=case["root"], seed=5)
        pl.reset([prob])
        pl.load_tree(0, states, t, parent)
        if tune:
            chosen, ms = pl.autotune([prob], 0, 0, reps=2)
            assert 0 <= chosen < 4 and len(ms) == 4 and all(m > 0 for m in ms)
        pl.iterate([prob], 0, 0)
        trees.append(pl.get_tree(0))
        pl.close()
    a, b = trees
    assert a["n"] == b["n"] and np.array_equal(a["states"], b["states"])
    assert np.array_equal(a["parent"], b["parent"]) and np.array_equal(a["t"], b["t"])


def test_plan_round_nary_refinement(P, orc, arm):
    """FN_PLAN_NARY: the free edges' grid durations are refined by the N-ary
    search before the attach.  Every attached free node must carry a valid
    refined duration (its check passes in FP64 within the margin, eps below
    it fails within the margin, and it is not above the grid duration), and
    the round must match the oracle's refined round candidate by candidate,
    except where one of the candidate's edges has a refined decision within
    the margin class (refined points sit within ~3e-5 T of the boundary)."""
    case = make_case(arm, orc, 3, N=400, n_goal_draw=256, n_free=192)
    # free candidates near the root, so that short free edges exist
    G = case["n_goal"]
    rng = np.random.default_rng(3)
    near = np.repeat(case["root"][None].astype(np.float64), case["cand"].shape[0] - G, axis=0)
    near[:, :7] += rng.normal(0, 0.15, (len(near), 7))
    near[:, 8:15] = rng.normal(0, 0.2, (len(near), 7))
    near[:, 7] = near[:, 15] = 0
    lo, hi = arm["q_lo"].astype(np.float64), arm["q_hi"].astype(np.float64)
    near[:, :7] = np.clip(near[:, :7], lo + 0.05, hi - 0.05)
    case["cand"] = np.concatenate([case["cand"][:G], near.astype(np.float32)])
    grid = synth.duration_grid(K_GRID)
    states, t, parent = case["tree"]
    N, B, k, eps = states.shape[0], case["cand"].shape[0], 5, 2e-4
    pl = P.Planner(arm, P=1, n_cap=N + B + 8, b_max=B, k=k, K=K_GRID, S=S_COLL, S_clear=8)
    pl.set_refine(eps, 8)
    prob = P.problem_struct(case["pr"], B, case["n_goal"], root=case["root"])
    pl.reset([prob])
    pl.load_tree(0, states, t, parent)
    pl.set_candidates(0, case["cand"], case["n_goal"], case["T_req"], case["v_rel"])
    pl.work_counts(reset=True)
    pl.iterate([prob], 0, P.FN_PLAN_EXTERNAL | P.FN_PLAN_NARY)
    wc = pl.work_counts()
    gtree = pl.get_tree(0)
    pl.close()
    assert wc["refine"] > 0
    inc = dict(id=-1, J=-np.inf, t_best=float(np.float32(case["pr"]["t_fall"])))
    rtree, _, det = OP.plan_round(arm, case["pr"], OP.Tree(states, t, parent), case["cand"],
                                  case["n_goal"], case["T_req"], case["v_rel"], inc, k, grid,
                                  S_COLL, S_clear=8, nary=(eps, 8))
    free_new = [i for i in range(N, gtree["n"]) if not np.isfinite(gtree["J"][i])]
    assert len(free_new) >= 10
    for i in free_new:
        p = int(gtree["parent"][i])
        T = float(gtree["t"][i]) - float(gtree["t"][p])
        s0, s1 = gtree["states"][p][None], gtree["states"][i][None]
        r_hi = orc.rho_batch(arm, s0, s1, [T], S_COLL)[0]
        assert max(r_hi[0], r_hi[1]) <= 1 + 1e-4 + 1e-5
        r_lo = orc.rho_batch(arm, s0, s1, [T - eps - 2e-6], S_COLL)[0]
        kg = int(np.searchsorted(grid, np.float32(T) - np.float32(1e-6), side="left"))
        assert kg < len(grid) and T <= float(grid[kg]) + 1e-6
        if T - eps > 1e-3:
            assert max(r_lo[0], r_lo[1]) > 1 - 1e-4
    # against the oracle's refined round, candidate by candidate: the same
    # parent and a time within the refined bracket, or else one of the
    # candidate's edges has its refined decision within the margin class:
    # some duration the oracle's N-ary search checked has max(rho_tau,
    # rho_P) within 1e-4 of 1 (its `margin` output), or rho_v at the refined
    # duration lies in its joint-box band
    from tests.parity import RHO_MARGIN, rho_v_ambiguous
    g_new = {gtree["states"][i].tobytes(): i for i in range(N, gtree["n"])}
    r_new = {rtree.states[i].tobytes(): i for i in range(N, rtree.n)}
    par, tree_t = det["parents"], t
    same, explained, total = 0, 0, 0
    for b in range(G, B):
        key = case["cand"][b].tobytes()
        gi, ri = g_new.get(key), r_new.get(key)
        if gi is None and ri is None:
            continue
        total += 1
        if gi is not None and ri is not None and gtree["parent"][gi] == rtree.parent[ri] and \
                abs(float(gtree["t"][gi]) - float(rtree.t[ri])) <= eps + 1e-4 * float(rtree.t[ri]):
            same += 1
            continue
        ok = False
        for j in range(k):
            pj = int(par[b, j])
            if pj < 0:
                continue
            cap = np.array([np.float32(np.float32(inc["t_best"]) - np.float32(tree_t[pj]))])
            s0, s1 = states[pj][None], case["cand"][b][None]
            rn = orc.time_edges_nary(arm, s0, s1, grid, S_COLL, eps, 8, T_cap=cap)
            if rn["margin"][0] <= RHO_MARGIN or (
                    rn["k_star"][0] >= 0 and
                    rho_v_ambiguous(orc, arm, s0[0], s1[0], float(rn["T_star"][0]), S_COLL)):
                ok = True
                break
        explained += ok
        assert ok, f"candidate {b} differs from the oracle's refined round outside the margin class"
    assert total >= 10 and same + explained == total, (same, explained, total)
