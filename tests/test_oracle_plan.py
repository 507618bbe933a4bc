"""Pins of the oracle's planning round (Algorithm 1's inner body, oracle/plan.py)
against the algorithm's rules, with the per-edge verdicts taken as given (the
edge check itself is pinned in test_oracle_edges.py):

* Parents: the root plus the k-1 nearest non-root nodes, recomputed here by a
  brute-force numpy scan of the metric.
* Goal edges take T_p = T_req - t(p); free edges a grid duration with
  t(p) + T <= t_best; both in single precision.
* Attach: each candidate goes to the ok parent of least t(p) + T_p (ties to
  the lower slot), new nodes appended in candidate order, t(node) = t(p) + T_p.
* nu is the largest rho_v along the path; J is set on goal nodes only.
* The incumbent is the best new rendezvous node (lower id on ties) and only
  replaces a strictly worse one.
* A planted tie (a duplicated tree node) goes to the lower slot.
"""
import numpy as np

import oracle.plan as OP
from paper_2609_22608_gb300 import synth

F32 = np.float32
K_GRID, S_COLL, K_PAR, W_VEL = 64, 32, 5, 0.1


def _case(arm, orc, seed, N=120, n_goal_draw=512, n_free=40):
    """A random tree plus, for each decoded goal, an approach node 0.1 s
    before it on its own velocity (so that goal edges can pass), decoded
    goal candidates, and free candidates near the root at low speed (so
    that free edges fit under the cap)."""
    toss = synth.random_toss(arm, seed)
    root = synth.random_states(arm, 1, 5000 + seed)[0]
    pr = synth.make_problem(toss, root=root)
    states, parent, t = synth.random_tree(arm, N, seed, root=root)
    st, Tq, vr, valid = orc.sample_goals(arm, pr, 100 + seed, 0, 0, 0, n_goal_draw)
    gi = np.nonzero(valid)[0]
    goal = st[gi].astype(F32)
    appr = goal.astype(np.float64)
    appr[:, :7] -= 0.1 * appr[:, 8:15]
    states = np.concatenate([states, appr.astype(F32)])
    t = np.concatenate([t, (Tq[gi] - 0.1).astype(F32)])
    parent = np.concatenate([parent, np.zeros(len(gi), parent.dtype)])
    rng = np.random.default_rng(seed)
    free = np.repeat(np.asarray(root, F32)[None], n_free, axis=0)
    free[:, :7] += rng.uniform(-0.3, 0.3, (n_free, 7)).astype(F32)
    free[:, 8:15] = rng.uniform(-0.2, 0.2, (n_free, 7)).astype(F32)
    free[:, 7] = free[:, 15] = 0.0
    cand = np.concatenate([goal, free])
    nu = rng.uniform(0.0, 1.0, states.shape[0])   # path maxima of rho_v carried by the nodes
    nu[0] = 0.0
    return dict(pr=pr, tree=OP.Tree(states, t, parent, nu=nu), cand=cand, n_goal=len(gi),
                T_req=Tq[gi].astype(F32), v_rel=vr[gi].astype(F32))


def _metric(a, b):
    a = a.astype(np.float64)
    b = b.astype(np.float64)
    return np.sum((a[..., :7] - b[..., :7]) ** 2, -1) + W_VEL * np.sum((a[..., 8:15] - b[..., 8:15]) ** 2, -1)


def _check_round(arm, orc, case, inc0, grid):
    tree = case["tree"]
    out, inc, det = OP.plan_round(arm, case["pr"], tree, case["cand"], case["n_goal"],
                                  case["T_req"], case["v_rel"], inc0, K_PAR, grid, S_COLL)
    par, ok, T, rv = det["parents"], det["ok"], det["T"], det["rv"]
    B, G, N0 = case["cand"].shape[0], case["n_goal"], tree.n
    # parents: root + the k-1 nearest non-root nodes by brute force
    for b in range(B):
        d = _metric(tree.states[1:], case["cand"][b])
        order = np.argsort(d, kind="stable")[:K_PAR - 1] + 1
        assert par[b, 0] == 0
        got = par[b, 1:]
        if not np.array_equal(got, order):
            dg = _metric(tree.states[got], case["cand"][b])
            do = _metric(tree.states[order], case["cand"][b])
            assert np.allclose(np.sort(dg), np.sort(do), rtol=1e-6)
    # durations: goal T_p = T_req - t(p); free within the cap, on the grid
    tp = tree.t[par]
    for b in range(B):
        for j in range(K_PAR):
            if b < G:
                assert T[b, j] == F32(F32(case["T_req"][b]) - tp[b, j])
            elif ok[b, j]:
                assert T[b, j] <= F32(F32(inc0["t_best"]) - tp[b, j])
                assert np.any(grid.astype(F32) == T[b, j])
    # attach: argmin of t(p) + T_p over the ok parents, ties to the lower
    # slot, appended in candidate order
    attached = {b: (j, bt) for b, j, bt in det["attached"]}
    assert [b for b, _, _ in det["attached"]] == sorted(attached)
    for b in range(B):
        okj = [j for j in range(K_PAR) if ok[b, j]]
        if not okj:
            assert b not in attached
            continue
        tt = [F32(tp[b, j] + T[b, j]) for j in okj]
        best = okj[int(np.argmin(tt))]          # argmin takes the first minimum
        j, bt = attached[b]
        assert j == best and bt == min(tt)
    # the new nodes
    assert out.n == N0 + len(attached)
    for r, (b, j, bt) in enumerate(det["attached"]):
        nd = N0 + r
        p = int(par[b, j])
        assert out.parent[nd] == p and np.array_equal(out.states[nd], case["cand"][b])
        assert out.t[nd] == F32(out.t[p] + T[b, j])
        assert out.nu[nd] == max(float(out.nu[p]), float(rv[b, j]))
        assert np.isfinite(out.J[nd]) == (b < G)
    # the incumbent
    new = np.arange(N0, out.n)
    Jn = out.J[new]
    fin = np.isfinite(Jn)
    if fin.any() and Jn[fin].max() > inc0["J"]:
        best = new[fin][np.argmax(Jn[fin])]       # the lowest id among equal maxima
        assert inc["id"] == best and inc["J"] == out.J[best]
        assert inc["t_best"] == float(out.t[best])
    else:
        assert inc == inc0
    return out, inc, det


def test_round_follows_algorithm_rules(orc, arm):
    grid = synth.duration_grid(K_GRID)
    for seed in (3, 4):
        case = _case(arm, orc, seed)
        assert case["n_goal"] >= 2
        inc0 = dict(id=-1, J=-np.inf, t_best=float(F32(case["pr"]["t_fall"])))
        out, inc, det = _check_round(arm, orc, case, inc0, grid)
        assert len(det["attached"]) >= 5
        assert inc["id"] >= case["tree"].n          # a new rendezvous node became incumbent
        # a strictly better incumbent is required: an incumbent as good as the
        # round's best new node is kept
        _, inc2, _ = _check_round(arm, orc, case, dict(id=7, J=inc["J"], t_best=inc0["t_best"]),
                                  grid)
        assert inc2["id"] == 7


def test_attach_tie_goes_to_lower_slot(orc, arm):
    """A tree node duplicated at the end of the tree ties with its original
    in distance and in t(p) + T_p; the candidate must attach to the
    original (the lower parent slot)."""
    grid = synth.duration_grid(K_GRID)
    case = _case(arm, orc, 5, n_free=12)
    tree = case["tree"]
    G = case["n_goal"]
    # free candidates placed next to node 7, which is duplicated
    src = 7
    dup = OP.Tree(np.concatenate([tree.states, tree.states[src:src + 1]]),
                  np.concatenate([tree.t, tree.t[src:src + 1]]),
                  np.concatenate([tree.parent, tree.parent[src:src + 1]]),
                  nu=np.concatenate([tree.nu, tree.nu[src:src + 1]]))
    rng = np.random.default_rng(0)
    free = np.repeat(tree.states[src:src + 1], 12, axis=0).astype(F32)
    free[:, :7] += rng.uniform(-0.05, 0.05, (12, 7)).astype(F32)
    free[:, 8:15] *= F32(0.5)
    case2 = dict(case, tree=dup, cand=np.concatenate([case["cand"][:G], free]))
    inc0 = dict(id=-1, J=-np.inf, t_best=10.0)
    out, inc, det = _check_round(arm, orc, case2, inc0, grid)
    N0 = dup.n
    hits = 0
    for b, j, bt in det["attached"]:
        if b < G:
            continue
        slots = list(det["parents"][b])
        assert src in slots and N0 - 1 in slots
        assert slots.index(src) < slots.index(N0 - 1)
        p = int(det["parents"][b, j])
        if det["ok"][b, slots.index(src)]:
            assert p != N0 - 1            # the duplicate never wins the tie
            hits += p == src
    assert hits >= 3


def test_incumbent_tie_goes_to_lower_id(orc, arm):
    """The best goal candidate duplicated right after the goals attaches
    twice with the same J; the incumbent must be the earlier node."""
    grid = synth.duration_grid(K_GRID)
    case = _case(arm, orc, 3)
    G = case["n_goal"]
    inc0 = dict(id=-1, J=-np.inf, t_best=float(F32(case["pr"]["t_fall"])))
    _, inc, det = OP.plan_round(arm, case["pr"], case["tree"], case["cand"], G, case["T_req"],
                                case["v_rel"], inc0, K_PAR, grid, S_COLL)
    b_best = [b for b, _, _ in det["attached"]][inc["id"] - case["tree"].n]
    assert b_best < G
    sel = list(range(G)) + [b_best]
    case2 = dict(case, cand=np.concatenate([case["cand"][sel], case["cand"][G:]]), n_goal=G + 1,
                 T_req=case["T_req"][sel], v_rel=case["v_rel"][sel])
    out, inc2, det2 = _check_round(arm, orc, case2, inc0, grid)
    rows = {b: case2["tree"].n + r for r, (b, _, _) in enumerate(det2["attached"])}
    assert b_best in rows and G in rows
    assert out.J[rows[b_best]] == out.J[rows[G]] == inc2["J"]
    assert inc2["id"] == rows[b_best]


def test_prune_rules(orc, arm):
    """Eq. (reach) pruning: the root and the incumbent's path stay; any other
    node stays only if its reach time exists, is no later than t_best and
    its parent stays; the kept nodes keep their order and their parents are
    re-indexed; the incumbent id follows its node."""
    toss = synth.random_toss(arm, 9)
    root = synth.random_states(arm, 1, 59)[0]
    pr = synth.make_problem(toss, root=root)
    states, parent, t = synth.random_tree(arm, 150, 9, root=root)
    tree = OP.Tree(states, t, parent)
    # the incumbent: a deep node
    depth = np.zeros(tree.n, int)
    for i in range(1, tree.n):
        depth[i] = depth[tree.parent[i]] + 1
    inc_id = int(np.argmax(depth))
    path = set()
    c = inc_id
    while c > 0:
        path.add(c)
        c = int(tree.parent[c])
    reach = {}
    for i in range(1, tree.n):
        g, Tn = orc.reach_time(arm, pr, tree.states[i, :7].astype(np.float64), float(tree.t[i]), 64)
        reach[i] = (g, Tn)
    t_best = float(np.median([Tn for g, Tn in reach.values() if g >= 0]))
    inc = dict(id=inc_id, J=1.0, t_best=t_best)
    out, inc2, alive = OP.prune_tree(arm, pr, tree, inc, G=64)

    def stays(i):
        if i == 0 or i in path:
            return True
        g, Tn = reach[i]
        return g >= 0 and Tn <= t_best and stays(int(tree.parent[i]))

    expect = np.array([stays(i) for i in range(tree.n)])
    assert np.array_equal(alive, expect)
    assert 0 < expect.sum() < tree.n
    assert any(not (reach[i][0] >= 0 and reach[i][1] <= t_best) for i in path)   # kept by the path rule
    assert any(reach[i][0] >= 0 and reach[i][1] <= t_best and not expect[i]
               for i in range(1, tree.n))                                       # removed with an ancestor
    idx = np.nonzero(expect)[0]
    assert np.array_equal(out.states, tree.states[idx]) and np.array_equal(out.t, tree.t[idx])
    for new, old in enumerate(idx):
        if old == 0:
            assert out.parent[new] == -1
        else:
            assert idx[out.parent[new]] == tree.parent[old]
    assert idx[inc2["id"]] == inc_id
