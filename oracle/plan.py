"""One round of Algorithm 1 on the FP64 oracle -- TEST INFRASTRUCTURE ONLY.

Follows the algorithm's inner body in its order (Parents, the goal / free
branches, Clear, attach, incumbent, Prune) over the oracle's C primitives.
Where floating point decides an integer (the duration cap t_best - t(p), the
goal duration T_req - t(p), the time-to-come t(p) + T_p and its argmin), the
decision is taken in FP32 like the library's kernels.  Readings:
  * parents are the root plus the k-1 nearest non-root nodes;
  * free candidates take the first feasible grid duration with
    t(p) + T <= t_best (time-to-come bound), refined by the N-ary search
    when `nary` = (eps, max_rounds) is given (Clear then at the refined T);
  * ties of the attach argmin go to the lower parent slot, of the incumbent
    argmax to the lower node id; a new incumbent must be strictly better;
  * a rendezvous node's nu is the largest rho_v along its path;
  * pruning keeps the root and the incumbent's path, removes the other nodes
    whose Eq. (reach) time is missing or later than t_best, and removes
    descendants of removed nodes.
"""
from __future__ import annotations

import numpy as np

import oracle as O

F32 = np.float32


def fsub(a, b):
    return F32(F32(a) - F32(b))


def fadd(a, b):
    return F32(F32(a) + F32(b))


class Tree:
    def __init__(self, states, t, parent, J=None, nu=None, eT=None):
        n = states.shape[0]
        self.states = np.asarray(states, F32).copy()
        self.t = np.asarray(t, F32).copy()
        self.parent = np.asarray(parent, np.int64).copy()
        self.J = np.full(n, np.nan) if J is None else np.asarray(J, np.float64).copy()
        self.nu = np.zeros(n) if nu is None else np.asarray(nu, np.float64).copy()
        self.eT = np.full(n, np.nan, F32) if eT is None else np.asarray(eT, F32).copy()
        if eT is None and n:
            self.eT[0] = 0.0

    @property
    def n(self):
        return self.states.shape[0]


def plan_round(arm, pr, tree: Tree, cand, n_goal, T_req, v_rel, inc, k, grid, S, S_clear=8,
               w_vel=0.1, obstacles=None, margin=0.02, prune=False, reach_grid=256, nary=None):
    """Returns (tree, incumbent dict, details).  inc = dict(id, J, t_best)."""
    cand = np.asarray(cand, F32)
    B = cand.shape[0]
    inc = dict(inc)
    # Parents: root + (k-1) nearest non-root nodes
    if k > 1 and tree.n > 1:
        nn, _ = O.knn(tree.states, cand, k - 1, w_vel, first=1)
    else:
        nn = np.full((B, max(k - 1, 0)), -1, np.int64)
    par = np.concatenate([np.zeros((B, 1), np.int64), nn.astype(np.int64)], axis=1)
    tp = np.where(par >= 0, tree.t[np.clip(par, 0, None)], F32(0)).astype(F32)
    valid_par = par >= 0
    E = B * k
    s0 = tree.states[np.clip(par, 0, None).reshape(-1)]
    s1 = np.repeat(cand, k, axis=0)
    ok = np.zeros((B, k), bool)
    Tedge = np.full((B, k), np.inf, F32)
    rv = np.full((B, k), np.nan)
    # goal branch: one check at T_req - t(p)
    if n_goal > 0:
        g = slice(0, n_goal * k)
        Tg = np.array([fsub(T_req[b], tp[b, j]) for b in range(n_goal) for j in range(k)], F32)
        rg = O.time_edges(arm, s0[g], s1[g], grid, S, mode=1, T_fixed=Tg)
        ok[:n_goal] = (rg["ok"] == 1).reshape(n_goal, k)
        Tedge[:n_goal] = Tg.reshape(n_goal, k)
        rv[:n_goal] = rg["rho3"][:, 2].reshape(n_goal, k)
    # free branch: first feasible grid duration with t(p) + T <= t_best
    if B > n_goal:
        f = slice(n_goal * k, E)
        cap = np.array([fsub(inc["t_best"], tp[b, j]) for b in range(n_goal, B) for j in range(k)], F32)
        if nary is None:
            rf = O.time_edges(arm, s0[f], s1[f], grid, S, T_cap=cap)
        else:   # the grid duration refined by the N-ary search, rho_v at the refined T
            rf = O.time_edges_nary(arm, s0[f], s1[f], grid, S, nary[0], nary[1], T_cap=cap)
        ok[n_goal:] = (rf["ok"] == 1).reshape(B - n_goal, k)
        Tedge[n_goal:] = rf["T_star"].reshape(B - n_goal, k)
        rv[n_goal:] = rf["rho3"][:, 2].reshape(B - n_goal, k)
    ok &= valid_par
    # Clear
    if obstacles is not None and len(obstacles) > 0:
        for b in range(B):
            for j in range(k):
                if ok[b, j]:
                    c = O.edge_clearance(arm, s0[b * k + j], s1[b * k + j], float(Tedge[b, j]),
                                         S_clear, obstacles)
                    ok[b, j] = c >= margin
    # attach: argmin_p t(p) + T_p over ok parents, ties to the lower slot,
    # appended in candidate order
    new = []
    for b in range(B):
        best, bt = -1, np.inf
        for j in range(k):
            if not ok[b, j]:
                continue
            tt = fadd(tp[b, j], Tedge[b, j])
            if tt < bt:
                bt, best = tt, j
        if best >= 0:
            new.append((b, best, bt))
    n0 = tree.n
    st = [tree.states]
    t_new, par_new, J_new, nu_new, eT_new = [], [], [], [], []
    bestJ, bestI = -np.inf, None
    for r, (b, j, bt) in enumerate(new):
        p = int(par[b, j])
        nu = max(float(tree.nu[p]), float(rv[b, j]))
        Jv = np.nan
        if b < n_goal:
            Jv = O.objective(pr, float(bt), float(v_rel[b]), nu)
            if Jv > bestJ:
                bestJ, bestI = Jv, n0 + r
        st.append(cand[b:b + 1])
        t_new.append(bt); par_new.append(p); J_new.append(Jv); nu_new.append(nu)
        eT_new.append(Tedge[b, j])
    out = Tree(np.concatenate(st), np.concatenate([tree.t, np.array(t_new, F32)]),
               np.concatenate([tree.parent, np.array(par_new, np.int64)]),
               np.concatenate([tree.J, np.array(J_new)]), np.concatenate([tree.nu, np.array(nu_new)]),
               np.concatenate([tree.eT, np.array(eT_new, F32)]))
    # incumbent: argmax J over rendezvous nodes (only new nodes can change it)
    if bestI is not None and bestJ > inc["J"]:
        inc = dict(id=bestI, J=bestJ, t_best=float(out.t[bestI]))
    details = dict(parents=par, ok=ok, T=Tedge, rv=rv, attached=new)
    if prune:
        out, inc, kept = prune_tree(arm, pr, out, inc, reach_grid)
        details["kept"] = kept
    return out, inc, details


def prune_tree(arm, pr, tree: Tree, inc, G=256):
    """Eq. (reach) pruning (readings in the module docstring)."""
    n = tree.n
    keep = np.zeros(n, bool)
    keep[0] = True
    for i in range(1, n):
        g, Tn = O.reach_time(arm, pr, tree.states[i, :7].astype(np.float64), float(tree.t[i]), G)
        keep[i] = g >= 0 and Tn <= inc["t_best"]
    c = inc["id"]
    while c is not None and c > 0:
        keep[c] = True
        c = int(tree.parent[c])
    alive = keep.copy()
    for i in range(1, n):   # parents precede children
        alive[i] = alive[i] and alive[tree.parent[i]]
    newidx = np.cumsum(alive) - 1
    idx = np.nonzero(alive)[0]
    par = np.array([newidx[tree.parent[i]] if tree.parent[i] >= 0 else -1 for i in idx], np.int64)
    out = Tree(tree.states[idx], tree.t[idx], par, tree.J[idx], tree.nu[idx], tree.eT[idx])
    inc = dict(inc)
    if inc["id"] >= 0:
        inc["id"] = int(newidx[inc["id"]])
    return out, inc, alive


def first_segment(tree: Tree, inc):
    """End state and duration of the incumbent plan's first edge."""
    c = inc["id"]
    if c is None or c <= 0:
        return None
    while tree.parent[c] > 0:
        c = int(tree.parent[c])
    return tree.states[c], float(tree.eT[c])
