"""Comparison rules between the CUDA path and the FP64 oracle.

* torques: per sample, max_j |tau_gpu - tau_ref| <= 1e-5 * max(|tau_ref|_inf, 1 N m)
  (the 1e-5 relative FP32 bar, measured against the sample's torque scale so
  that near-zero components do not make it ill-posed);
* minimum-time index: k_gpu == k_ref, except where some grid index j between
  the two (inclusive) has |max(rho_tau, rho_P)(T_j) - 1| <= 1e-4 in the oracle;
* kNN: index lists equal, except positions where the two distances at the
  k/k+1 boundary differ by <= 1e-6 relative.
"""
import numpy as np

TAU_REL = 1e-5
RHO_MARGIN = 1e-4
KNN_REL = 1e-6


def torque_ok(tau_gpu, tau_ref):
    tau_gpu = np.asarray(tau_gpu, np.float64)
    scale = np.maximum(np.abs(tau_ref).max(axis=-1), 1.0)
    err = np.abs(tau_gpu - tau_ref).max(axis=-1)
    return err <= TAU_REL * scale, err / scale


def kstar_mismatches(orc, arm, s0, s1, grid, S, k_gpu, k_ref, T_cap=None):
    """Indices of edges whose k* differ beyond the margin rule."""
    bad = []
    K = len(grid)
    for e in np.nonzero(k_gpu != k_ref)[0]:
        kg, kr = int(k_gpu[e]), int(k_ref[e])
        if kg == -2 or kr == -2:
            bad.append(e)
            continue
        Kadm = K
        if T_cap is not None:
            Kadm = int(np.sum(grid <= T_cap[e]))
        a = kg if kg >= 0 else Kadm - 1
        b = kr if kr >= 0 else Kadm - 1
        lo, hi = min(a, b), max(a, b)
        js = np.arange(lo, hi + 1)
        rr = orc.rho_batch(arm, np.repeat(s0[e:e + 1], len(js), 0), np.repeat(s1[e:e + 1], len(js), 0),
                           grid[js].astype(np.float64), S)
        m = np.maximum(rr[:, 0], rr[:, 1])
        if not np.any(np.abs(m - 1.0) <= RHO_MARGIN):
            bad.append(e)
    return bad


def knn_mismatches(idx_gpu, d_gpu, idx_ref, d_ref):
    bad = []
    for b in range(idx_ref.shape[0]):
        if np.array_equal(idx_gpu[b], idx_ref[b]):
            continue
        # allow permutations/substitutions among near-equal distances
        ok = True
        for j in range(idx_ref.shape[1]):
            if idx_gpu[b, j] == idx_ref[b, j]:
                continue
            da, db = float(d_ref[b, j]), float(d_gpu[b, j])
            if not (np.isfinite(da) and np.isfinite(db)):
                ok = False
                break
            # the swapped entries must be near-ties in the exact distances
            tol = KNN_REL * max(abs(da), abs(db))
            if abs(da - db) > tol + 1e-6 * max(da, 1e-12):
                ok = False
                break
        if not ok:
            bad.append(b)
    return bad


def near_margin(orc, arm, s0, s1, grid, S, T_goal=None):
    """Is the edge's decision within the margin class?  For a free edge, any
    grid duration with max(rho_tau, rho_P) or rho_v within 1e-4 of 1; for a
    goal edge (T_goal = its fixed duration T_p), the same at T_p alone, with
    rho_v's joint-box band (rho_v_ambiguous)."""
    if T_goal is not None:
        T = np.array([float(T_goal)])
        if not (T[0] > 0):
            return False
        rr = orc.rho_batch(arm, s0[None], s1[None], T, S)
        return bool(abs(max(rr[0, 0], rr[0, 1]) - 1) <= RHO_MARGIN or
                    rho_v_ambiguous(orc, arm, s0, s1, T[0], S))
    rr = orc.rho_batch(arm, np.repeat(s0[None], len(grid), 0), np.repeat(s1[None], len(grid), 0),
                       grid.astype(np.float64), S)
    m = np.maximum(rr[:, 0], rr[:, 1])
    return bool(np.any(np.abs(m - 1) <= 1e-4) or np.any(np.abs(rr[:, 2] - 1) <= 1e-4))


def compare_round(orc, arm, case, gpu_tree, ref_tree, ref_details, n_old, grid, S=16):
    """Map new nodes to candidates by state and compare (parent, t)."""
    cand = case["cand"]
    g_new = {gpu_tree["states"][i].tobytes(): i for i in range(n_old, gpu_tree["n"])}
    r_new = {ref_tree.states[i].tobytes(): i for i in range(n_old, ref_tree.n)}
    bad = []
    for b in range(cand.shape[0]):
        key = cand[b].tobytes()
        gi, ri = g_new.get(key), r_new.get(key)
        if gi is None and ri is None:
            continue
        if gi is not None and ri is not None:
            if gpu_tree["parent"][gi] == ref_tree.parent[ri] and \
                    gpu_tree["t"][gi] == ref_tree.t[ri]:
                continue
        # disagreement: must be explained by a near-margin edge of this candidate
        par = ref_details["parents"][b]
        goal = b < case["n_goal"]
        explained = False
        for j, p in enumerate(par):
            if p < 0:
                continue
            s0 = ref_tree.states[p] if p < n_old else None
            if s0 is None:
                continue
            Tg = ref_details["T"][b, j] if goal else None
            if near_margin(orc, arm, s0, cand[b], grid, S, T_goal=Tg):
                explained = True
                break
        if not explained:
            bad.append(b)
    return bad


def arm_limits_moved(arm, delta):
    """Copy of `arm` with every joint box widened by `delta` (narrowed if < 0)."""
    a = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in arm.items()}
    a["q_lo"] = (arm["q_lo"].astype(np.float64) - delta).astype(np.float32)
    a["q_hi"] = (arm["q_hi"].astype(np.float64) + delta).astype(np.float32)
    return a


RHO_REL = 2e-5
# rho_v divides by the sqrt taper, whose slope is unbounded at a joint limit;
# a decision rho_v <= 1 counts as ambiguous when the oracle's rho_v with the
# joint boxes widened and narrowed by RHO_V_BOX rad straddles 1 (widened by
# RHO_REL).  RHO_V_BOX is about 2 ulp of a joint angle near pi in single
# precision, the rounding the kernels' positions carry.
RHO_V_BOX = 4e-6


def rho_v_ambiguous(orc, arm, s0, s1, T, S):
    """Can the FP32 rounding of the positions flip rho_v(T) <= 1?"""
    s0 = np.asarray(s0, np.float32)[None]
    s1 = np.asarray(s1, np.float32)[None]
    Ta = np.array([float(T)])
    lo = orc.rho_batch(arm_limits_moved(arm, RHO_V_BOX), s0, s1, Ta, S)[0, 2]
    hi = orc.rho_batch(arm_limits_moved(arm, -RHO_V_BOX), s0, s1, Ta, S)[0, 2]
    return bool(lo * (1 - RHO_REL) <= 1.0 <= hi * (1 + RHO_REL) or
                (np.isinf(hi) and lo <= 1.0 + RHO_REL))


def edge_distance(tree, q, w_vel):
    """Exact (FP64) parent distance of Sec. IV-E "Parents" from query row q
    to every row of tree: sum (q - q')^2 + w_v sum (qd - qd')^2."""
    t = np.asarray(tree, np.float64)
    q = np.asarray(q, np.float64)
    return ((t[:, :7] - q[:7]) ** 2).sum(1) + w_vel * ((t[:, 8:15] - q[8:15]) ** 2).sum(1)


def verify_iteration(orc, arm, pr, tree, t_best, cand, n_goal, nn_gpu, edges_gpu, tree_gpu,
                     grid, S, k, w_vel=0.1, S_clear=8, obstacles=None, margin=0.02,
                     inc_before=None, inc_gpu=None):
    """Every edge of one planner iteration against the oracle (Algorithm 1's
    inner body: Parents, the goal / free branches, Clear, attach, incumbent).

    tree: dict(states, t, parent[, nu]) before the iteration; t_best: the
    incumbent bound it ran with; cand: fn_planner_get_candidates' dict
    (slots < n_goal are goal draws); nn_gpu: fn_planner_get_parents;
    edges_gpu: fn_planner_get_edges; tree_gpu: fn_planner_get_tree after it;
    inc_before / inc_gpu: dict(id, J) before and the rendezvous after.

    Rules: parent lists equal except near-ties (KNN_REL) at differing
    positions; every edge of the GPU's parent lists re-timed by the oracle
    (goal: one check at T_p = T_req - t(p) in FP32; free: the first feasible
    grid index with T_k <= t_best - t(p)), with the k* margin rule and the
    rho_v band; the attach (argmin t(p) + T over ok edges, ties to the lower
    slot, appended in candidate order) exact given the GPU's edges; new
    nodes' nu exact, J within 1e-4 relative of the FP64 objective; the
    incumbent the strictly better argmax (ties to the lower id).
    Returns counts; "edge_mismatches", "parent_mismatches",
    "attach_mismatches" and "incumbent_ok" are the verdict."""
    F32 = np.float32
    st = np.asarray(tree["states"], F32)
    tt = np.asarray(tree["t"], F32)
    nu0 = np.asarray(tree.get("nu", np.zeros(len(tt))), np.float64)
    n_old = st.shape[0]
    states = np.asarray(cand["states"], F32)
    B = states.shape[0]
    valid = np.asarray(cand["valid"]) == 1
    KN = k - 1
    out = dict(candidates=int(B), valid_candidates=int(valid.sum()),
               valid_goals=int(valid[:n_goal].sum()), parent_mismatches=0, edge_mismatches=0,
               edges_explained_by_margin=0, attach_mismatches=0)
    # parents
    par = np.full((B, k), -1, np.int64)
    par[:, 0] = 0
    if KN > 0:
        par[:, 1:] = np.asarray(nn_gpu, np.int64)[:, :KN]
    vb = np.nonzero(valid)[0]
    if KN > 0 and n_old > 1 and len(vb):
        ref_i, ref_d = orc.knn(st, states[vb], KN, w_vel, first=1)
        bad = 0
        for r, b in enumerate(vb):
            gi = par[b, 1:]
            if np.array_equal(gi, ref_i[r]):
                continue
            good = len(set(gi[gi >= 0])) == int((gi >= 0).sum()) and np.all((gi >= 1) | (gi == -1))
            d_all = edge_distance(st, states[b], w_vel)
            for j in range(KN):
                if not good:
                    break
                if gi[j] == ref_i[r, j]:
                    continue
                if gi[j] < 0 or ref_i[r, j] < 0:
                    good = False
                    break
                da, db = float(ref_d[r, j]), float(d_all[gi[j]])
                good = abs(da - db) <= KNN_REL * max(abs(da), abs(db)) + 1e-12
            bad += 0 if good else 1
        out["parent_mismatches"] = bad
    # edges over the GPU's parent lists
    eb, ej = np.nonzero(valid[:, None] & (par >= 0))
    out["edges_formed"] = int(len(eb))
    goal = eb < n_goal
    pp = par[eb, ej]
    s0 = st[pp]
    s1 = states[eb]
    ok_ref = np.zeros(len(eb), bool)
    k_ref = np.full(len(eb), -1, np.int64)
    T_ref = np.full(len(eb), np.nan, F32)
    rv_ref = np.full(len(eb), np.nan)
    T_goal = np.array([F32(F32(cand["T_req"][b]) - tt[p]) for b, p in zip(eb[goal], pp[goal])], F32)
    if goal.any():
        r = orc.time_edges(arm, s0[goal], s1[goal], grid, S, mode=1, T_fixed=T_goal)
        ok_ref[goal] = r["ok"] == 1
        k_ref[goal] = r["k_star"]
        T_ref[goal] = T_goal
        rv_ref[goal] = r["rho3"][:, 2]
    fr = ~goal
    cap = np.array([F32(F32(t_best) - tt[p]) for p in pp[fr]], F32)
    if fr.any():
        r = orc.time_edges(arm, s0[fr], s1[fr], grid, S, T_cap=cap)
        ok_ref[fr] = r["ok"] == 1
        k_ref[fr] = r["k_star"]
        T_ref[fr] = r["T_star"]
        rv_ref[fr] = r["rho3"][:, 2]
    out["edges_with_duration"] = int((T_goal > 0).sum() + (cap >= grid[0]).sum())
    clear_ref = np.full(len(eb), np.inf)
    if obstacles is not None and len(obstacles):
        for i in np.nonzero(ok_ref)[0]:
            clear_ref[i] = orc.edge_clearance(arm, s0[i], s1[i], float(T_ref[i]), S_clear, obstacles)
        ok_ref &= clear_ref >= margin
    pos = np.zeros(len(eb), np.int64)      # index of each edge among its branch's edges
    pos[goal] = np.arange(int(goal.sum()))
    pos[fr] = np.arange(int(fr.sum()))
    kg = np.asarray(edges_gpu["k_star"])[eb, ej]
    Tg = np.asarray(edges_gpu["T"])[eb, ej]
    okg = np.asarray(edges_gpu["ok"])[eb, ej] == 1
    K = len(grid)
    for i in range(len(eb)):
        same_k = True
        if goal[i]:
            T_ok = Tg[i] == T_goal[pos[i]] or (np.isnan(Tg[i]) and np.isnan(T_goal[pos[i]]))
            same_k = (kg[i] == 0) == (k_ref[i] == 0)
        else:
            T_ok = (kg[i] < 0 and not np.isfinite(Tg[i])) or (0 <= kg[i] < K and Tg[i] == grid[kg[i]])
            same_k = kg[i] == k_ref[i]
        if T_ok and same_k and okg[i] == ok_ref[i]:
            continue
        if not T_ok:
            out["edge_mismatches"] += 1
            if len(out.setdefault("first_mismatches", [])) < 8:
                out["first_mismatches"].append(dict(
                    candidate=int(eb[i]), slot=int(ej[i]), goal=bool(goal[i]), k_gpu=int(kg[i]),
                    T_gpu=float(Tg[i]), T_ref=float(T_ref[i]), why="duration"))
            continue
        # a difference: must lie in the margin class of its own decision
        explained = False
        if goal[i]:
            explained = near_margin(orc, arm, s0[i], s1[i], grid, S, T_goal=Tg[i])
        elif not same_k:
            Tc = cap[pos[i]]
            explained = not kstar_mismatches(orc, arm, s0[i:i + 1], s1[i:i + 1], grid, S,
                                             np.array([kg[i]]), np.array([k_ref[i]]),
                                             T_cap=np.array([Tc]))
        else:
            explained = rho_v_ambiguous(orc, arm, s0[i], s1[i], float(Tg[i]), S)
        if not explained and np.isfinite(clear_ref[i]):
            explained = abs(clear_ref[i] - margin) <= 1e-4
        if explained:
            out["edges_explained_by_margin"] += 1
        else:
            out["edge_mismatches"] += 1
            if len(out.setdefault("first_mismatches", [])) < 8:
                out["first_mismatches"].append(dict(
                    candidate=int(eb[i]), slot=int(ej[i]), parent=int(pp[i]), goal=bool(goal[i]),
                    k_gpu=int(kg[i]), k_ref=int(k_ref[i]), T_gpu=float(Tg[i]),
                    T_ref=float(T_ref[i]), ok_gpu=bool(okg[i]), ok_ref=bool(ok_ref[i]),
                    rho_v_ref=float(rv_ref[i])))
    # attach, exact given the GPU's edges
    okG = np.asarray(edges_gpu["ok"]) == 1
    TG = np.asarray(edges_gpu["T"], F32)
    rvG = np.asarray(edges_gpu["rho_v"], F32)
    new = []
    for b in vb:
        best, bt = -1, F32(np.inf)
        for j in range(k):
            if par[b, j] < 0 or not okG[b, j]:
                continue
            t2 = F32(tt[par[b, j]] + TG[b, j])
            if t2 < bt:
                best, bt = j, t2
        if best >= 0:
            new.append((b, best, bt))
    gst = np.asarray(tree_gpu["states"], F32)
    n_new = int(tree_gpu["n"]) - n_old
    out["nodes_added"] = n_new
    if n_new != len(new):
        out["attach_mismatches"] = abs(n_new - len(new)) + 1
    else:
        bad = 0
        bestJ, bestI = -np.inf, -1
        for r, (b, j, t2) in enumerate(new):
            i = n_old + r
            p = int(par[b, j])
            nu = max(float(nu0[p]), float(rvG[b, j]))
            same = (np.array_equal(gst[i], states[b]) and int(tree_gpu["parent"][i]) == p
                    and F32(tree_gpu["t"][i]) == t2 and F32(tree_gpu["nu"][i]) == F32(nu))
            if same and b < n_goal:
                Jr = orc.objective(pr, float(t2), float(cand["v_rel"][b]), nu)
                same = abs(float(tree_gpu["J"][i]) - Jr) <= 1e-4 * max(1.0, abs(Jr))
                if float(tree_gpu["J"][i]) > bestJ:
                    bestJ, bestI = float(tree_gpu["J"][i]), i
            bad += 0 if same else 1
        out["attach_mismatches"] = bad
        if inc_gpu is not None:
            before = -np.inf if inc_before is None else inc_before.get("J", -np.inf)
            want = bestI if bestI >= 0 and bestJ > before else (
                -1 if inc_before is None else inc_before.get("id", -1))
            out["incumbent_ok"] = bool(int(inc_gpu["incumbent"]) == want)
    return out


def rho_matches(orc, arm, s0, s1, T, S, rho_gpu, rho_ref, delta=4e-6):
    """Per-edge check of (rho_tau, rho_P, rho_v) at duration T[e].

    rho_tau and rho_P compare within RHO_REL (relative, absolute below 1).
    rho_v divides by the sqrt taper, which is ill-conditioned next to a joint
    limit (a one-ulp position change moves it by percents): the GPU value
    must lie between the oracle's rho_v with the joint boxes widened and
    narrowed by `delta` radians, widened by RHO_REL.  Returns the indices of
    edges that fail."""
    rho_gpu = np.asarray(rho_gpu, np.float64)
    bad = []
    tp_ok = np.all(np.abs(rho_gpu[:, :2] - rho_ref[:, :2]) <= RHO_REL * np.maximum(1, np.abs(rho_ref[:, :2])), axis=1)
    lo = orc.rho_batch(arm_limits_moved(arm, delta), s0, s1, T, S)[:, 2]
    hi = orc.rho_batch(arm_limits_moved(arm, -delta), s0, s1, T, S)[:, 2]
    v = rho_gpu[:, 2]
    v_ok = (v >= lo * (1 - RHO_REL) - 1e-12) & ((v <= hi * (1 + RHO_REL) + 1e-12) | np.isinf(hi))
    for e in np.nonzero(~(tp_ok & v_ok))[0]:
        bad.append(int(e))
    return bad
