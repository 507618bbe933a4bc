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


def near_margin(orc, arm, s0, s1, grid, S):
    """Is any admissible grid duration of this edge within the 1e-4 margin?"""
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
        explained = False
        for j, p in enumerate(par):
            if p < 0:
                continue
            s0 = ref_tree.states[p] if p < n_old else None
            if s0 is None:
                continue
            if near_margin(orc, arm, s0, cand[b], grid, S):
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
