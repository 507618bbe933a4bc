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
