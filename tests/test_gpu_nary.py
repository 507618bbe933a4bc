"""Parity of the CUDA N-ary refinement (fn_time_edges_nary) with the FP64
oracle, through the C ABI.

Rule: the grid index follows the k* margin rule.  Where the two k* agree and
every duration the oracle checked has |max(rho_tau, rho_P) - 1| > 1e-4, both
sides check the same single-precision points and take the same decisions,
so T_star, T_lo and the round count must be bit-identical.  This holds for
most edges after one round; from the second round on, the points lie within
about 3e-5 T of T*, where max(rho_tau, rho_P) is within the margin of 1 and
either decision is correct.  So for every edge the GPU's bracket must be
valid in FP64 within the margin (its upper end passes the check, its lower
end fails it or is 0), lie in the grid cell and be no wider than eps (unless
the round cap ended it); and on 99 % of edges |T_gpu - T_ref| stays within
both bracket widths plus 1e-4 T, the spread of durations whose ratio lies
within the margin when the ratios fall like 1/T^2.
"""
import math

import numpy as np
import pytest
import torch

from paper_2609_22608_gb300 import synth
from tests.parity import RHO_MARGIN, kstar_mismatches, rho_matches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ops():
    from paper_2609_22608_gb300 import ops as o
    return o


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _check(ops, orc, arm, s0, s1, grid, S, eps, max_rounds=8, T_cap=None, sample=None):
    cap_d = None if T_cap is None else dev(T_cap)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    r = ops.time_edges_nary(arm, dev(s0), dev(s1), grid, S, eps, max_rounds, T_cap=cap_d,
                            sample_count=cnt)
    out = {k: v.cpu().numpy() for k, v in r.items()}
    idx = np.arange(s0.shape[0]) if sample is None else sample
    cap = None if T_cap is None else T_cap[idx]
    a, b = s0[idx], s1[idx]
    ref = orc.time_edges_nary(arm, a, b, grid, S, eps, max_rounds, T_cap=cap)
    k = out["k_star"][idx]
    bad = kstar_mismatches(orc, arm, a, b, grid, S, k, ref["k_star"], cap)
    assert not bad, f"{len(bad)} k* mismatches beyond the margin, e.g. {bad[:5]}"
    Ts, Tl, rounds = out["T_star"][idx], out["T_lo"][idx], out["rounds"][idx]
    same = (k == ref["k_star"]) & (k >= 0)
    exact = same & (ref["margin"] > RHO_MARGIN)
    assert np.array_equal(Ts[exact], ref["T_star"][exact])
    assert np.array_equal(Tl[exact], ref["T_lo"][exact])
    assert np.array_equal(rounds[exact], ref["rounds"][exact])
    ie = np.flatnonzero(exact)
    rho = out["rho3"][idx]
    badr = rho_matches(orc, arm, a[ie], b[ie], Ts[ie].astype(np.float64), S, rho[ie], ref["rho3"][ie])
    assert not badr, [(int(ie[j]), rho[ie[j]].tolist(), ref["rho3"][ie[j]].tolist()) for j in badr[:3]]
    clear_v = np.abs(ref["rho3"][ie, 2] - 1) > RHO_MARGIN
    assert np.array_equal(out["ok"][idx][ie][clear_v], ref["ok"][ie][clear_v])
    # every edge: the GPU's bracket must be a valid one
    near = np.flatnonzero(same)
    if len(near):
        hi = Ts[near].astype(np.float64)
        r_hi = orc.rho_batch(arm, a[near], b[near], hi, S)
        assert np.all(np.maximum(r_hi[:, 0], r_hi[:, 1]) <= 1 + RHO_MARGIN)
        lo = Tl[near].astype(np.float64)
        pos = lo > 0
        if pos.any():
            r_lo = orc.rho_batch(arm, a[near][pos], b[near][pos], lo[pos], S)
            assert np.all(np.maximum(r_lo[:, 0], r_lo[:, 1]) > 1 - RHO_MARGIN)
        kk = k[near]
        cell_lo = np.where(kk > 0, grid[np.maximum(kk - 1, 0)], 0.0)
        assert np.all(lo >= cell_lo) and np.all(hi <= grid[kk])
        capped = rounds[near] >= max_rounds
        assert np.all((hi - lo <= eps) | capped)
        w_ref = ref["T_star"][near].astype(np.float64) - ref["T_lo"][near]
        tol = (hi - lo) + w_ref + RHO_MARGIN * hi
        close = np.abs(hi - ref["T_star"][near]) <= tol
        assert close.mean() >= 0.99, np.flatnonzero(~close)[:5]
    none = k == -1
    assert np.all(np.isinf(Ts[none])) and np.all(np.isnan(Tl[none]))
    assert int(cnt.item()) > 0 or not (k >= 0).any()
    return dict(k=k, ref=ref, exact=exact, same=same, out=out)


def test_nary_small_config(ops, orc, arm):
    """256 random edges, 64 log-spaced durations in [0.05, 2] s, 32 samples;
    eps = 5e-3 takes one round, whose decisions are clear of the margin and
    results bit-identical on ~90 % of the edges; eps = 1e-4 takes two."""
    s0, s1 = synth.random_edges(arm, 256, 0)
    grid = synth.duration_grid(64)
    res = _check(ops, orc, arm, s0, s1, grid, 32, 5e-3)
    assert res["same"].sum() >= 150
    assert res["exact"].sum() >= 0.8 * res["same"].sum()
    res = _check(ops, orc, arm, s0, s1, grid, 32, 1e-4)
    assert np.all(res["out"]["rounds"][res["same"]] >= 1)


@pytest.mark.parametrize("E,K,S,eps", [(300, 128, 64, 1e-4), (33, 7, 5, 1e-3), (1, 1, 2, 1e-2),
                                       (65, 256, 33, 1e-6), (97, 128, 64, 5e-2)])
def test_nary_shapes(ops, orc, arm, E, K, S, eps):
    s0, s1 = synth.random_edges(arm, E, 200 + E + K)
    _check(ops, orc, arm, s0, s1, synth.duration_grid(K), S, eps)


def test_nary_with_cap_and_round_cap(ops, orc, arm):
    s0, s1 = synth.random_edges(arm, 200, 6)
    rng = np.random.default_rng(6)
    cap = rng.uniform(0.0, 2.5, 200).astype(np.float32)
    cap[:5] = [0.0, 0.05, 2.0, np.inf, -1.0]
    grid = synth.duration_grid(128)
    _check(ops, orc, arm, s0, s1, grid, 64, 1e-5, T_cap=cap)
    _check(ops, orc, arm, s0, s1, grid, 64, 1e-7, max_rounds=1, T_cap=cap)


def test_zero_rounds_is_the_grid_scan(ops, arm):
    s0, s1 = synth.random_edges(arm, 128, 8)
    grid = synth.duration_grid(128)
    g = ops.time_edges(arm, dev(s0), dev(s1), grid, 64)
    n = ops.time_edges_nary(arm, dev(s0), dev(s1), grid, 64, 1e-4, max_rounds=0)
    for key in ("k_star", "T_star", "ok"):
        assert torch.equal(g[key], n[key]), key
    # same decisions; the ratios come from another kernel's code, whose
    # contractions may differ in the last bit
    assert torch.allclose(torch.nan_to_num(g["rho3"], 7.0), torch.nan_to_num(n["rho3"], 7.0),
                          rtol=1e-6, atol=0)
    assert int(n["rounds"].max()) == 0


def test_closed_form_bracket_on_gpu(ops, arm):
    """One link, rest to rest: the bracket holds sqrt(6 I |dq| / tau_max)."""
    from tests.test_oracle_edges import _itot, one_link_arm
    a = one_link_arm(arm)
    I = _itot(a)
    grid = synth.duration_grid(64)
    rng = np.random.default_rng(78)
    E = 200
    s0 = np.zeros((E, 16), np.float32)
    s1 = np.zeros((E, 16), np.float32)
    s0[:, 0] = 0.3
    s1[:, 0] = 0.3 + rng.uniform(-3, 3, E).astype(np.float32)
    eps = 1e-5
    r = ops.time_edges_nary(a, dev(s0), dev(s1), grid, 32, eps)
    lo, hi = r["T_lo"].cpu().numpy(), r["T_star"].cpu().numpy()
    k = r["k_star"].cpu().numpy()
    n_in = 0
    for e in range(E):
        dq = float(s1[e, 0]) - float(s0[e, 0])
        Tstar = math.sqrt(6 * I * abs(dq) / float(a["tau_max"][0]))
        if k[e] < 0:
            assert Tstar > float(grid[-1]) * (1 - 1e-5)
            continue
        assert hi[e] - lo[e] <= eps
        # single-precision torques place the crossing within ~1e-6 of T*
        # (relative), more than the last bracket's width (~5e-7 s)
        tol = 2e-6 * Tstar
        assert lo[e] - tol < Tstar <= hi[e] + tol, (e, lo[e], hi[e], Tstar)
        n_in += 1
    assert n_in >= 150


def test_invalid_inputs(ops, arm):
    s0, s1 = synth.random_edges(arm, 40, 9)
    s0[3, 2] = np.nan
    s1[7, 9] = np.inf
    grid = synth.duration_grid(64)
    r = ops.time_edges_nary(arm, dev(s0), dev(s1), grid, 16, 1e-4)
    k = r["k_star"].cpu().numpy()
    assert k[3] == -2 and k[7] == -2
    assert np.isnan(r["T_star"].cpu().numpy()[[3, 7]]).all()
    empty = torch.empty(0, 16, device="cuda")
    ops.time_edges_nary(arm, empty, empty, grid, 16, 1e-4)
    from paper_2609_22608_gb300._lib import FnError
    for eps, rounds in ((0.0, 8), (float("nan"), 8), (1e-4, -1), (1e-4, 17)):
        with pytest.raises(FnError):
            ops.time_edges_nary(arm, dev(s0), dev(s1), grid, 16, eps, rounds)


def test_nary_full_size_sampled(ops, orc, arm):
    """65 536 random edges, K = 128, S = 64 (the surrogate workload's size),
    checked on 192 sampled edges."""
    s0, s1 = synth.random_edges(arm, 65536, 12)
    sample = np.random.default_rng(12).choice(65536, 192, replace=False)
    res = _check(ops, orc, arm, s0, s1, synth.duration_grid(128), 64, 1e-4, sample=sample)
    assert res["same"].sum() >= 60
