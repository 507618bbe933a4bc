"""Parity of the CUDA edge timing (fn_time_edges, fn_rnea_dump) with the FP64
oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from paper_2609_22608_gb300 import synth
from tests.parity import kstar_mismatches, rho_matches, torque_ok

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ops():
    from paper_2609_22608_gb300 import ops as o
    return o


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("E,S", [(256, 32), (97, 64), (1, 2), (33, 255)])
def test_torque_parity(ops, orc, arm, E, S):
    s0, s1 = synth.random_edges(arm, E, 21 + E)
    rng = np.random.default_rng(E)
    T = rng.uniform(0.05, 2.0, E).astype(np.float32)
    tau = ops.rnea_dump(arm, dev(s0), dev(s1), dev(T), S).cpu().numpy()
    ref = orc.torque_dump(arm, s0, s1, T, S)
    ok, rel = torque_ok(tau, ref)
    assert ok.all(), f"worst normalised torque error {rel.max():.3e}"


def _check_full(ops, orc, arm, s0, s1, grid, S, T_cap=None):
    cap_d = None if T_cap is None else dev(T_cap)
    r = ops.time_edges(arm, dev(s0), dev(s1), grid, S, T_cap=cap_d)
    k = r["k_star"].cpu().numpy()
    ref = orc.time_edges(arm, s0, s1, grid, S, T_cap=T_cap)
    bad = kstar_mismatches(orc, arm, s0, s1, grid, S, k, ref["k_star"], T_cap)
    assert not bad, f"{len(bad)} k* mismatches beyond the 1e-4 margin, e.g. {bad[:5]}"
    same = (k == ref["k_star"]) & (k >= 0)
    Ts = r["T_star"].cpu().numpy()
    assert np.array_equal(Ts[same], grid[k[same]])
    rho = r["rho3"].cpu().numpy()
    idx = np.nonzero(same)[0]
    bad = rho_matches(orc, arm, s0[idx], s1[idx], grid[k[idx]].astype(np.float64), S, rho[idx],
                      ref["rho3"][idx])
    assert not bad, [(int(idx[b]), rho[idx[b]].tolist(), ref["rho3"][idx[b]].tolist()) for b in bad[:3]]
    none = k == -1
    assert np.all(np.isinf(Ts[none]))
    okg = r["ok"].cpu().numpy()
    # ok agrees wherever k* agrees and rho_v is not within rounding of 1
    clear = same & (np.abs(ref["rho3"][:, 2] - 1) > 1e-3)
    assert np.array_equal(okg[clear], ref["ok"][clear])
    return k, ref


def test_full_scan_small_config(ops, orc, arm):
    """256 random edges, 64 log-spaced durations in [0.05, 2] s, 32 samples."""
    s0, s1 = synth.random_edges(arm, 256, 0)
    k, ref = _check_full(ops, orc, arm, s0, s1, synth.duration_grid(64), 32)
    assert (k == ref["k_star"]).mean() > 0.98


@pytest.mark.parametrize("E,K,S", [(300, 128, 64), (33, 7, 5), (1, 1, 2), (65, 256, 33)])
def test_full_scan_shapes(ops, orc, arm, E, K, S):
    s0, s1 = synth.random_edges(arm, E, 100 + E + K)
    _check_full(ops, orc, arm, s0, s1, synth.duration_grid(K), S)


def test_full_scan_with_cap(ops, orc, arm):
    s0, s1 = synth.random_edges(arm, 200, 5)
    rng = np.random.default_rng(5)
    cap = rng.uniform(0.0, 2.5, 200).astype(np.float32)
    cap[:5] = [0.0, 0.05, 2.0, np.inf, -1.0]
    _check_full(ops, orc, arm, s0, s1, synth.duration_grid(128), 64, T_cap=cap)


def test_closed_form_min_time_on_gpu(ops, arm):
    """One-link rest-to-rest edges: k* = first T_k >= sqrt(6 I |dq| / tau_max)."""
    from tests.test_oracle_edges import _itot, one_link_arm
    import math
    a = one_link_arm(arm)
    I = _itot(a)
    grid = synth.duration_grid(64)
    rng = np.random.default_rng(77)
    E = 200
    s0 = np.zeros((E, 16), np.float32)
    s1 = np.zeros((E, 16), np.float32)
    s1[:, 0] = rng.uniform(-3, 3, E)
    r = ops.time_edges(a, dev(s0), dev(s1), grid, 32)
    k = r["k_star"].cpu().numpy()
    for e in range(E):
        Tstar = math.sqrt(6 * I * abs(float(s1[e, 0])) / float(a["tau_max"][0]))
        ks = np.nonzero(grid.astype(np.float64) >= Tstar)[0]
        expect = int(ks[0]) if len(ks) else -1
        near = expect > 0 and abs(float(grid[expect]) / Tstar - 1) < 1e-5
        near |= expect >= 1 and abs(float(grid[expect - 1]) / Tstar - 1) < 1e-5
        if not near:
            assert k[e] == expect


def test_fixed_mode(ops, orc, arm):
    s0, s1 = synth.random_edges(arm, 260, 9)
    rng = np.random.default_rng(9)
    T = rng.uniform(0.05, 2.0, 260).astype(np.float32)
    T[:4] = [0.0, -0.5, np.nan, np.inf]
    _check_fixed(ops, orc, arm, s0, s1, T)


def _check_fixed(ops, orc, arm, s0, s1, T):
    r = ops.time_edges(arm, dev(s0), dev(s1), None, 64, mode=ops.FN_MODE_FIXED, T_fixed=dev(T))
    ref = orc.time_edges(arm, s0, s1, synth.duration_grid(2), 64, mode=1, T_fixed=T)
    k = r["k_star"].cpu().numpy()
    assert list(k[:4]) == [-2, -2, -2, -2]
    rho = r["rho3"].cpu().numpy()
    valid = ref["k_star"] != -2
    idx = np.nonzero(valid)[0]
    bad = rho_matches(orc, arm, s0[idx], s1[idx], T[idx].astype(np.float64), 64, rho[idx],
                      ref["rho3"][idx])
    assert not bad, [(int(idx[b]), rho[idx[b]].tolist(), ref["rho3"][idx[b]].tolist()) for b in bad[:3]]
    m = np.maximum(ref["rho3"][:, 0], ref["rho3"][:, 1])
    clear = valid & (np.abs(m - 1) > 1e-4) & (np.abs(ref["rho3"][:, 2] - 1) > 1e-3)
    assert np.array_equal(k[clear], ref["k_star"][clear])
    assert np.array_equal(r["ok"].cpu().numpy()[clear], ref["ok"][clear])


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_every_schedule_variant(ops, orc, arm, variant):
    """Each compiled schedule of fn_time_edges, pinned for the shape (0-2: one
    sample per lane at three register budgets; 3: two samples per lane with
    the recursion's records in tensor memory): FULL mode with a cap and FIXED
    mode against the oracle."""
    E, K, S = 300, 128, 64
    s0, s1 = synth.random_edges(arm, E, 300 + variant)
    rng = np.random.default_rng(300 + variant)
    cap = rng.uniform(0.3, 2.5, E).astype(np.float32)
    T = rng.uniform(0.05, 2.0, E).astype(np.float32)
    T[:4] = [0.0, -0.5, np.nan, np.inf]
    try:
        ops.set_time_edges_variant(ops.FN_MODE_FULL, E, K, S, variant)
        ops.set_time_edges_variant(ops.FN_MODE_FIXED, E, 1, S, variant)
        _check_full(ops, orc, arm, s0, s1, synth.duration_grid(K), S, T_cap=cap)
        _check_fixed(ops, orc, arm, s0, s1, T)
    finally:
        ops.set_time_edges_variant(ops.FN_MODE_FULL, E, K, S, 3)
        ops.set_time_edges_variant(ops.FN_MODE_FIXED, E, 1, S, 3)


def test_scalar_variants_identical(ops, arm):
    """Variants 0-2 differ only in their register budget: bit-identical outputs."""
    E, K, S = 500, 128, 64
    s0, s1 = synth.random_edges(arm, E, 77)
    grid = synth.duration_grid(K)
    outs = []
    try:
        for v in (0, 1, 2):
            ops.set_time_edges_variant(ops.FN_MODE_FULL, E, K, S, v)
            r = ops.time_edges(arm, dev(s0), dev(s1), grid, S)
            outs.append({k: t.cpu().numpy() for k, t in r.items()})
    finally:
        ops.set_time_edges_variant(ops.FN_MODE_FULL, E, K, S, 3)
    for o in outs[1:]:
        for k in o:
            assert np.array_equal(o[k], outs[0][k], equal_nan=True), k


def test_autotune_time_edges(ops, orc, arm):
    """The tuner times the four schedules and keeps one; later calls of the
    shape use it, and its results match the oracle."""
    E, K, S = 400, 128, 64
    s0, s1 = synth.random_edges(arm, E, 91)
    grid = synth.duration_grid(K)
    try:
        chosen, ms = ops.autotune_time_edges(arm, dev(s0), dev(s1), grid, S, reps=1)
        assert 0 <= chosen < 4 and len(ms) == 4 and all(m > 0 for m in ms)
        assert ms[chosen] == min(ms)
        _check_full(ops, orc, arm, s0, s1, grid, S)
    finally:
        ops.set_time_edges_variant(ops.FN_MODE_FULL, E, K, S, 3)
    for bad in ((ops.FN_MODE_FULL, E, K, S, 4), (ops.FN_MODE_FULL, E, K, S, -1),
                (7, E, K, S, 0), (ops.FN_MODE_FULL, 0, K, S, 0), (ops.FN_MODE_FULL, E, 0, S, 0)):
        with pytest.raises(Exception):
            ops.set_time_edges_variant(*bad)


def test_invalid_edges_and_arguments(ops, orc, arm):
    s0, s1 = synth.random_edges(arm, 8, 2)
    s0[1, 3] = np.nan
    s1[2, 9] = np.inf
    r = ops.time_edges(arm, dev(s0), dev(s1), synth.duration_grid(16), 8)
    k = r["k_star"].cpu().numpy()
    assert k[1] == -2 and k[2] == -2 and r["ok"].cpu().numpy()[1] == 0
    from paper_2609_22608_gb300._lib import FnError
    with pytest.raises(FnError):
        ops.time_edges(arm, dev(s0), dev(s1), np.array([0.5, 0.4], np.float32), 8)  # not ascending
    with pytest.raises(FnError):
        ops.time_edges(arm, dev(s0), dev(s1), synth.duration_grid(16), 1)  # S < 2
    bad_arm = dict(arm); bad_arm["dof"] = 6
    with pytest.raises(FnError):
        ops.time_edges(bad_arm, dev(s0), dev(s1), synth.duration_grid(16), 8)
    # E = 0 is a no-op
    z = torch.empty(0, 16, device="cuda")
    out = ops.time_edges(arm, z, z, synth.duration_grid(16), 8)
    assert out["k_star"].numel() == 0


def test_full_size_sampled(ops, orc, arm):
    """The bench's edge workload size (16384 edges, K = 128, S = 64): every
    output is checked on a seeded sample of 256 edges and by invariants that
    hold at any size (T* on the grid, rho <= 1 at k*)."""
    E = 16384
    s0, s1 = synth.random_edges(arm, E, 123)
    grid = synth.duration_grid(128)
    r = ops.time_edges(arm, dev(s0), dev(s1), grid, 64)
    k = r["k_star"].cpu().numpy()
    Ts = r["T_star"].cpu().numpy()
    rho = r["rho3"].cpu().numpy()
    f = k >= 0
    assert np.array_equal(Ts[f], grid[k[f]])
    assert np.all(rho[f, :2] <= 1.0)
    sel = np.random.default_rng(0).choice(E, 256, replace=False)
    ref = orc.time_edges(arm, s0[sel], s1[sel], grid, 64)
    bad = kstar_mismatches(orc, arm, s0[sel], s1[sel], grid, 64, k[sel], ref["k_star"])
    assert not bad
