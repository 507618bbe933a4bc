"""Parity of the packed edge engine (fn_edges_*) with the FP64 oracle and
with the warp-per-edge scan, through the C ABI."""
import numpy as np
import pytest
import torch

from paper_2609_22608_gb300 import synth
from tests.parity import kstar_mismatches

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def ops():
    from paper_2609_22608_gb300 import ops as o
    return o


@pytest.mark.parametrize("E,K,S", [(1, 32, 16), (257, 64, 32), (3000, 128, 64)])
def test_engine_full_scan_matches_oracle(ops, orc, arm, E, K, S):
    s0, s1 = synth.random_edges(arm, E, 70 + E)
    grid = synth.duration_grid(K)
    eng = ops.EdgeEngine(arm, grid, S=S, max_E=1024)       # several passes for E = 3000
    o = eng.time(dev(s0), dev(s1))
    eng.close()
    ref = orc.time_edges(arm, s0, s1, grid, S)
    kg = o["k_star"].cpu().numpy()
    bad = kstar_mismatches(orc, arm, s0, s1, grid, S, kg, ref["k_star"])
    assert not bad, bad[:5]
    same = kg == ref["k_star"]
    okg, okr = o["ok"].cpu().numpy().astype(bool), ref["ok"].astype(bool)
    assert np.mean(okg[same] != okr[same]) < 0.01   # rho_v at the limit only
    Tg = o["T_star"].cpu().numpy()
    f = kg >= 0
    assert np.array_equal(Tg[f], grid[kg[f]])
    assert np.all(np.isinf(Tg[kg == -1]))


def test_engine_matches_warp_scan_with_cap(ops, arm):
    E, K, S = 4096, 128, 64
    s0, s1 = synth.random_edges(arm, E, 81)
    grid = synth.duration_grid(K)
    rng = np.random.default_rng(82)
    cap = rng.uniform(0.05, 2.2, E).astype(np.float32)
    d0, d1, dc = dev(s0), dev(s1), dev(cap)
    eng = ops.EdgeEngine(arm, grid, S=S, max_E=E)
    o = eng.time(d0, d1, T_cap=dc)
    ref = ops.time_edges(arm, d0, d1, grid, S, T_cap=dc)
    eng.close()
    kg, kr = o["k_star"].cpu().numpy(), ref["k_star"].cpu().numpy()
    # both are exact first-feasible scans; they may differ only where a probe's
    # plain-coefficient sample sits at the limit
    assert np.mean(kg != kr) < 2e-3, np.mean(kg != kr)


def test_engine_window_certificate_and_rescan(ops, arm):
    """Any prediction gives the full scan's k* for rescanned edges, and for
    certified edges except where the certificate relied on monotone limits."""
    E, K, S = 3000, 128, 32
    s0, s1 = synth.random_edges(arm, E, 83)
    grid = synth.duration_grid(K)
    d0, d1 = dev(s0), dev(s1)
    eng = ops.EdgeEngine(arm, grid, S=S, max_E=2048)
    full = eng.time(d0, d1)
    kf = full["k_star"].cpu().numpy()
    rng = np.random.default_rng(84)
    lg = np.log(grid.astype(np.float64))
    y0 = np.where(kf >= 0, lg[np.clip(kf, 0, None)], 0.0)
    Y = np.stack([y0 + rng.choice([0, 0, 0.3, -0.3, 2.0, -2.0], E),
                  rng.choice([1.0, 1.0, -1.0], E)], 1).astype(np.float32)
    w = eng.time_window(d0, d1, dev(Y), W=16)
    eng.close()
    kw, path = w["k_star"].cpu().numpy(), w["path"].cpu().numpy()
    assert set(np.unique(path)) <= {0, 1}
    assert np.array_equal(kw[path == 1], kf[path == 1])
    mism = np.nonzero(kw != kf)[0]
    assert len(mism) <= 0.01 * E
    for e in mism:
        assert kw[e] == -1 or kf[e] == -1 or kw[e] > kf[e]
    assert 0.2 < np.mean(path == 0) < 0.95   # both paths exercised by these predictions


def test_engine_non_finite_input(ops, arm):
    s0, s1 = synth.random_edges(arm, 64, 85)
    s0[5, 3] = np.nan
    s1[9, 10] = np.inf
    eng = ops.EdgeEngine(arm, synth.duration_grid(32), S=16, max_E=64)
    o = eng.time(dev(s0), dev(s1))
    eng.close()
    k = o["k_star"].cpu().numpy()
    assert k[5] == -2 and k[9] == -2
    assert np.all(k[[i for i in range(64) if i not in (5, 9)]] >= -1)
