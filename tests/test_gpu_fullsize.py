"""The headline workload at full size, in the configuration the benchmark
times: one planning iteration (tree 4096, batch 2048 of which half goal
draws, k = 8, K = 128, S = 64) captured as a CUDA graph and replayed, with
the free queries' parent search beside the goal chart's IK.  Checked in full
against the oracle:
  * every free candidate: the oracle's uniform sampler on the same Philox
    counters;
  * every goal draw: the oracle's chart decoding (acceptance except at a
    tolerance edge, T_req, q);
  * every parent list, every (candidate, parent) edge, the attach, the
    scores and the incumbent: verify_iteration (tests/parity.py).
"""
import numpy as np
import pytest
import torch

import bench
from tests.parity import verify_iteration

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [0, 1])
def test_fullsize_iteration_every_edge(orc, seed):
    from paper_2609_22608_gb300 import planner as P
    w = bench.make_workload(seed)
    arm, pr = w["arm"], w["pr"]
    N, B, k, K, S = bench.N_TREE, bench.B_CAND, bench.K_PAR, bench.K_GRID, bench.S_COLL
    G = B // 2
    rseed, it = 1000 + w["seed"], 7
    pl = P.Planner(arm, P=1, n_cap=N + 2 * B, b_max=B, k=k, K=K, S=S)
    prob = P.problem_struct(pr, B, G, root=w["root"], seed=rseed)
    stream = torch.cuda.Stream()
    pl.reset([prob], stream=stream)
    pl.load_tree(0, w["tree"], w["t_node"], w["parent"], stream=stream)
    pl.capture(0, stream=stream)
    for rep in range(2):            # the replay is repeatable on a restored tree
        pl.reset([prob], stream=stream)
        pl.load_tree(0, w["tree"], w["t_node"], w["parent"], stream=stream)
        if rep == 1:
            stream.synchronize()
            pl.work_counts(reset=True)
        out = pl.replay([prob], it, stream=stream)[0]
    stream.synchronize()
    rb = bench.readback(pl, B)
    work = pl.work_counts()
    pl.close()
    cand = rb["cand"]

    # every free candidate
    ref = orc.sample_uniform(arm, rseed, it, 0, G, B - G, 0.5)
    assert np.abs(cand["states"][G:, :7] - ref[:, :7]).max() < 1e-5
    assert np.abs(cand["states"][G:, 8:15] - ref[:, 8:15]).max() < 1e-5

    # every goal draw: acceptance agrees except where a start's residual sits
    # at the IK tolerance (FP32 vs FP64 iterates), well under 1 % of draws
    st, Tq, vr, valid, why = orc.sample_goals(arm, pr, rseed, it, 0, 0, G, reasons=True)
    gv = cand["valid"][:G] == 1
    assert np.mean(gv != (valid == 1)) <= 0.01
    both = gv & (valid == 1)
    assert both.sum() >= 0.08 * G, f"goal yield {both.mean():.3f}"
    assert np.allclose(cand["T_req"][:G][both], Tq[both], rtol=1e-6)
    assert np.abs(cand["states"][:G][both, :7] - st[both, :7]).max() < 2e-3
    # the device's per-reason counts follow the same draws
    assert work["goal_defined"] == gv.sum()
    assert work["goal_speed"] == np.sum(why == 1)

    # every edge, the attach and the incumbent
    tree = dict(states=w["tree"], t=w["t_node"], parent=w["parent"])
    r = verify_iteration(orc, arm, pr, tree, float(np.float32(pr["t_fall"])), cand, G, rb["nn"],
                         rb["edges"], rb["tree"], w["grid"], S, k, inc_gpu=out)
    assert r["parent_mismatches"] == 0, r
    assert r["edge_mismatches"] == 0, r
    assert r["attach_mismatches"] == 0, r
    assert r["incumbent_ok"], r
    assert r["edges_formed"] == int((cand["valid"] == 1).sum()) * k
    assert rb["tree"]["n"] - N == out["n_added"]
