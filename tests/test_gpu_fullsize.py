"""The headline workload at full size, in the configuration the benchmark
times: one planning iteration (tree 4096, batch 2048 of which half goal
candidates, k = 8, K = 128, S = 64) captured as a CUDA graph and replayed,
with the free queries' parent search beside the goal chart's IK.  Checked on
sampled outputs the oracle computes one by one:
  * free candidates: the oracle's uniform sampler on the same Philox
    counters;
  * goal candidates: the oracle's chart decoding (acceptance, T_req, q);
  * parents of the sampled queries: the oracle's brute-force scan;
  * the round on the sampled candidates (the GPU's own states): the oracle's
    Algorithm 1 round attaches them to the same parent at the same time,
    except where an edge sits within the 1e-4 limit margin.
"""
import numpy as np
import pytest
import torch

import bench
import oracle.plan as OP
from tests.parity import compare_round, knn_mismatches

pytestmark = pytest.mark.gpu


def test_fullsize_iteration_sampled(orc):
    from paper_2609_22608_gb300 import planner as P
    w = bench.make_workload(0)
    arm, pr = w["arm"], w["pr"]
    N, B, k, K, S = bench.N_TREE, bench.B_CAND, bench.K_PAR, bench.K_GRID, bench.S_COLL
    G = B // 2
    seed, it = 1000 + w["seed"], 7
    pl = P.Planner(arm, P=1, n_cap=N + 2 * B, b_max=B, k=k, K=K, S=S)
    prob = P.problem_struct(pr, B, G, root=w["root"], seed=seed)
    stream = torch.cuda.Stream()
    pl.reset([prob], stream=stream)
    pl.load_tree(0, w["tree"], w["t_node"], w["parent"], stream=stream)
    pl.capture(0, stream=stream)
    out = pl.replay([prob], it, stream=stream)[0]
    stream.synchronize()
    cand = pl.get_candidates(0, B)
    nn = pl.get_parents(0, B)
    gtree = pl.get_tree(0)
    pl.close()
    rng = np.random.default_rng(11)

    # free candidates
    fs = np.sort(rng.choice(np.arange(G, B), 64, replace=False))
    for b in fs:
        ref = orc.sample_uniform(arm, seed, it, 0, int(b), 1, 0.5)[0]
        assert np.abs(cand["states"][b, :7] - ref[:7]).max() < 1e-5

    # goal candidates
    gs = np.sort(rng.choice(G, 256, replace=False))
    agree = 0
    for b in gs:
        st, Tq, vr, valid = orc.sample_goals(arm, pr, seed, it, 0, int(b), 1)
        gv = cand["valid"][b] == 1
        agree += gv == (valid[0] == 1)
        if gv and valid[0] == 1:
            assert cand["T_req"][b] == pytest.approx(Tq[0], rel=1e-6)
            assert np.abs(cand["states"][b, :7] - st[0, :7]).max() < 2e-3
    assert agree >= 0.98 * len(gs)

    # parents: the sampled free queries and every decoded goal
    vg = np.flatnonzero(cand["valid"][:G] == 1)
    qs = np.concatenate([fs, vg])
    ri, rd = orc.knn(w["tree"], cand["states"][qs].astype(np.float32), k - 1, 0.1)
    d_gpu = np.zeros_like(rd)
    for a, b in enumerate(qs):
        x = cand["states"][b].astype(np.float64)
        for j in range(k - 1):
            y = w["tree"][nn[b, j]].astype(np.float64)
            d_gpu[a, j] = np.sum((x[:7] - y[:7]) ** 2) + 0.1 * np.sum((x[8:15] - y[8:15]) ** 2)
    bad = knn_mismatches(nn[qs], d_gpu, ri, rd)
    assert not bad, bad[:5]

    # the round on the sampled candidates (goals first, as the planner orders them)
    sub = np.concatenate([vg, fs])
    case = dict(cand=cand["states"][sub].astype(np.float32), n_goal=len(vg),
                T_req=cand["T_req"][vg].astype(np.float32),
                v_rel=cand["v_rel"][vg].astype(np.float32))
    inc = dict(id=-1, J=-np.inf, t_best=float(np.float32(pr["t_fall"])))
    rtree, _, det = OP.plan_round(arm, pr, OP.Tree(w["tree"], w["t_node"], w["parent"]),
                                  case["cand"], case["n_goal"], case["T_req"], case["v_rel"],
                                  inc, k, w["grid"], S)
    bad = compare_round(orc, arm, case, gtree, rtree, det, N, w["grid"], S=S)
    assert not bad, f"sampled candidates attached differently without a near-margin edge: {bad[:5]}"
    assert gtree["n"] - N == out["n_added"]
