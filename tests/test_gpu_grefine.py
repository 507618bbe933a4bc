"""Gradient refinement of the incumbent rendezvous (FN_PLAN_GREFINE) against
the FP64 oracle of the same reading (oracle/refine.py).  A round whose goal
edges succeed (each decoded goal has an approach node 0.1 s before it on its
own velocity; the goal candidates come with their chart parameters) runs
with and without the refinement:
  * without it, the tree and the incumbent are the plain round's;
  * with it, a refined node is appended beside the incumbent (same parent)
    and becomes the incumbent;
  * the refined node passes the oracle's exact check at its duration, its J
    equals the oracle's objective for its chart parameters, and it is better
    than the original by at least half of what the oracle's own refinement
    gains from the same start.
"""
import numpy as np
import pytest

import oracle.refine as R
from paper_2609_22608_gb300 import synth

pytestmark = pytest.mark.gpu
F32 = np.float32
K_GRID, S_COLL = 32, 16


@pytest.fixture(scope="module")
def P():
    from paper_2609_22608_gb300 import planner as pl
    return pl


def _case(arm, orc, seed):
    toss = synth.random_toss(arm, seed)
    root = synth.random_states(arm, 1, 5000 + seed)[0]
    pr = synth.make_problem(toss, root=root)
    states, parent, t = synth.random_tree(arm, 120, seed, root=root, t_max=pr["t_fall"])
    st, Tq, vr, valid, Z = orc.sample_goals_density(arm, pr, dict(C=0, w_u=0.25), 300 + seed, 0, 0,
                                                    0, 512)
    gi = np.nonzero(valid)[0][:24]
    goal = st[gi].astype(F32)
    appr = goal.astype(np.float64)
    appr[:, :7] -= 0.1 * appr[:, 8:15]
    states = np.concatenate([states, appr.astype(F32)])
    t = np.concatenate([t, (Tq[gi] - 0.1).astype(F32)])
    parent = np.concatenate([parent, np.zeros(len(gi), parent.dtype)])
    return dict(pr=pr, root=root, tree=(states, t, parent), cand=goal, n_goal=len(gi),
                T_req=Tq[gi].astype(F32), v_rel=vr[gi].astype(F32), z=Z[gi].astype(F32))


def _round(P, arm, case, flags):
    states, t, parent = case["tree"]
    N, B = states.shape[0], case["cand"].shape[0]
    pl = P.Planner(arm, P=1, n_cap=N + B + 8, b_max=B, k=5, K=K_GRID, S=S_COLL)
    prob = P.problem_struct(case["pr"], B, case["n_goal"], root=case["root"])
    pl.reset([prob])
    pl.load_tree(0, states, t, parent)
    pl.set_candidates(0, case["cand"], case["n_goal"], case["T_req"], case["v_rel"])
    pl.set_candidate_params(0, case["z"])
    out = pl.iterate([prob], 0, P.FN_PLAN_EXTERNAL | flags)[0]
    tree = pl.get_tree(0)
    zn = pl.get_node_params(0, tree["n"])
    pl.close()
    return out, tree, zn


@pytest.mark.parametrize("seed", [3, 4])
def test_grefine_improves_the_incumbent(P, orc, arm, seed):
    case = _case(arm, orc, seed)
    out0, tree0, zn0 = _round(P, arm, case, 0)
    assert out0["incumbent"] >= 0, "the plain round attached no rendezvous"
    out1, tree1, zn1 = _round(P, arm, case, P.FN_PLAN_GREFINE)
    n0 = tree0["n"]
    # the rounds agree up to the refinement's appended node
    assert tree1["n"] in (n0, n0 + 1)
    assert np.array_equal(tree1["states"][:n0], tree0["states"][:n0])
    inc = out0["incumbent"]
    par = int(tree0["parent"][inc])
    z0 = zn0[inc].astype(np.float64)
    ps, tp, nup = tree0["states"][par], float(tree0["t"][par]), float(tree0["nu"][par])
    J0, feas0, _ = R.node_eval(arm, case["pr"], z0, ps, tp, nup, S_COLL)
    ref = R.refine_node(arm, case["pr"], z0, ps, tp, nup, S_COLL)
    gain_ref = ref["J"] - J0
    if tree1["n"] == n0:                      # nothing accepted on the GPU
        assert out1["incumbent"] == inc
        assert gain_ref < 1e-3, (gain_ref, "the oracle's refinement improved; the GPU's did not")
        return
    m = n0                                    # the appended node
    assert out1["incumbent"] == m and int(tree1["parent"][m]) == par
    zg = zn1[m].astype(np.float64)
    Jg, feas, det = R.node_eval(arm, case["pr"], zg, ps, tp, nup, S_COLL)
    assert feas, "the refined node fails the oracle's exact check"
    assert float(tree1["J"][m]) == pytest.approx(Jg, rel=1e-4, abs=1e-4)
    assert np.abs(tree1["states"][m, :7] - det["state"][:7]).max() < 2e-3
    assert Jg > J0
    assert out1["J"] == pytest.approx(float(tree1["J"][m]), rel=1e-6)
    if gain_ref > 1e-3:
        assert Jg - J0 >= 0.5 * gain_ref, (Jg - J0, gain_ref)
