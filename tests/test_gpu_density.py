"""Parity of the planner's sampling densities (Sec. IV-E, batched expansion)
with the FP64 oracle, through the C ABI: goal parameters from p_theta, the
chord free sampler, the best-plans archive and the EM refit.

Rules: the integer choices (uniform component or not, which component,
chord or not, which goal) are taken in single precision on both sides and
must agree exactly; drawn parameters and configurations agree to FP32
rounding (angle parameters compared modulo 1); the refit's parameters agree
within 1e-4 (FP32 EM against FP64)."""
import numpy as np
import pytest

from oracle import density as OD
from paper_2609_22608_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2609_22608_gb300 import planner as pl
    return pl


def _theta():
    rng = np.random.default_rng(3)
    mu = rng.uniform(0.05, 0.95, (3, 9)).astype(np.float32)
    mu[0, 2] = 0.99                      # an angle parameter next to its wrap
    mu[1, 0] = 0.02                      # a reflected one next to 0
    sd = rng.uniform(0.02, 0.08, (3, 9)).astype(np.float32)
    return dict(C=3, w_u=0.25, pi=np.array([0.5, 0.3, 0.2], np.float32), mu=mu, sd=sd)


def _zdiff(a, b):
    d = np.abs(a - b)
    for i in (2, 3, 4):
        d[:, i] = np.minimum(d[:, i], 1 - d[:, i])
    return d


def test_goal_parameters_from_density(P, orc, arm):
    toss = synth.random_toss(arm, 5)
    pr = synth.make_problem(toss, root=synth.random_states(arm, 1, 10)[0])
    B = 4096
    pl = P.Planner(arm, P=1, n_cap=64, b_max=B, k=1, K=8, S=8)
    prob = P.problem_struct(pr, B, B, seed=77)
    pl.reset([prob])
    th = _theta()
    pl.set_density(0, th)
    pl.iterate([prob], 2, P.FN_PLAN_DENSITY)
    z = pl.get_candidate_params(0, B).astype(np.float64)
    c = pl.get_candidates(0, B)
    pl.close()
    zr = np.array([orc.density_z(th, 77, b, 2, 0) for b in range(B)])
    d = _zdiff(z, zr)
    assert d.max() < 2e-5, (np.unravel_index(np.argmax(d), d.shape), d.max())
    # the uniform draws are the plain sampler's
    ref = orc.sample_goals_density(arm, pr, th, 77, 2, 0, 0, B)
    gv = c["valid"] == 1
    assert np.mean(gv != (ref[3] == 1)) < 0.01
    both = gv & (ref[3] == 1)
    assert both.sum() >= 10
    assert np.allclose(c["T_req"][both], ref[1][both], rtol=1e-6)
    assert np.abs(c["states"][both, :7] - ref[0][both, :7]).max() < 2e-3


def test_density_off_is_the_uniform_sampler(P, orc, arm):
    toss = synth.random_toss(arm, 5)
    pr = synth.make_problem(toss, root=synth.random_states(arm, 1, 10)[0])
    B = 512
    pl = P.Planner(arm, P=1, n_cap=64, b_max=B, k=1, K=8, S=8)
    prob = P.problem_struct(pr, B, B, seed=5)
    pl.reset([prob])
    pl.set_density(0, _theta())
    pl.iterate([prob], 1, 0)                         # flag off: p_theta unused
    z = pl.get_candidate_params(0, B)
    pl.close()
    zr = np.array([orc.density_z(dict(C=0, w_u=0.25), 5, b, 1, 0) for b in range(B)])
    assert np.array_equal(z.astype(np.float64), zr)


def test_chord_sampler(P, orc, arm):
    toss = synth.random_toss(arm, 5)
    root = synth.random_states(arm, 1, 10)[0]
    pr = synth.make_problem(toss, root=root)
    B, G = 3072, 2048
    pl = P.Planner(arm, P=1, n_cap=64, b_max=B, k=1, K=8, S=8)
    pl.set_sampler(w_chord=0.6, chord_sigma=0.15)
    prob = P.problem_struct(pr, B, G, root=root, seed=31)
    pl.reset([prob])
    pl.iterate([prob], 4, P.FN_PLAN_CHORD)
    c = pl.get_candidates(0, B)
    pl.close()
    gv = np.flatnonzero(c["valid"][:G] == 1)
    assert len(gv) >= 5
    goals = c["states"][gv].astype(np.float64)
    q0 = np.asarray(root[:7], np.float64)
    ref = orc.sample_chord(arm, 31, 4, 0, G, B - G, 0.5, q0, goals, 0.6, 0.15)
    q = c["states"][G:, :7].astype(np.float64)
    assert np.allclose(q, ref[:, :7], rtol=0, atol=2e-6)
    # velocities: (2u - 1) vel_frac qdbar(q), the taper taken at the GPU's q
    for j in range(7):
        tr = np.array([orc.taper(arm, j, x) for x in ref[:, j]])
        tg = np.array([orc.taper(arm, j, x) for x in q[:, j]])
        s = np.where(tr > 0, ref[:, 8 + j] / np.where(tr > 0, 0.5 * tr, 1), 0)
        assert np.allclose(c["states"][G:, 8 + j], s * 0.5 * tg, rtol=0,
                           atol=1e-5 * float(arm["qd_max"][j]))
    uni = orc.sample_uniform(arm, 31, 4, 0, G, B - G, 0.5)
    chord = np.any(np.abs(ref[:, :7] - uni[:, :7]) > 0, axis=1)
    assert 0.5 < chord.mean() < 0.7


def test_archive_and_refit(P, orc, arm):
    """The goal-attach round (approach nodes loaded before each decoded goal)
    with the goals' chart parameters given: the archive holds the attached
    rendezvous plans, best first, and the refit matches the oracle's EM."""
    from tests.test_gpu_planner import K_GRID, S_COLL, make_case
    case = make_case(arm, orc, 41, N=150, n_free=32)
    states, t, parent = case["tree"]
    G = case["n_goal"]
    g = case["cand"][:G].astype(np.float64)
    appr = g.copy()
    appr[:, :7] = g[:, :7] - 0.1 * g[:, 8:15]
    states = np.concatenate([states, appr.astype(np.float32)])
    t = np.concatenate([t, (case["T_req"] - np.float32(0.1)).astype(np.float32)])
    parent = np.concatenate([parent, np.zeros(G, parent.dtype)])
    # the goals' chart parameters: make_case decodes uniform draws of seed 141
    draws = orc.sample_goals_density(arm, case["pr"], dict(C=0, w_u=0.25), 141, 0, 0, 0, 512)
    zs = draws[4][np.flatnonzero(draws[3])].astype(np.float32)
    assert zs.shape[0] == G
    N, B = states.shape[0], case["cand"].shape[0]
    pl = P.Planner(arm, P=1, n_cap=N + B + 8, b_max=B, k=5, K=K_GRID, S=S_COLL, S_clear=8)
    pl.set_sampler(C=2, n_fit=8, em_iters=5, sd_floor=0.02, sd_init=0.1, w_u=0.3)
    prob = P.problem_struct(case["pr"], B, G, root=case["root"])
    pl.reset([prob])
    pl.load_tree(0, states, t, parent)
    pl.set_candidates(0, case["cand"], G, case["T_req"], case["v_rel"])
    pl.set_candidate_params(0, zs)
    pl.iterate([prob], 0, P.FN_PLAN_EXTERNAL | P.FN_PLAN_REFIT)
    th, aJ, aZ = pl.get_density(0)
    tree = pl.get_tree(0)
    pl.reset([prob])                                  # a new cycle: archive cleared, p_theta kept
    th2, aJ2, _ = pl.get_density(0)
    pl.close()
    # the archive: the attached rendezvous plans by J, best first
    new = np.arange(N, tree["n"])
    J = tree["J"][new]
    rz = []
    for nd in new[np.isfinite(J)]:
        b = int(np.flatnonzero(np.all(case["cand"][:G] == tree["states"][nd], axis=1))[0])
        rz.append((float(tree["J"][nd]), zs[b]))
    assert len(rz) >= 2
    arc = []
    for Jv, z in rz:
        arc = OD.archive_insert(arc, Jv, z, 8)
    assert np.array_equal(aJ, np.array([j for j, _ in arc], np.float32))
    assert np.array_equal(aZ, np.array([z for _, z in arc], np.float32))
    # the refit
    ref = OD.em_refit(np.array([z for _, z in arc], np.float64), dict(C=0, w_u=0.3), 2, 5, 0.02, 0.1)
    assert th["C"] == ref["C"] and th["w_u"] == pytest.approx(0.3)
    assert np.allclose(th["pi"], ref["pi"], atol=1e-4)
    assert np.allclose(th["mu"], ref["mu"], atol=1e-4)
    assert np.allclose(th["sd"], ref["sd"], atol=1e-4)
    assert len(aJ2) == 0 and th2["C"] == th["C"] and np.array_equal(th2["mu"], th["mu"])


def test_density_arguments(P, arm):
    pl = P.Planner(arm, P=2, n_cap=64, b_max=64, k=1, K=8, S=8)
    from paper_2609_22608_gb300._lib import FnError
    bad = _theta()
    bad["pi"] = np.array([0.5, 0.3, 0.3], np.float32)
    with pytest.raises(FnError):
        pl.set_density(0, bad)
    bad = _theta()
    bad["sd"][1, 4] = 0.0
    with pytest.raises(FnError):
        pl.set_density(1, bad)
    with pytest.raises(FnError):
        pl.set_sampler(C=5)
    with pytest.raises(FnError):
        pl.set_sampler(w_chord=1.5)
    pl.set_density(1, _theta())
    th, aJ, _ = pl.get_density(1)
    assert th["C"] == 3 and np.allclose(th["mu"], _theta()["mu"]) and len(aJ) == 0
    th0, _, _ = pl.get_density(0)
    assert th0["C"] == 0 and th0["w_u"] == pytest.approx(0.25)
    pl.close()
