"""Pins of the oracle's sampling densities (Sec. IV-E, "Batched expansion").

* p_theta with no Gaussian component (or the uniform component drawn) is the
  uniform chart sampler; the component frequencies follow (w_u, pi); a narrow
  component reproduces its mean and deviation (Box-Muller normals); draws are
  folded into [0, 1] (angles wrap, the others reflect).
* The chord sampler with w_chord = 0 is the uniform free sampler; with zero
  spread its configurations lie on the chords from the root to the given
  goals, choosing the goals uniformly.
* The EM refit: one component gives the sample mean and the sample variance
  plus the floor; two separated clusters are found with their weights; the
  mixture log-likelihood never decreases over the iterations.
* The best-plans archive keeps the n_fit best (J, z), best first, with
  earlier entries winning ties.
"""
import numpy as np
import pytest

from oracle import density as OD
from paper_2609_22608_gb300 import synth


def _theta(C, w_u, pi, mu, sd):
    return dict(C=C, w_u=w_u, pi=np.asarray(pi, np.float32),
                mu=np.asarray(mu, np.float32).reshape(C, 9),
                sd=np.asarray(sd, np.float32).reshape(C, 9))


def test_empty_density_is_uniform_sampler(orc, arm):
    toss = synth.random_toss(arm, 4)
    pr = synth.make_problem(toss, root=synth.random_states(arm, 1, 4)[0])
    ref = orc.sample_goals(arm, pr, 55, 3, 1, 0, 256)
    for th in (dict(C=0, w_u=0.25, pi=[], mu=[], sd=[]),
               _theta(1, 1.0, [1.0], np.full(9, 0.3), np.full(9, 0.01))):
        st, Tq, vr, valid, z = orc.sample_goals_density(arm, pr, th, 55, 3, 1, 0, 256)
        assert np.array_equal(valid, ref[3])
        assert np.array_equal(st, ref[0]) and np.array_equal(Tq, ref[1])


def test_component_frequencies_and_moments(orc):
    mu = np.array([np.full(9, 0.2), np.full(9, 0.5), np.full(9, 0.8)])
    th = _theta(3, 0.25, [0.5, 0.3, 0.2], mu, np.full((3, 9), 0.01))
    n = 20000
    zs = np.array([orc.density_z(th, 9, i, 0, 0) for i in range(n)])
    d = np.linalg.norm(zs[:, None, :] - mu[None], axis=2)
    near = np.min(d, axis=1) < 0.1
    which = np.argmin(d, axis=1)
    expect = {"uniform": 0.25, 0: 0.75 * 0.5, 1: 0.75 * 0.3, 2: 0.75 * 0.2}
    # a uniform draw lands within 0.1 of a mean with negligible probability
    f_u = np.mean(~near)
    assert abs(f_u - expect["uniform"]) < 4 * np.sqrt(0.25 * 0.75 / n)
    for m in range(3):
        f = np.mean(near & (which == m))
        assert abs(f - expect[m]) < 4 * np.sqrt(expect[m] * (1 - expect[m]) / n)
    # moments of one component (Box-Muller normals)
    th1 = _theta(1, 0.0, [1.0], np.full(9, 0.5), np.full(9, 0.05))
    z1 = np.array([orc.density_z(th1, 10, i, 1, 2) for i in range(n)])
    assert np.all(np.abs(z1.mean(axis=0) - 0.5) < 4 * 0.05 / np.sqrt(n))
    assert np.all(np.abs(z1.std(axis=0) / 0.05 - 1) < 0.03)


def test_folding_into_the_cube(orc):
    th = _theta(1, 0.0, [1.0], np.full(9, 0.98), np.full(9, 0.05))
    zs = np.array([orc.density_z(th, 3, i, 0, 0) for i in range(4000)])
    assert np.all((zs >= 0) & (zs <= 1))
    for i in range(9):
        if i in (2, 3, 4):          # angles wrap past 1 to near 0
            assert np.mean(zs[:, i] < 0.1) > 0.2
        else:                       # reflected at 1: nothing near 0
            assert np.min(zs[:, i]) > 0.7
            assert np.mean(zs[:, i] > 0.98) < 0.5


def test_chord_sampler(orc, arm):
    q0 = synth.random_states(arm, 1, 1)[0, :7].astype(np.float64)
    goals = synth.random_states(arm, 5, 2).astype(np.float64)
    n = 3000
    uni = orc.sample_uniform(arm, 21, 4, 0, 100, n, 0.5)
    none = orc.sample_chord(arm, 21, 4, 0, 100, n, 0.5, q0, goals, 0.0, 0.1)
    assert np.array_equal(none, uni)
    nog = orc.sample_chord(arm, 21, 4, 0, 100, n, 0.5, q0, goals[:0], 1.0, 0.1)
    assert np.array_equal(nog, uni)
    on = orc.sample_chord(arm, 21, 4, 0, 100, n, 0.5, q0, goals, 1.0, 0.0)
    lo, hi = np.asarray(arm["q_lo"], np.float64), np.asarray(arm["q_hi"], np.float64)
    counts = np.zeros(5)
    for c in range(n):
        q = on[c, :7]
        # on the chord to one goal: q - q0 = lambda (q_g - q0), 0 <= lambda <= 1
        best = None
        for g in range(5):
            dg = goals[g, :7] - q0
            lam = float((q - q0) @ dg / (dg @ dg))
            err = np.abs(q - q0 - lam * dg).max()
            if err < 1e-12 and -1e-12 <= lam <= 1 + 1e-12:
                best = g
                break
        assert best is not None
        counts[best] += 1
        assert np.all(q >= lo) and np.all(q <= hi)
    assert np.all(np.abs(counts / n - 0.2) < 4 * np.sqrt(0.2 * 0.8 / n))
    spread = orc.sample_chord(arm, 21, 4, 0, 100, n, 0.5, q0, goals, 1.0, 0.2)
    assert np.all(spread[:, :7] >= lo) and np.all(spread[:, :7] <= hi)
    assert np.any(np.abs(spread[:, :7] - on[:, :7]) > 1e-3)


def test_em_one_component_closed_form():
    rng = np.random.default_rng(1)
    zs = rng.uniform(0.3, 0.6, (20, 9))
    th0 = dict(C=0, w_u=0.25, pi=[], mu=[], sd=[])
    th = OD.em_refit(zs, th0, 1, 1, 0.02, 0.1)
    assert th["C"] == 1 and th["pi"][0] == pytest.approx(1.0)
    assert np.allclose(th["mu"][0], zs.mean(axis=0), rtol=1e-12)
    assert np.allclose(th["sd"][0], np.sqrt(zs.var(axis=0) + 0.02 ** 2), rtol=1e-12)


def test_em_two_clusters_and_monotone_likelihood():
    rng = np.random.default_rng(2)
    a = 0.25 + 0.02 * rng.standard_normal((30, 9))
    b = 0.75 + 0.02 * rng.standard_normal((10, 9))
    zs = np.concatenate([a[:1], b[:1], a[1:], b[1:]])    # best two first: one per cluster
    th = dict(C=0, w_u=0.25, pi=[], mu=[], sd=[])
    lls = []
    cur = OD.em_refit(zs, th, 2, 1, 0.01, 0.1)
    lls.append(OD.mixture_loglik(zs, cur))
    for _ in range(6):
        cur = OD.em_refit(zs, cur, 2, 1, 0.0, 0.1)
        lls.append(OD.mixture_loglik(zs, cur))
    assert all(y >= x - 1e-9 for x, y in zip(lls[1:], lls[2:]))
    order = np.argsort(cur["mu"][:, 0])
    assert np.allclose(cur["mu"][order[0]], a.mean(axis=0), atol=1e-6)
    assert np.allclose(cur["mu"][order[1]], b.mean(axis=0), atol=1e-6)
    assert np.allclose(np.sort(cur["pi"]), [0.25, 0.75], atol=1e-6)


def test_archive_order_ties_and_capacity():
    arc = []
    for J, tag in [(1.0, 0), (3.0, 1), (2.0, 2), (3.0, 3), (0.5, 4), (2.5, 5)]:
        arc = OD.archive_insert(arc, J, np.full(9, tag), 4)
    assert [j for j, _ in arc] == [3.0, 3.0, 2.5, 2.0]
    assert [int(z[0]) for _, z in arc] == [1, 3, 5, 2]
    arc = OD.archive_insert(arc, 2.0, np.full(9, 9), 4)     # ties the last: dropped
    assert [int(z[0]) for _, z in arc] == [1, 3, 5, 2]
