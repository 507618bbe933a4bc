"""Pins of the oracle's N-ary refinement of the minimum feasible time.

The paper finds T* of Def. "Minimum feasible time" by an N-ary search: the
bracket is split into N equal slots, all slot boundaries are checked, and the
slot where the check first passes is split again, until it is narrower than
eps, in ceil(log_N(width / eps)) rounds.

* One link turning about a vertical axis, rest to rest, no friction or
  gravity: rho_tau = 6 I |dq| / (T^2 tau_max) at the end samples, so
  T* = sqrt(6 I |dq| / tau_max) in closed form; the refined bracket must hold
  it and be no wider than eps.
* On random 7-DOF edges: the bracket lies inside the grid cell of the grid
  scan's k*, its upper end passes the check and its lower end fails it;
  the ratios and ok are those at the refined T*.
* Where max(rho_tau, rho_P) is monotone on the cell (seen on a dense sweep),
  the dense sweep's first passing duration lies in the bracket: a brute-force
  search that shares nothing with the N-ary loop.
* The number of rounds is ceil(log_32(cell width / eps)) (the slot width
  shrinks by exactly 32 per round, up to the rounding of the single-precision
  bracket ends), capped by max_rounds; a
  tolerance wider than the cell leaves the grid result unchanged.
"""
import math

import numpy as np
import pytest

from paper_2609_22608_gb300 import synth
from tests.test_oracle_edges import _itot, one_link_arm


def test_closed_form_bracket(orc, arm):
    a = one_link_arm(arm)
    I = _itot(a)
    Tg = synth.duration_grid(64)
    rng = np.random.default_rng(17)
    dqs = rng.uniform(-3, 3, 48)
    s0 = np.zeros((48, 16), np.float32)
    s1 = np.zeros((48, 16), np.float32)
    s0[:, 0] = 0.3
    s1[:, 0] = 0.3 + dqs
    eps = 1e-5
    res = orc.time_edges_nary(a, s0, s1, Tg, 32, eps)
    n_in = 0
    for e in range(48):
        dq = float(s1[e, 0]) - float(s0[e, 0])
        Tstar = math.sqrt(6 * I * abs(dq) / float(a["tau_max"][0]))
        if res["k_star"][e] < 0:
            assert Tstar > float(Tg[-1])
            continue
        lo, hi = float(res["T_lo"][e]), float(res["T_star"][e])
        assert hi - lo <= eps
        # stay clear of the bracket's ends so rounding cannot decide them
        if min(abs(Tstar - lo), abs(Tstar - hi)) < 1e-9 * Tstar:
            continue
        assert lo < Tstar <= hi
        assert res["ok"][e] == 1
        assert res["rho3"][e, 0] == pytest.approx(6 * I * abs(dq) / (hi * hi * float(a["tau_max"][0])), rel=1e-9)
        n_in += 1
    assert n_in >= 30


def test_bracket_invariants(orc, arm):
    s0, s1 = synth.random_edges(arm, 64, 23)
    Tg = synth.duration_grid(64)
    S = 16
    grid = orc.time_edges(arm, s0, s1, Tg, S)
    res = orc.time_edges_nary(arm, s0, s1, Tg, S, 2e-4)
    assert np.array_equal(res["k_star"], grid["k_star"])
    hit = np.flatnonzero(res["k_star"] >= 0)
    assert len(hit) >= 20
    miss = res["k_star"] < 0
    assert np.all(np.isnan(res["T_lo"][miss]))
    assert np.array_equal(res["T_star"][miss], grid["T_star"][miss], equal_nan=True)
    lo, hi = res["T_lo"][hit].astype(np.float64), res["T_star"][hit].astype(np.float64)
    k = res["k_star"][hit]
    cell_lo = np.where(k > 0, Tg[np.maximum(k - 1, 0)], 0.0)
    assert np.all(lo >= cell_lo) and np.all(hi <= Tg[k]) and np.all(lo < hi)
    assert np.all(hi - lo <= 2e-4)
    r_hi = orc.rho_batch(arm, s0[hit], s1[hit], hi, S)
    assert np.all((r_hi[:, 0] <= 1) & (r_hi[:, 1] <= 1))
    assert np.allclose(res["rho3"][hit], r_hi, rtol=0, atol=0)
    assert np.array_equal(res["ok"][hit], (r_hi[:, 2] <= 1).astype(np.uint8))
    pos = lo > 0
    r_lo = orc.rho_batch(arm, s0[hit][pos], s1[hit][pos], lo[pos], S)
    assert np.all(np.maximum(r_lo[:, 0], r_lo[:, 1]) > 1)


def test_dense_sweep_lies_in_bracket(orc, arm):
    s0, s1 = synth.random_edges(arm, 24, 31)
    Tg = synth.duration_grid(32)
    S = 12
    res = orc.time_edges_nary(arm, s0, s1, Tg, S, 1e-4)
    checked = 0
    for e in np.flatnonzero(res["k_star"] > 0):
        k = int(res["k_star"][e])
        ts = np.linspace(float(Tg[k - 1]), float(Tg[k]), 801)
        r = orc.rho_batch(arm, np.repeat(s0[e:e + 1], len(ts), 0), np.repeat(s1[e:e + 1], len(ts), 0), ts, S)
        m = np.maximum(r[:, 0], r[:, 1])
        if np.any(np.diff(m) > 0):
            continue                      # not monotone on this cell: no claim
        first = ts[np.argmax(m <= 1)]
        step = ts[1] - ts[0]
        # the sweep's first passing point is within one sweep step above T*
        assert float(res["T_lo"][e]) - 1e-12 <= first <= float(res["T_star"][e]) + step
        checked += 1
    assert checked >= 5


@pytest.mark.parametrize("eps", [3e-3, 1e-4, 2e-6])
def test_round_count(orc, arm, eps):
    s0, s1 = synth.random_edges(arm, 48, 41)
    Tg = synth.duration_grid(64)
    res = orc.time_edges_nary(arm, s0, s1, Tg, 8, eps, max_rounds=8)
    hit = np.flatnonzero(res["k_star"] >= 0)
    n = 0
    for e in hit:
        k = int(res["k_star"][e])
        w0 = float(Tg[k]) - (float(Tg[k - 1]) if k > 0 else 0.0)
        x = math.log(w0 / eps, 32)
        if x <= 0:
            assert res["rounds"][e] == 0
            n += 1
            continue
        # the bracket's ends are single-precision values: its width carries
        # an error of a few ulp of T, which can decide the last round
        if abs(w0 / 32 ** math.ceil(x) - eps) <= 4 * float(np.spacing(np.float32(Tg[k]))):
            continue
        assert res["rounds"][e] == math.ceil(x)
        n += 1
    assert n >= 20


def test_wide_tolerance_and_round_cap(orc, arm):
    s0, s1 = synth.random_edges(arm, 32, 43)
    Tg = synth.duration_grid(64)
    grid = orc.time_edges(arm, s0, s1, Tg, 16)
    wide = orc.time_edges_nary(arm, s0, s1, Tg, 16, 10.0)
    assert np.all(wide["rounds"] == 0)
    assert np.array_equal(wide["T_star"], grid["T_star"], equal_nan=True)
    assert np.array_equal(wide["ok"], grid["ok"])
    capped = orc.time_edges_nary(arm, s0, s1, Tg, 16, 1e-7, max_rounds=1)
    hit = capped["k_star"] >= 0
    assert np.all(capped["rounds"][hit] == 1)
    k = capped["k_star"][hit]
    w0 = Tg[k].astype(np.float64) - np.where(k > 0, Tg[np.maximum(k - 1, 0)], 0.0)
    width = capped["T_star"][hit].astype(np.float64) - capped["T_lo"][hit]
    ulp = np.spacing(Tg[k]).astype(np.float64)
    assert np.all(np.abs(width - w0 / 32) <= 2 * ulp)


def test_invalid_and_capped_edges(orc, arm):
    s0, s1 = synth.random_edges(arm, 8, 47)
    s1[2, 3] = np.nan
    Tg = synth.duration_grid(64)
    cap = np.full(8, 0.2, np.float32)
    res = orc.time_edges_nary(arm, s0, s1, Tg, 16, 1e-4, T_cap=cap)
    assert res["k_star"][2] == -2 and np.isnan(res["T_star"][2])
    ok = res["k_star"] >= 0
    assert np.all(res["T_star"][ok] <= 0.2)
