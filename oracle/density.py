"""FP64 restatement of the goal density's refit (Sec. IV-E, "Batched
expansion"): p_theta is a Gaussian mixture over the chart parameters mixed
with a uniform component, refit between anytime iterations to the parameters
that produced the best plans.  TEST INFRASTRUCTURE ONLY (see fn_oracle.h).

Readings:
  * the best plans are an archive of (J, z) of rendezvous nodes, best J
    first, at most n_fit entries; a new entry goes after the entries with the
    same J (earlier plans win ties), and entries past n_fit are dropped;
  * the refit runs em_iters EM iterations on the archive's z with diagonal
    covariances; the first fit starts from the min(C, n) best z with
    standard deviation sd_init and equal weights, later fits from the
    current mixture; variances get sd_floor^2 added; a component whose
    responsibility sum is below 1e-4 keeps its mean and deviation (its
    weight becomes that sum / n); the uniform weight w_u is not fit.
"""
import math

import numpy as np


def archive_insert(archive, J, z, n_fit):
    """archive: list of (J, z) best first; returns the updated list."""
    out = list(archive)
    pos = len(out)
    for i, (Ji, _) in enumerate(out):
        if J > Ji:
            pos = i
            break
    if pos >= n_fit:
        return out
    out.insert(pos, (float(J), np.asarray(z, np.float64)))
    return out[:n_fit]


def em_refit(zs, theta, C_max, em_iters, sd_floor, sd_init):
    """zs [n][9] (archive order); theta dict(C, w_u, pi, mu, sd); returns a new
    theta dict with float64 arrays."""
    zs = np.asarray(zs, np.float64)
    n = zs.shape[0]
    if n == 0:
        return theta
    if theta["C"] == 0:
        C = min(C_max, n)
        mu = zs[:C].copy()
        sd = np.full((C, 9), float(sd_init))
        pi = np.full(C, 1.0 / C)
    else:
        C = int(theta["C"])
        mu = np.asarray(theta["mu"], np.float64)[:C].copy()
        sd = np.asarray(theta["sd"], np.float64)[:C].copy()
        pi = np.asarray(theta["pi"], np.float64)[:C].copy()
    for _ in range(em_iters):
        # E-step: responsibilities r[i, m] proportional to pi_m N(z_i; mu_m, sd_m^2)
        logp = np.zeros((n, C))
        for m in range(C):
            d = (zs - mu[m]) / sd[m]
            with np.errstate(divide="ignore"):
                logp[:, m] = math.log(pi[m]) if pi[m] > 0 else -math.inf
            logp[:, m] += -0.5 * np.sum(d * d, axis=1) - np.sum(np.log(sd[m]))
        top = np.max(logp, axis=1, keepdims=True)
        w = np.exp(logp - top)
        r = w / np.sum(w, axis=1, keepdims=True)
        # M-step
        Nm = r.sum(axis=0)
        for m in range(C):
            pi[m] = Nm[m] / n
            if Nm[m] < 1e-4:
                continue
            mu[m] = (r[:, m:m + 1] * zs).sum(axis=0) / Nm[m]
            var = (r[:, m:m + 1] * (zs - mu[m]) ** 2).sum(axis=0) / Nm[m]
            sd[m] = np.sqrt(var + sd_floor * sd_floor)
    return dict(C=C, w_u=theta["w_u"], pi=pi, mu=mu, sd=sd)


def mixture_loglik(zs, theta):
    """sum_i log sum_m pi_m N(z_i; mu_m, sd_m^2) (the Gaussian part only)."""
    zs = np.asarray(zs, np.float64)
    tot = 0.0
    for z in zs:
        acc = 0.0
        for m in range(theta["C"]):
            d = (z - theta["mu"][m]) / theta["sd"][m]
            acc += theta["pi"][m] * math.exp(-0.5 * float(d @ d)) / (
                np.prod(theta["sd"][m]) * (2 * math.pi) ** 4.5)
        tot += math.log(acc)
    return tot
