"""Pins of the surrogate's FP64 reference (oracle/mlp.py): the bf16 rounding
against torch's bfloat16 conversion, and the backward pass of the exact
network against central finite differences of the loss."""
import numpy as np
import pytest
import torch

import oracle.mlp as M


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 10, 20000), rng.uniform(-1e-3, 1e-3, 2000),
                        [0.0, -0.0, 1.0, 65504.0, 1e-30, 3.0e38]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(x), ref)


def _params(rng, dims=(32, 16, 16, 16, 2)):
    return [(rng.normal(0, 1 / np.sqrt(dims[l]), (dims[l], dims[l + 1])), rng.normal(0, 0.1, dims[l + 1]))
            for l in range(4)]


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    params = _params(rng)
    X = rng.normal(0, 1, (24, 32))
    logT = rng.normal(-0.5, 0.5, 24)
    feas = rng.uniform(size=24) < 0.7
    ident = lambda a: np.asarray(a, np.float64)
    y, cache = M.forward(params, X, rnd=ident)
    L, dy = M.loss_and_grad_y(y, logT, feas)
    grads = M.backward(params, cache, dy, rnd=ident)
    h = 1e-6

    def loss_at(ps):
        yy, _ = M.forward(ps, X, rnd=ident)
        return M.loss_and_grad_y(yy, logT, feas)[0]

    for l in range(4):
        W, b = params[l]
        for (i, j) in [(0, 0), (3, min(5, W.shape[1] - 1)), (W.shape[0] - 1, W.shape[1] - 1)]:
            Wp = W.copy(); Wp[i, j] += h
            Wm = W.copy(); Wm[i, j] -= h
            pp = list(params); pp[l] = (Wp, b)
            pm = list(params); pm[l] = (Wm, b)
            fd = (loss_at(pp) - loss_at(pm)) / (2 * h)
            assert grads[l][0][i, j] == pytest.approx(fd, rel=1e-5, abs=1e-9)
        for j in (0, b.shape[0] - 1):
            bp = b.copy(); bp[j] += h
            bm = b.copy(); bm[j] -= h
            pp = list(params); pp[l] = (W, bp)
            pm = list(params); pm[l] = (W, bm)
            fd = (loss_at(pp) - loss_at(pm)) / (2 * h)
            assert grads[l][1][j] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_adam_first_step_is_signed_lr():
    """Adam's first step from zero moments moves each parameter by
    lr * g / (|g| + eps) (bias-corrected moments equal g and g^2)."""
    rng = np.random.default_rng(2)
    params = _params(rng)
    grads = [(rng.normal(0, 1, W.shape), rng.normal(0, 1, b.shape)) for W, b in params]
    zeros = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    out, m, v = M.adam(params, grads, zeros, zeros, 1, 1e-3)
    for (W, b), (W2, b2), (gW, gb) in zip(params, out, grads):
        assert np.allclose(W2 - W, -1e-3 * gW / (np.abs(gW) + 1e-8), rtol=1e-10, atol=1e-15)
        assert np.allclose(b2 - b, -1e-3 * gb / (np.abs(gb) + 1e-8), rtol=1e-10, atol=1e-15)
