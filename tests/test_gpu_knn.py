"""Parity of the CUDA nearest-parent search (fn_knn_tree) with the oracle's
brute force."""
import numpy as np
import pytest
import torch

from paper_2609_22608_gb300 import synth
from tests.parity import knn_mismatches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ops():
    from paper_2609_22608_gb300 import ops as o
    return o


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("B,N,k,first,ws", [
    (2048, 4096, 8, 1, True),     # planning-iteration shape
    (2048, 4096, 8, 1, False),    # single-pass path (no workspace)
    (300, 1000, 16, 1, True),
    (129, 257, 5, 0, True),
    (7, 3, 4, 1, True),           # fewer candidates than k
    (1, 1, 1, 1, True),           # only the root: nothing to return
    (64, 130, 16, 0, False),
])
def test_knn_parity(ops, orc, arm, B, N, k, first, ws):
    tree = synth.random_states(arm, N, 5 + N)
    q = synth.random_states(arm, B, 6 + B)
    if N > 20:
        tree[N // 2] = tree[3]          # exact duplicates: ties go to the lower index
        q[0] = tree[3]
    workspace = None
    if ws:
        need = ops.knn_workspace_bytes(B, N, k)
        workspace = torch.empty(max(need, 1) + 256, dtype=torch.uint8, device="cuda")
    idx, d2 = ops.knn_tree(dev(tree), dev(q), k, 0.1, first=first, workspace=workspace)
    ig, dg = idx.cpu().numpy(), d2.cpu().numpy()
    ri, rd = orc.knn(tree, q, k, 0.1, first=first)
    bad = knn_mismatches(ig, dg, ri, rd)
    assert not bad, (bad[:4], ig[bad[0]], ri[bad[0]])
    fin = np.isfinite(rd)
    assert np.allclose(dg[fin], rd[fin], rtol=1e-5, atol=1e-6)
    assert np.all(ig[~fin] == -1)
    if N > 20 and first <= 3:
        assert ig[0, 0] == 3 and ig[0, 1] == N // 2


def test_knn_full_size_sampled(ops, orc, arm):
    """The anytime-stress shape (8192 queries, 65536 nodes, k = 16): sampled
    queries against the brute force, and sortedness everywhere."""
    B, N, k = 8192, 65536, 16
    tree = synth.random_states(arm, N, 99)
    q = synth.random_states(arm, B, 98)
    idx, d2 = ops.knn_tree(dev(tree), dev(q), k, 0.1)
    ig, dg = idx.cpu().numpy(), d2.cpu().numpy()
    assert np.all(np.diff(dg, axis=1) >= 0)
    sel = np.random.default_rng(1).choice(B, 64, replace=False)
    ri, rd = orc.knn(tree, q[sel], k, 0.1)
    assert not knn_mismatches(ig[sel], dg[sel], ri, rd)
