"""fn_knn_tree_static: the parent search for callers that cannot allocate
device memory (a real-time planning thread that must stay out of the CUDA
allocator, or a host whose device memory is budgeted at start-up).  Called
through the C ABI and compared with fn_knn_tree (caller workspace) on two
calls in a row, and with the FP64 oracle's brute-force scan, with the kNN
parity rule of the other tests.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2609_22608_gb300 import synth
from tests.parity import knn_mismatches

pytestmark = pytest.mark.gpu


def _static_fn():
    from paper_2609_22608_gb300._lib import lib
    L = lib()
    f = L.fn_knn_tree_static
    f.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_float,
                  C.c_void_p, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return f


def _static_call(f, tree, N, first, q, B, k, stream):
    idx = torch.full((B, k), -7, dtype=torch.int32, device="cuda")
    d2 = torch.full((B, k), -7.0, device="cuda")
    st = f(C.c_void_p(tree.data_ptr()), N, first, C.c_void_p(q.data_ptr()), B, k, 0.1,
           C.c_void_p(idx.data_ptr()), C.c_void_p(d2.data_ptr()), C.c_void_p(stream.cuda_stream))
    return st, idx, d2


@pytest.mark.parametrize("k", [8, 16])
def test_static_knn_matches_workspace_knn(arm, orc, k):
    """Two calls in a row (the second sees the first's array contents), the
    split pass in use (B = 2048 over 4096 nodes), k on both list widths."""
    from paper_2609_22608_gb300 import ops
    f = _static_fn()
    B, N = 2048, 4096
    tree_h = synth.random_states(arm, N, 41)
    tree = torch.from_numpy(tree_h).cuda()
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((42, 43)):
        q_h = synth.random_states(arm, B, seed)
        q = torch.from_numpy(q_h).cuda()
        st, idx_s, d2_s = _static_call(f, tree, N, 1, q, B, k, stream)
        assert st == 0, f"call {call}: status {st}"
        ws = torch.empty(ops.knn_workspace_bytes(B, N, k) + 256, dtype=torch.uint8, device="cuda")
        idx_w, d2_w = ops.knn_tree(tree, q, k, 0.1, first=1, workspace=ws)
        torch.cuda.synchronize()
        a_i, a_d = idx_s.cpu().numpy(), d2_s.cpu().numpy()
        b_i, b_d = idx_w.cpu().numpy(), d2_w.cpu().numpy()
        assert not knn_mismatches(a_i, a_d, b_i, b_d), f"call {call}"
        assert np.allclose(a_d, b_d, rtol=1e-6, atol=0)
        r_i, r_d = orc.knn(tree_h, q_h, k, 0.1, first=1)
        assert not knn_mismatches(a_i, a_d, r_i, r_d), f"call {call} vs oracle"
        assert np.allclose(a_d, r_d, rtol=1e-5, atol=1e-6)


def test_static_knn_largest_batch(arm, orc):
    """B at the entry point's limit (65536 queries), k = 16, against the
    oracle on a sample of the queries."""
    f = _static_fn()
    B, N, k = 65536, 2000, 16
    tree_h = synth.random_states(arm, N, 51)
    q_h = synth.random_states(arm, B, 52)
    tree = torch.from_numpy(tree_h).cuda()
    q = torch.from_numpy(q_h).cuda()
    st, idx, d2 = _static_call(f, tree, N, 1, q, B, k, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert st == 0
    rows = np.random.default_rng(5).choice(B, 512, replace=False)
    a_i, a_d = idx.cpu().numpy()[rows], d2.cpu().numpy()[rows]
    r_i, r_d = orc.knn(tree_h, q_h[rows], k, 0.1, first=1)
    assert not knn_mismatches(a_i, a_d, r_i, r_d)


def test_static_knn_empty_candidate_set(arm):
    """first == N: no candidates, every slot idx -1 and d2 +inf."""
    f = _static_fn()
    N, B, k = 64, 32, 8
    tree = torch.from_numpy(synth.random_states(arm, N, 61)).cuda()
    q = torch.from_numpy(synth.random_states(arm, B, 62)).cuda()
    st, idx, d2 = _static_call(f, tree, N, N, q, B, k, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert st == 0
    assert np.all(idx.cpu().numpy() == -1)
    assert np.all(np.isinf(d2.cpu().numpy()))


def test_static_knn_rejects_oversize(arm):
    f = _static_fn()
    q = torch.zeros(16, 16, device="cuda")
    out_i = torch.zeros(16, 4, dtype=torch.int32, device="cuda")
    out_d = torch.zeros(16, 4, device="cuda")
    # B beyond FN_KNN_STATIC_MAX_QUERIES (65536) is refused before any launch
    st = f(C.c_void_p(q.data_ptr()), 16, 1, C.c_void_p(q.data_ptr()), 65537, 4, 0.1,
           C.c_void_p(out_i.data_ptr()), C.c_void_p(out_d.data_ptr()), None)
    assert st == -1
