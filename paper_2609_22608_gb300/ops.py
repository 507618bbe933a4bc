"""Python entry points with the C ABI's names (include/fn_api.h).

Tensors are torch CUDA tensors (PyTorch provides device memory and streams);
each call forwards pointers and the current stream to libfruitninja.so and
returns the output tensors.  All arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import FN_MODE_FIXED, FN_MODE_FULL, arm_struct, check, lib

__all__ = ["time_edges", "time_edges_nary", "autotune_time_edges", "set_time_edges_variant", "check_edges_full",
           "controller_torque", "rnea_dump", "knn_tree", "knn_workspace_bytes", "make_edges", "EdgeEngine",
           "FN_MODE_FULL", "FN_MODE_FIXED", "version"]


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _states(x, name):
    if not (x.is_cuda and x.dtype == torch.float32 and x.dim() == 2 and x.shape[1] == 16
            and x.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA float32 [n][16] tensor")
    return x


def version() -> str:
    return lib().fn_version().decode()


def time_edges(arm, s0, s1, T_grid=None, S=32, mode=FN_MODE_FULL, T_fixed=None, T_cap=None,
               out=None, stream=None, sample_count=None):
    """fn_time_edges: returns dict(k_star i32, T_star f32, rho3 f32 [E,3], ok u8).
    With `sample_count` (a CUDA int64 tensor of one element) the call goes
    through fn_time_edges_counted and adds its torque evaluations to it."""
    _states(s0, "s0"); _states(s1, "s1")
    E = s0.shape[0]
    A = arm_struct(arm)
    if out is None:
        dev = s0.device
        out = dict(k_star=torch.empty(E, dtype=torch.int32, device=dev),
                   T_star=torch.empty(E, dtype=torch.float32, device=dev),
                   rho3=torch.empty(E, 3, dtype=torch.float32, device=dev),
                   ok=torch.empty(E, dtype=torch.uint8, device=dev))
    if T_grid is None:
        grid = None
        K = 0
    else:
        g = np.ascontiguousarray(np.asarray(T_grid, np.float32))
        grid = g.ctypes.data_as(C.c_void_p)
        K = int(g.size)
    if sample_count is None:
        st = lib().fn_time_edges(C.byref(A), _ptr(s0), _ptr(s1), E, grid, K, int(S), int(mode),
                                 _ptr(T_fixed), _ptr(T_cap), _ptr(out["k_star"]),
                                 _ptr(out["T_star"]), _ptr(out["rho3"]), _ptr(out["ok"]),
                                 _stream(stream))
    else:
        st = lib().fn_time_edges_counted(C.byref(A), _ptr(s0), _ptr(s1), E, grid, K, int(S),
                                         int(mode), _ptr(T_fixed), _ptr(T_cap),
                                         _ptr(out["k_star"]), _ptr(out["T_star"]),
                                         _ptr(out["rho3"]), _ptr(out["ok"]), _ptr(sample_count),
                                         _stream(stream))
    check(st, "fn_time_edges")
    return out


def autotune_time_edges(arm, s0, s1, T_grid, S, reps=3, T_cap=None, stream=None):
    """fn_autotune_time_edges (FULL mode): times every schedule variant of the
    edge kernels on this workload (three register budgets of the scalar scan,
    then the paired scan with tensor-memory records) and keeps the fastest for
    its shape (the N-ary refinement follows a scalar choice).  Returns
    (variant, ms[4])."""
    _states(s0, "s0"); _states(s1, "s1")
    E = s0.shape[0]
    A = arm_struct(arm)
    dev = s0.device
    out = dict(k_star=torch.empty(E, dtype=torch.int32, device=dev),
               T_star=torch.empty(E, dtype=torch.float32, device=dev),
               rho3=torch.empty(E, 3, dtype=torch.float32, device=dev),
               ok=torch.empty(E, dtype=torch.uint8, device=dev))
    g = np.ascontiguousarray(np.asarray(T_grid, np.float32))
    chosen = C.c_int(-1)
    ms = (C.c_float * 4)()
    st = lib().fn_autotune_time_edges(C.byref(A), _ptr(s0), _ptr(s1), E,
                                      g.ctypes.data_as(C.c_void_p), int(g.size), int(S),
                                      FN_MODE_FULL, None, _ptr(T_cap), _ptr(out["k_star"]),
                                      _ptr(out["T_star"]), _ptr(out["rho3"]), _ptr(out["ok"]),
                                      int(reps), C.byref(chosen), ms, _stream(stream))
    check(st, "fn_autotune_time_edges")
    return int(chosen.value), [float(x) for x in ms]


def set_time_edges_variant(mode, E, K, S, variant):
    """fn_time_edges_set_variant: pin the schedule variant (0-2 scalar
    register budgets, 3 paired with tensor-memory records) that time_edges
    uses for this shape on the current device."""
    L = lib()
    L.fn_time_edges_set_variant.argtypes = [C.c_int] * 5
    L.fn_time_edges_set_variant.restype = C.c_int
    check(L.fn_time_edges_set_variant(int(mode), int(E), int(K), int(S), int(variant)),
          "fn_time_edges_set_variant")


def time_edges_nary(arm, s0, s1, T_grid, S, eps, max_rounds=8, T_cap=None, out=None,
                    stream=None, sample_count=None):
    """fn_time_edges_nary: grid scan refined by the N-ary search (N = 32) to a
    bracket (T_lo, T_star] no wider than eps.  Returns dict(k_star, T_star,
    T_lo, rho3, ok, rounds)."""
    _states(s0, "s0"); _states(s1, "s1")
    E = s0.shape[0]
    A = arm_struct(arm)
    if out is None:
        dev = s0.device
        out = dict(k_star=torch.empty(E, dtype=torch.int32, device=dev),
                   T_star=torch.empty(E, dtype=torch.float32, device=dev),
                   T_lo=torch.empty(E, dtype=torch.float32, device=dev),
                   rho3=torch.empty(E, 3, dtype=torch.float32, device=dev),
                   ok=torch.empty(E, dtype=torch.uint8, device=dev),
                   rounds=torch.empty(E, dtype=torch.int32, device=dev))
    g = np.ascontiguousarray(np.asarray(T_grid, np.float32))
    st = lib().fn_time_edges_nary(C.byref(A), _ptr(s0), _ptr(s1), E, g.ctypes.data_as(C.c_void_p),
                                  int(g.size), int(S), _ptr(T_cap), float(eps), int(max_rounds),
                                  _ptr(out["k_star"]), _ptr(out["T_star"]), _ptr(out.get("T_lo")),
                                  _ptr(out["rho3"]), _ptr(out["ok"]), _ptr(out.get("rounds")),
                                  _ptr(sample_count), _stream(stream))
    check(st, "fn_time_edges_nary")
    return out


def check_edges_full(arm, s0, s1, T, S, S_clear=64, obs=None, margin=0.02, E_dev=None,
                     out=None, stream=None):
    """fn_check_edges_full: the full-resolution recheck of edges at their own
    durations.  Returns dict(rho3 f32 [E,3], clearance f32 [E], ok u8 [E])."""
    _states(s0, "s0"); _states(s1, "s1")
    E = s0.shape[0]
    A = arm_struct(arm)
    if out is None:
        dev = s0.device
        out = dict(rho3=torch.empty(E, 3, dtype=torch.float32, device=dev),
                   clearance=torch.empty(E, dtype=torch.float32, device=dev),
                   ok=torch.empty(E, dtype=torch.uint8, device=dev))
    ob = np.zeros((0, 4), np.float32) if obs is None else np.ascontiguousarray(
        np.asarray(obs, np.float32).reshape(-1, 4))
    st = lib().fn_check_edges_full(C.byref(A), _ptr(s0), _ptr(s1), _ptr(T), E, _ptr(E_dev),
                                   int(S), int(S_clear), len(ob),
                                   ob.ctypes.data_as(C.c_void_p) if len(ob) else None,
                                   float(margin), _ptr(out["rho3"]), _ptr(out["clearance"]),
                                   _ptr(out["ok"]), _stream(stream))
    check(st, "fn_check_edges_full")
    return out


def controller_torque(arm, state, goal, T, dt=1e-3, tau_prev=None, tau_rate_max=None, out=None,
                      stream=None):
    """fn_controller_torque: one cycle of Eq. (controller) for B instances.
    Returns dict(tau f32 [B,7], qdd f32 [B,7], flags u8 [B])."""
    _states(state, "state"); _states(goal, "goal")
    B = state.shape[0]
    A = arm_struct(arm)
    if out is None:
        dev = state.device
        out = dict(tau=torch.empty(B, 7, dtype=torch.float32, device=dev),
                   qdd=torch.empty(B, 7, dtype=torch.float32, device=dev),
                   flags=torch.empty(B, dtype=torch.uint8, device=dev))
    rate = None
    if tau_rate_max is not None:
        rate = np.ascontiguousarray(np.asarray(tau_rate_max, np.float32).reshape(7))
    st = lib().fn_controller_torque(C.byref(A), B, _ptr(state), _ptr(goal), _ptr(T),
                                    _ptr(tau_prev), float(dt),
                                    None if rate is None else rate.ctypes.data_as(C.c_void_p),
                                    _ptr(out["tau"]), _ptr(out.get("qdd")),
                                    _ptr(out.get("flags")), _stream(stream))
    check(st, "fn_controller_torque")
    return out


def make_edges(tree, t_node, cand, n_goal, nn_idx, T_req, t_best, out=None, stream=None):
    """fn_make_edges: (s0, s1, T_param, parent) for B (k_nn+1) edges."""
    B = cand.shape[0]
    k_nn = 0 if nn_idx is None else nn_idx.shape[1]
    E = B * (k_nn + 1)
    if out is None:
        d = cand.device
        out = (torch.empty(E, 16, device=d), torch.empty(E, 16, device=d),
               torch.empty(E, device=d), torch.empty(E, dtype=torch.int32, device=d))
    st = lib().fn_make_edges(_ptr(tree), _ptr(t_node), _ptr(cand), B, int(n_goal), _ptr(nn_idx),
                             k_nn, _ptr(T_req), float(t_best), _ptr(out[0]), _ptr(out[1]),
                             _ptr(out[2]), _ptr(out[3]), _stream(stream))
    check(st, "fn_make_edges")
    return out


def rnea_dump(arm, s0, s1, T, S, out=None, stream=None):
    """fn_rnea_dump: torques [E][S][7] along each edge at duration T[e]."""
    _states(s0, "s0"); _states(s1, "s1")
    E = s0.shape[0]
    if out is None:
        out = torch.empty(E, S, 7, dtype=torch.float32, device=s0.device)
    st = lib().fn_rnea_dump(C.byref(arm_struct(arm)), _ptr(s0), _ptr(s1), _ptr(T), E, int(S),
                            _ptr(out), _stream(stream))
    check(st, "fn_rnea_dump")
    return out


def knn_workspace_bytes(B, N, k) -> int:
    return int(lib().fn_knn_workspace_bytes(int(B), int(N), int(k)))


def knn_tree(tree, queries, k, w_vel, first=1, N=None, workspace=None, out=None, stream=None):
    """fn_knn_tree: (idx i32 [B][k], d2 f32 [B][k]).  `workspace` may be a
    uint8 CUDA tensor of knn_workspace_bytes(B, N, k) bytes; by default one is
    allocated with torch for the call."""
    _states(queries, "queries")
    B = queries.shape[0]
    if N is None:
        N = tree.shape[0]
    if out is None:
        out = (torch.empty(B, k, dtype=torch.int32, device=queries.device),
               torch.empty(B, k, dtype=torch.float32, device=queries.device))
    need = knn_workspace_bytes(B, N, k)
    if workspace is None and need > 0:
        workspace = torch.empty(need + 256, dtype=torch.uint8, device=queries.device)
    ws_ptr, ws_bytes = None, 0
    if workspace is not None:
        base = workspace.data_ptr()
        aligned = (base + 255) & ~255
        ws_ptr = C.c_void_p(aligned)
        ws_bytes = workspace.numel() - (aligned - base)
    st = lib().fn_knn_tree(_ptr(tree), int(N), int(first), _ptr(queries), B, int(k),
                           float(w_vel), _ptr(out[0]), _ptr(out[1]), ws_ptr, ws_bytes,
                           _stream(stream))
    check(st, "fn_knn_tree")
    return out


class EdgeEngine:
    """fn_edges_*: the planner's packed edge pipeline over caller-given edge
    arrays (full scan with an optional cap, or the surrogate's window with
    its certificate and exact rescan)."""

    def __init__(self, arm, T_grid, S=64, max_E=65536):
        L = lib()
        vp, i32 = C.c_void_p, C.c_int
        L.fn_edges_create.argtypes = [vp, vp, i32, i32, i32, C.POINTER(vp)]
        L.fn_edges_destroy.argtypes = [vp]
        L.fn_edges_time.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, vp, vp]
        L.fn_edges_time_window.argtypes = [vp, vp, vp, i32, vp, i32, vp, vp, vp, vp, vp, vp]
        L.fn_edges_work_counts.argtypes = [vp, vp, i32, i32]
        for n in ("fn_edges_create", "fn_edges_destroy", "fn_edges_time", "fn_edges_time_window",
                  "fn_edges_work_counts"):
            getattr(L, n).restype = i32
        g = np.ascontiguousarray(np.asarray(T_grid, np.float32))
        self.K = g.size
        self.arm = arm_struct(arm)
        h = C.c_void_p()
        check(L.fn_edges_create(C.byref(self.arm), g.ctypes.data, int(g.size), int(S), int(max_E),
                                C.byref(h)), "fn_edges_create")
        self.h = h

    def close(self):
        if self.h:
            lib().fn_edges_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _outs(self, E, dev):
        return dict(k_star=torch.empty(E, dtype=torch.int32, device=dev),
                    T_star=torch.empty(E, dtype=torch.float32, device=dev),
                    rho_v=torch.empty(E, dtype=torch.float32, device=dev),
                    ok=torch.empty(E, dtype=torch.uint8, device=dev))

    def time(self, s0, s1, T_cap=None, stream=None):
        _states(s0, "s0"), _states(s1, "s1")
        E = s0.shape[0]
        o = self._outs(E, s0.device)
        check(lib().fn_edges_time(self.h, _ptr(s0), _ptr(s1), E, _ptr(T_cap), _ptr(o["k_star"]),
                                  _ptr(o["T_star"]), _ptr(o["rho_v"]), _ptr(o["ok"]),
                                  _stream(stream)), "fn_edges_time")
        return o

    def time_window(self, s0, s1, Y, W=16, stream=None):
        _states(s0, "s0"), _states(s1, "s1")
        E = s0.shape[0]
        o = self._outs(E, s0.device)
        o["path"] = torch.empty(E, dtype=torch.uint8, device=s0.device)
        check(lib().fn_edges_time_window(self.h, _ptr(s0), _ptr(s1), E, _ptr(Y.contiguous()), int(W),
                                         _ptr(o["k_star"]), _ptr(o["T_star"]), _ptr(o["rho_v"]),
                                         _ptr(o["ok"]), _ptr(o["path"]), _stream(stream)),
              "fn_edges_time_window")
        return o

    def work_counts(self, reset=False):
        c = (C.c_ulonglong * 7)()
        check(lib().fn_edges_work_counts(self.h, c, 7, int(bool(reset))), "fn_edges_work_counts")
        return dict(zip(("probe", "verify", "mprobe", "knn_pairs", "ik_starts", "window_edges",
                         "rescans"), [int(x) for x in c]))
