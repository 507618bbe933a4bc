"""Python binding of the duration surrogate (fn_mlp_*) and the windowed scan
(fn_time_edges_window).  Argument marshalling only; all arithmetic runs in
libfruitninja.so.  `train` is a small driver that labels edges with the exact
scan (fn_time_edges) and calls fn_mlp_train_step on minibatches."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import ops
from ._lib import arm_struct, check, lib

DIMS = (32, 256, 256, 256, 2)


def _bind():
    L = lib()
    if getattr(L, "_mlp_bound", False):
        return L
    vp, i32, f32 = C.c_void_p, C.c_int, C.c_float
    L.fn_mlp_create.argtypes = [i32, C.c_ulonglong, C.POINTER(vp)]
    L.fn_mlp_destroy.argtypes = [vp]
    L.fn_mlp_predict.argtypes = [vp, vp, vp, vp, i32, vp, vp]
    L.fn_mlp_predict_ref.argtypes = [vp, vp, vp, vp, i32, vp, vp]
    L.fn_mlp_error.argtypes = [vp, C.POINTER(C.c_int), i32]
    L.fn_mlp_backward.argtypes = [vp, vp, vp, vp, vp, vp, i32, i32, vp, vp]
    L.fn_mlp_adam_step.argtypes = [vp, f32, vp]
    L.fn_mlp_train_step.argtypes = [vp, vp, vp, vp, vp, vp, i32, i32, f32, vp, vp]
    for n in ("fn_mlp_get_params", "fn_mlp_set_params", "fn_mlp_get_grads", "fn_mlp_set_grads"):
        getattr(L, n).argtypes = [vp, i32, vp, vp]
    L.fn_mlp_save.argtypes = [vp, C.c_char_p]
    L.fn_mlp_load.argtypes = [vp, C.c_char_p]
    L.fn_time_edges_window.argtypes = [vp, vp, vp, i32, vp, i32, i32, vp, i32, vp, vp, vp, vp, vp,
                                       vp, vp]
    for n in ("fn_mlp_create", "fn_mlp_destroy", "fn_mlp_predict", "fn_mlp_predict_ref",
              "fn_mlp_error", "fn_mlp_backward",
              "fn_mlp_adam_step", "fn_mlp_train_step", "fn_mlp_get_params", "fn_mlp_set_params",
              "fn_mlp_get_grads", "fn_mlp_set_grads", "fn_mlp_save", "fn_mlp_load",
              "fn_time_edges_window"):
        getattr(L, n).restype = i32
    L._mlp_bound = True
    return L


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _st(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _grid(T_grid):
    g = np.ascontiguousarray(np.asarray(T_grid, np.float32))
    return g, g.ctypes.data_as(C.c_void_p)


class MLP:
    def __init__(self, max_batch=65536, seed=0):
        L = _bind()
        h = C.c_void_p()
        check(L.fn_mlp_create(int(max_batch), int(seed), C.byref(h)), "fn_mlp_create")
        self.h = h
        self.max_batch = max_batch

    def close(self):
        if self.h:
            lib().fn_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def predict(self, arm, s0, s1, out=None, stream=None):
        E = s0.shape[0]
        if out is None:
            out = torch.empty(E, 2, device=s0.device)
        A = arm_struct(arm)
        check(lib().fn_mlp_predict(self.h, C.byref(A), _p(s0), _p(s1), E, _p(out), _st(stream)),
              "fn_mlp_predict")
        return out

    def predict_ref(self, arm, s0, s1, out=None, stream=None):
        """fn_mlp_predict_ref: the forward on the training kernels' path."""
        E = s0.shape[0]
        if out is None:
            out = torch.empty(E, 2, device=s0.device)
        A = arm_struct(arm)
        check(lib().fn_mlp_predict_ref(self.h, C.byref(A), _p(s0), _p(s1), E, _p(out),
                                       _st(stream)), "fn_mlp_predict_ref")
        return out

    def error(self, reset=False):
        """fn_mlp_error: 1 if the tensor-core kernel timed out on a wait."""
        f = C.c_int()
        check(lib().fn_mlp_error(self.h, C.byref(f), int(bool(reset))), "fn_mlp_error")
        return int(f.value)

    def backward(self, arm, s0, s1, k_star, T_grid, stream=None):
        A = arm_struct(arm)
        g, gp = _grid(T_grid)
        loss = C.c_float()
        check(lib().fn_mlp_backward(self.h, C.byref(A), _p(s0), _p(s1), _p(k_star), gp, g.size,
                                    s0.shape[0], C.byref(loss), _st(stream)), "fn_mlp_backward")
        return float(loss.value)

    def adam_step(self, lr, stream=None):
        check(lib().fn_mlp_adam_step(self.h, float(lr), _st(stream)), "fn_mlp_adam_step")

    def train_step(self, arm, s0, s1, k_star, T_grid, lr, stream=None):
        A = arm_struct(arm)
        g, gp = _grid(T_grid)
        loss = C.c_float()
        check(lib().fn_mlp_train_step(self.h, C.byref(A), _p(s0), _p(s1), _p(k_star), gp, g.size,
                                      s0.shape[0], float(lr), C.byref(loss), _st(stream)),
              "fn_mlp_train_step")
        return float(loss.value)

    def _io(self, fn, l, a, b):
        check(fn(self.h, int(l), None if a is None else a.ctypes.data_as(C.c_void_p),
                 None if b is None else b.ctypes.data_as(C.c_void_p)), fn.__name__)

    def get_params(self, l):
        W = np.zeros((DIMS[l], DIMS[l + 1]), np.float32)
        b = np.zeros(DIMS[l + 1], np.float32)
        self._io(lib().fn_mlp_get_params, l, W, b)
        return W, b

    def set_params(self, l, W, b):
        self._io(lib().fn_mlp_set_params, l, np.ascontiguousarray(W, np.float32),
                 np.ascontiguousarray(b, np.float32))

    def get_grads(self, l):
        W = np.zeros((DIMS[l], DIMS[l + 1]), np.float32)
        b = np.zeros(DIMS[l + 1], np.float32)
        self._io(lib().fn_mlp_get_grads, l, W, b)
        return W, b

    def set_grads(self, l, gW, gb):
        self._io(lib().fn_mlp_set_grads, l, np.ascontiguousarray(gW, np.float32),
                 np.ascontiguousarray(gb, np.float32))

    def save(self, path):
        check(lib().fn_mlp_save(self.h, str(path).encode()), "fn_mlp_save")

    def load(self, path):
        check(lib().fn_mlp_load(self.h, str(path).encode()), "fn_mlp_load")


def time_edges_window(arm, s0, s1, T_grid, S, Y, W=16, out=None, with_path=True,
                      sample_count=None, stream=None):
    """fn_time_edges_window: dict(k_star, T_star, rho3, ok, path)."""
    _bind()
    E = s0.shape[0]
    d = s0.device
    if out is None:
        out = dict(k_star=torch.empty(E, dtype=torch.int32, device=d),
                   T_star=torch.empty(E, device=d), rho3=torch.empty(E, 3, device=d),
                   ok=torch.empty(E, dtype=torch.uint8, device=d),
                   path=torch.empty(E, dtype=torch.uint8, device=d) if with_path else None)
    g, gp = _grid(T_grid)
    A = arm_struct(arm)
    check(lib().fn_time_edges_window(C.byref(A), _p(s0), _p(s1), E, gp, g.size, int(S), _p(Y),
                                     int(W), _p(out["k_star"]), _p(out["T_star"]),
                                     _p(out["rho3"]), _p(out["ok"]), _p(out.get("path")),
                                     _p(sample_count), _st(stream)), "fn_time_edges_window")
    return out


def label_edges(arm, s0, s1, T_grid, S, stream=None):
    """Labels for training: k* of the exact full scan (fn_time_edges)."""
    return ops.time_edges(arm, s0, s1, T_grid, S, stream=stream)["k_star"]


def train(mlp, arm, s0, s1, k_star, T_grid, epochs=4, batch=4096, lr=1e-3, seed=0, stream=None):
    """Minibatch Adam over (s0, s1, k_star) (device tensors); returns the
    mean loss of every epoch."""
    E = s0.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(E, generator=g).to(s0.device)
        a, b, k = s0[perm].contiguous(), s1[perm].contiguous(), k_star[perm].contiguous()
        losses = []
        for i in range(0, E - batch + 1, batch):
            losses.append(mlp.train_step(arm, a[i:i + batch], b[i:i + batch], k[i:i + batch],
                                         T_grid, lr, stream=stream))
        hist.append(float(np.mean(losses)))
    return hist
