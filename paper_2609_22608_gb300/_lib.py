"""ctypes binding of libfruitninja.so (argument marshalling only).

Every function here forwards device pointers (from torch CUDA tensors), sizes
and the current CUDA stream to the C ABI declared in include/fn_api.h and
raises on a non-OK status.  There is no fallback: if the library is missing
the import of this module fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfruitninja.so")

F7 = C.c_float * 7
F73 = (C.c_float * 3) * 7
F3 = C.c_float * 3

FN_MODE_FULL = 0
FN_MODE_FIXED = 1


class FnArm(C.Structure):
    _fields_ = [
        ("dof", C.c_int),
        ("dh_a", F7), ("dh_alpha", F7), ("dh_d", F7), ("dh_theta0", F7),
        ("mass", F7), ("com", F73), ("inertia", F73),
        ("armature", F7), ("fric", F73),
        ("q_lo", F7), ("q_hi", F7), ("qd_max", F7), ("qd_taper_a", F7),
        ("tau_max", F7), ("w_max", C.c_float),
        ("gravity", F3),
        ("flange_d", C.c_float),
        ("blade_base", F3), ("blade_axis", F3), ("blade_normal", F3), ("blade_len", C.c_float),
        ("link_radius", F7),
    ]


class FnError(RuntimeError):
    pass


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FnError(f"{LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
    L = C.CDLL(LIB_PATH)
    vp, i32, f32, sz = C.c_void_p, C.c_int, C.c_float, C.c_size_t
    L.fn_status_str.argtypes = [i32]
    L.fn_status_str.restype = C.c_char_p
    L.fn_version.restype = C.c_char_p
    L.fn_time_edges.argtypes = [C.POINTER(FnArm), vp, vp, i32, vp, i32, i32, i32, vp, vp, vp, vp,
                                vp, vp, vp]
    L.fn_rnea_dump.argtypes = [C.POINTER(FnArm), vp, vp, vp, i32, i32, vp, vp]
    L.fn_knn_workspace_bytes.argtypes = [i32, i32, i32]
    L.fn_knn_workspace_bytes.restype = sz
    L.fn_knn_tree.argtypes = [vp, i32, i32, vp, i32, i32, f32, vp, vp, vp, sz, vp]
    L.fn_time_edges_counted.argtypes = [C.POINTER(FnArm), vp, vp, i32, vp, i32, i32, i32, vp, vp,
                                        vp, vp, vp, vp, vp, vp]
    L.fn_make_edges.argtypes = [vp, vp, vp, i32, i32, vp, i32, vp, f32, vp, vp, vp, vp, vp]
    L.fn_time_edges_nary.argtypes = [C.POINTER(FnArm), vp, vp, i32, vp, i32, i32, vp, f32, i32,
                                     vp, vp, vp, vp, vp, vp, vp, vp]
    L.fn_autotune_time_edges.argtypes = [C.POINTER(FnArm), vp, vp, i32, vp, i32, i32, i32, vp,
                                         vp, vp, vp, vp, vp, i32, vp, vp, vp]
    L.fn_check_edges_full.argtypes = [C.POINTER(FnArm), vp, vp, vp, i32, vp, i32, i32, i32, vp,
                                      f32, vp, vp, vp, vp]
    L.fn_controller_torque.argtypes = [C.POINTER(FnArm), i32, vp, vp, vp, vp, f32, vp, vp, vp,
                                       vp, vp]
    for name in ("fn_time_edges", "fn_rnea_dump", "fn_knn_tree", "fn_time_edges_counted",
                 "fn_make_edges", "fn_time_edges_nary", "fn_autotune_time_edges",
                 "fn_check_edges_full", "fn_controller_torque"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def check(status: int, what: str) -> None:
    if status != 0:
        raise FnError(f"{what}: {lib().fn_status_str(status).decode()}")


def arm_struct(arm) -> FnArm:
    """FnArm from the dict produced by synth.make_arm (or an FnArm)."""
    if isinstance(arm, FnArm):
        return arm
    s = FnArm()
    s.dof = int(arm["dof"])
    for name in ("dh_a", "dh_alpha", "dh_d", "dh_theta0", "mass", "armature", "q_lo", "q_hi",
                 "qd_max", "qd_taper_a", "tau_max", "link_radius"):
        v = np.asarray(arm[name], np.float32)
        getattr(s, name)[:] = [float(x) for x in v]
    for name in ("com", "inertia", "fric"):
        v = np.asarray(arm[name], np.float32)
        tgt = getattr(s, name)
        for i in range(7):
            tgt[i][:] = [float(x) for x in v[i]]
    for name in ("gravity", "blade_base", "blade_axis", "blade_normal"):
        getattr(s, name)[:] = [float(x) for x in np.asarray(arm[name], np.float32)]
    s.w_max = float(arm["w_max"])
    s.flange_d = float(arm["flange_d"])
    s.blade_len = float(arm["blade_len"])
    return s
