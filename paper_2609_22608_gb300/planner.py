"""Python binding of the planner part of the C ABI (fn_planner_*, fn_plan_*).

Argument marshalling only: every step of an iteration runs in libfruitninja.so.
"""
from __future__ import annotations

import ctypes as C
import ctypes as _ct

import numpy as np
import torch

from ._lib import arm_struct, check, lib
from .synth import duration_grid

FN_PLAN_EXTERNAL = 1
FN_PLAN_PRUNE = 2
FN_PLAN_DENSITY = 4
FN_PLAN_CHORD = 8
FN_PLAN_REFIT = 16
FN_PLAN_NARY = 32
FN_PLAN_GREFINE = 64
FN_DENSITY_MAX_C = 4
FN_ARCHIVE_MAX = 64
FN_MAX_OBS = 8


class FnDensity(C.Structure):
    _fields_ = [("C", C.c_int), ("w_u", C.c_float), ("pi", C.c_float * FN_DENSITY_MAX_C),
                ("mu", (C.c_float * 9) * FN_DENSITY_MAX_C),
                ("sd", (C.c_float * 9) * FN_DENSITY_MAX_C)]


class FnSamplerCfg(C.Structure):
    _fields_ = [("w_u", C.c_float), ("C", C.c_int), ("n_fit", C.c_int), ("em_iters", C.c_int),
                ("sd_floor", C.c_float), ("sd_init", C.c_float), ("w_chord", C.c_float),
                ("chord_sigma", C.c_float)]


def density_to_dict(d: FnDensity) -> dict:
    Cn = int(d.C)
    return dict(C=Cn, w_u=float(d.w_u), pi=np.array(d.pi[:Cn], np.float32),
                mu=np.array([list(d.mu[m]) for m in range(Cn)], np.float32).reshape(Cn, 9),
                sd=np.array([list(d.sd[m]) for m in range(Cn)], np.float32).reshape(Cn, 9))


def density_from_dict(th: dict) -> FnDensity:
    d = FnDensity()
    d.C = int(th["C"])
    d.w_u = float(th["w_u"])
    for m in range(d.C):
        d.pi[m] = float(th["pi"][m])
        for k in range(9):
            d.mu[m][k] = float(th["mu"][m][k])
            d.sd[m][k] = float(th["sd"][m][k])
    return d


class FnPlannerCfg(C.Structure):
    _fields_ = [("P", C.c_int), ("n_cap", C.c_int), ("b_max", C.c_int), ("k", C.c_int),
                ("K", C.c_int), ("T_lo", C.c_float), ("T_hi", C.c_float), ("S", C.c_int),
                ("S_clear", C.c_int), ("reach_grid", C.c_int), ("w_vel", C.c_float),
                ("vel_frac", C.c_float), ("clear_margin", C.c_float), ("edge_blocks", C.c_int)]


class FnProblem(C.Structure):
    _fields_ = [("q0", C.c_float * 7), ("qd0", C.c_float * 7), ("x0", C.c_float * 3),
                ("v0", C.c_float * 3), ("g", C.c_float * 3), ("t_enter", C.c_float),
                ("t_fall", C.c_float), ("t_offset", C.c_float), ("sig_p", C.c_float),
                ("sig_v", C.c_float), ("sig_a", C.c_float), ("sig_linear", C.c_int),
                ("sig_lin_a", C.c_float), ("sig_lin_b", C.c_float), ("a_min", C.c_float),
                ("v_min", C.c_float), ("w_v", C.c_float), ("v_target", C.c_float),
                ("w_p", C.c_float), ("w_r", C.c_float), ("w_x", C.c_float),
                ("r_catch", C.c_float), ("nu0", C.c_float), ("lam", C.c_float),
                ("v_tip", C.c_float), ("batch", C.c_int), ("n_goal", C.c_int),
                ("n_obs", C.c_int), ("obs", (C.c_float * 4) * FN_MAX_OBS),
                ("seed", C.c_ulonglong)]


class FnRendezvous(C.Structure):
    _fields_ = [("q_g", C.c_float * 7), ("qd_g", C.c_float * 7), ("T", C.c_float),
                ("J", C.c_float), ("t_best", C.c_float), ("incumbent", C.c_int),
                ("n_nodes", C.c_int), ("n_added", C.c_int), ("status", C.c_int)]


def _bind():
    L = lib()
    if getattr(L, "_planner_bound", False):
        return L
    vp, i32 = C.c_void_p, C.c_int
    L.fn_planner_create.argtypes = [C.POINTER(FnPlannerCfg), vp, C.POINTER(vp)]
    L.fn_planner_destroy.argtypes = [vp]
    L.fn_planner_reset.argtypes = [vp, vp, vp]
    L.fn_planner_load_tree.argtypes = [vp, i32, vp, vp, vp, i32, vp]
    L.fn_planner_set_candidates.argtypes = [vp, i32, vp, i32, i32, vp, vp, vp]
    L.fn_plan_iteration.argtypes = [vp, vp, i32, C.c_uint, vp, vp]
    L.fn_planner_capture.argtypes = [vp, C.c_uint, vp]
    L.fn_plan_replay.argtypes = [vp, vp, i32, vp, vp]
    L.fn_plan_replay_async.argtypes = [vp, vp, i32, vp]
    L.fn_plan_result.argtypes = [vp, vp]
    L.fn_planner_get_tree.argtypes = [vp, i32, vp, vp, vp, vp, vp, C.POINTER(C.c_int), i32]
    L.fn_planner_get_candidates.argtypes = [vp, i32, vp, vp, vp, vp, i32]
    L.fn_planner_get_parents.argtypes = [vp, i32, vp, i32]
    L.fn_planner_get_edges.argtypes = [vp, i32, vp, vp, vp, vp, i32]
    L.fn_planner_get_node_params.argtypes = [vp, i32, vp, i32]
    L.fn_planner_sample_count.argtypes = [vp, vp, i32]
    L.fn_planner_phase_ms.argtypes = [vp, vp]
    L.fn_planner_kernel_ms.argtypes = [vp, vp, vp, i32, C.POINTER(C.c_int)]
    L.fn_planner_set_surrogate.argtypes = [vp, vp, i32]
    L.fn_planner_work_counts.argtypes = [vp, vp, i32, i32]
    L.fn_planner_autotune.argtypes = [vp, vp, i32, C.c_uint, i32, vp, vp, vp]
    L.fn_planner_set_schedule.argtypes = [vp, i32]
    L.fn_planner_incumbent_path.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp]
    L.fn_planner_set_sampler.argtypes = [vp, C.POINTER(FnSamplerCfg)]
    L.fn_planner_set_density.argtypes = [vp, i32, C.POINTER(FnDensity), vp]
    L.fn_planner_get_density.argtypes = [vp, i32, C.POINTER(FnDensity), vp, vp, C.POINTER(C.c_int)]
    L.fn_planner_set_candidate_params.argtypes = [vp, i32, vp, i32, vp]
    L.fn_planner_get_candidate_params.argtypes = [vp, i32, vp, i32]
    L.fn_planner_set_refine.argtypes = [vp, C.c_float, i32]
    L.fn_planner_set_grid.argtypes = [vp, vp, i32]
    L.fn_planner_set_grefine.argtypes = [vp, i32, C.c_float, C.c_float]
    for n in ("fn_planner_create", "fn_planner_destroy", "fn_planner_reset", "fn_planner_load_tree",
              "fn_planner_set_candidates", "fn_plan_iteration", "fn_planner_capture",
              "fn_plan_replay", "fn_plan_replay_async", "fn_plan_result", "fn_planner_get_tree", "fn_planner_get_candidates",
              "fn_planner_get_parents", "fn_planner_get_edges", "fn_planner_get_node_params",
              "fn_planner_sample_count", "fn_planner_phase_ms", "fn_planner_autotune",
              "fn_planner_set_schedule",
              "fn_planner_kernel_ms", "fn_planner_work_counts", "fn_planner_set_surrogate",
              "fn_planner_incumbent_path", "fn_planner_set_sampler", "fn_planner_set_density",
              "fn_planner_get_density", "fn_planner_set_candidate_params",
              "fn_planner_get_candidate_params", "fn_planner_set_refine",
              "fn_planner_set_grid", "fn_planner_set_grefine"):
        getattr(L, n).restype = i32
    L._planner_bound = True
    return L


def problem_struct(pr: dict, batch: int, n_goal: int, root=None, obstacles=None,
                   seed: int = 0) -> FnProblem:
    """FnProblem from synth.make_problem's dict, a root state [16] and an
    optional [n][4] obstacle array."""
    s = FnProblem()
    root = pr.get("root") if root is None else root
    root = np.zeros(16, np.float32) if root is None else np.asarray(root, np.float32)
    s.q0[:] = [float(x) for x in root[0:7]]
    s.qd0[:] = [float(x) for x in root[8:15]]
    for f in ("x0", "v0", "g"):
        getattr(s, f)[:] = [float(x) for x in np.asarray(pr[f], np.float32)]
    for f in ("t_enter", "t_fall", "t_offset", "sig_p", "sig_v", "sig_a", "sig_lin_a", "sig_lin_b",
              "a_min", "v_min", "w_v", "v_target", "w_p", "w_r", "w_x", "r_catch", "nu0", "lam",
              "v_tip"):
        setattr(s, f, float(np.float32(pr[f])))
    s.sig_linear = int(pr["sig_linear"])
    s.batch = int(batch)
    s.n_goal = int(n_goal)
    obs = np.zeros((0, 4), np.float32) if obstacles is None else np.asarray(obstacles, np.float32)
    if obs.shape[0] > FN_MAX_OBS:
        raise ValueError("too many obstacles")
    s.n_obs = int(obs.shape[0])
    for i in range(obs.shape[0]):
        s.obs[i][:] = [float(x) for x in obs[i]]
    s.seed = int(seed)
    return s


def rendezvous_dict(r: FnRendezvous) -> dict:
    return dict(q_g=np.array(r.q_g[:], np.float32), qd_g=np.array(r.qd_g[:], np.float32),
                T=float(r.T), J=float(r.J), t_best=float(r.t_best), incumbent=int(r.incumbent),
                n_nodes=int(r.n_nodes), n_added=int(r.n_added), status=int(r.status))


class Planner:
    def __init__(self, arm, P=1, n_cap=8192, b_max=2048, k=8, K=128, T_lo=0.05, T_hi=2.0, S=64,
                 S_clear=8, reach_grid=256, w_vel=0.1, vel_frac=0.5, clear_margin=0.02,
                 edge_blocks=0):
        L = _bind()
        self.cfg = FnPlannerCfg(P, n_cap, b_max, k, K, T_lo, T_hi, S, S_clear, reach_grid, w_vel,
                                vel_frac, clear_margin, edge_blocks)
        self.arm = arm_struct(arm)
        h = C.c_void_p()
        check(L.fn_planner_create(C.byref(self.cfg), C.byref(self.arm), C.byref(h)),
              "fn_planner_create")
        self.h = h
        self.P = P
        self._probs = (FnProblem * P)()
        self._out = (FnRendezvous * P)()
        # the duration grid of Sec. IV-D as every other component builds it
        # (FP64 log spacing of the exact endpoints, rounded to FP32)
        self.set_grid(duration_grid(K, T_lo, T_hi))

    def set_grid(self, grid):
        """fn_planner_set_grid: the planner's K grid durations (ascending)."""
        g = np.ascontiguousarray(grid, np.float32)
        check(lib().fn_planner_set_grid(self.h, g.ctypes.data, int(g.shape[0])),
              "fn_planner_set_grid")
        self.grid = g

    def close(self):
        if self.h:
            lib().fn_planner_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stage(self, probs):
        if len(probs) != self.P:
            raise ValueError("need one problem per planner slot")
        for i, p in enumerate(probs):
            self._probs[i] = p

    @staticmethod
    def _stream(stream):
        s = stream if stream is not None else torch.cuda.current_stream()
        return C.c_void_p(s.cuda_stream)

    def reset(self, probs, stream=None):
        """fn_planner_reset (asynchronous on the stream)."""
        self._stage(probs)
        check(lib().fn_planner_reset(self.h, self._probs, self._stream(stream)), "fn_planner_reset")

    def load_tree(self, p, states, t, parent, stream=None):
        """fn_planner_load_tree (asynchronous on the stream: arrays in page-locked
        memory must stay unchanged until the stream has executed the copies)."""
        st = np.ascontiguousarray(states, np.float32)
        t = np.ascontiguousarray(t, np.float32)
        par = np.ascontiguousarray(parent, np.int32)
        check(lib().fn_planner_load_tree(self.h, int(p), st.ctypes.data, t.ctypes.data,
                                         par.ctypes.data, int(st.shape[0]), self._stream(stream)),
              "fn_planner_load_tree")

    def set_candidates(self, p, states, n_goal, T_req=None, v_rel=None, stream=None):
        st = np.ascontiguousarray(states, np.float32)
        tq = np.ascontiguousarray(np.zeros(0) if T_req is None else T_req, np.float32)
        vr = np.ascontiguousarray(np.zeros(0) if v_rel is None else v_rel, np.float32)
        check(lib().fn_planner_set_candidates(self.h, int(p), st.ctypes.data, int(st.shape[0]),
                                              int(n_goal), tq.ctypes.data if n_goal else None,
                                              vr.ctypes.data if n_goal else None,
                                              self._stream(stream)), "fn_planner_set_candidates")

    def iterate(self, probs, it=0, flags=0, stream=None):
        self._stage(probs)
        check(lib().fn_plan_iteration(self.h, self._probs, int(it), int(flags), self._out,
                                      self._stream(stream)), "fn_plan_iteration")
        return [rendezvous_dict(self._out[i]) for i in range(self.P)]

    def capture(self, flags=0, stream=None):
        check(lib().fn_planner_capture(self.h, int(flags), self._stream(stream)),
              "fn_planner_capture")

    def replay(self, probs, it=0, stream=None):
        self._stage(probs)
        check(lib().fn_plan_replay(self.h, self._probs, int(it), self._out, self._stream(stream)),
              "fn_plan_replay")
        return [rendezvous_dict(self._out[i]) for i in range(self.P)]

    def replay_async(self, probs, it=0, stream=None):
        """fn_plan_replay_async: enqueue the captured graph and return; the
        rendezvous records come from result()."""
        self._stage(probs)
        check(lib().fn_plan_replay_async(self.h, self._probs, int(it), self._stream(stream)),
              "fn_plan_replay_async")

    def result(self):
        """fn_plan_result: wait for the last replay_async and return its records."""
        check(lib().fn_plan_result(self.h, self._out), "fn_plan_result")
        return [rendezvous_dict(self._out[i]) for i in range(self.P)]

    def get_tree(self, p, cap=None):
        cap = self.cfg.n_cap if cap is None else cap
        st = np.zeros((cap, 16), np.float32)
        t = np.zeros(cap, np.float32)
        par = np.zeros(cap, np.int32)
        J = np.zeros(cap, np.float32)
        nu = np.zeros(cap, np.float32)
        n = C.c_int()
        check(lib().fn_planner_get_tree(self.h, int(p), st.ctypes.data, t.ctypes.data,
                                        par.ctypes.data, J.ctypes.data, nu.ctypes.data,
                                        C.byref(n), int(cap)), "fn_planner_get_tree")
        m = min(n.value, cap)
        return dict(states=st[:m], t=t[:m], parent=par[:m], J=J[:m], nu=nu[:m], n=n.value)

    def get_candidates(self, p, B):
        st = np.zeros((B, 16), np.float32)
        tq = np.zeros(B, np.float32)
        vr = np.zeros(B, np.float32)
        va = np.zeros(B, np.uint8)
        check(lib().fn_planner_get_candidates(self.h, int(p), st.ctypes.data, tq.ctypes.data,
                                              vr.ctypes.data, va.ctypes.data, int(B)),
              "fn_planner_get_candidates")
        return dict(states=st, T_req=tq, v_rel=vr, valid=va)

    def get_parents(self, p, B):
        """fn_planner_get_parents: [B][k-1] nearest non-root tree nodes."""
        nn = np.zeros((B, max(self.cfg.k - 1, 0)), np.int32)
        check(_bind().fn_planner_get_parents(self.h, int(p), nn.ctypes.data, int(B)),
              "fn_planner_get_parents")
        return nn

    def get_edges(self, p, B):
        """fn_planner_get_edges: per (candidate, parent slot) results [B][k]
        of the last iteration: dict(k_star, T, rho_v, ok)."""
        k = self.cfg.k
        ks = np.zeros((B, k), np.int32)
        T = np.zeros((B, k), np.float32)
        rv = np.zeros((B, k), np.float32)
        ok = np.zeros((B, k), np.uint8)
        check(_bind().fn_planner_get_edges(self.h, int(p), ks.ctypes.data, T.ctypes.data,
                                           rv.ctypes.data, ok.ctypes.data, int(B)),
              "fn_planner_get_edges")
        return dict(k_star=ks, T=T, rho_v=rv, ok=ok)

    def get_node_params(self, p, n):
        """fn_planner_get_node_params: chart parameters [n][9] of the first n
        nodes (NaN where unknown)."""
        z = np.zeros((n, 9), np.float32)
        check(_bind().fn_planner_get_node_params(self.h, int(p), z.ctypes.data, int(n)),
              "fn_planner_get_node_params")
        return z

    def autotune(self, probs, it=0, flags=0, reps=3, stream=None):
        """fn_planner_autotune: returns (chosen variant, ms per variant)."""
        self._stage(probs)
        chosen = C.c_int()
        ms = (C.c_float * 4)()
        check(lib().fn_planner_autotune(self.h, self._probs, int(it), int(flags), int(reps),
                                        C.byref(chosen), ms, self._stream(stream)),
              "fn_planner_autotune")
        return chosen.value, [float(x) for x in ms]

    def set_schedule(self, variant):
        """fn_planner_set_schedule: the edge phase's schedule for later iterations."""
        check(lib().fn_planner_set_schedule(self.h, int(variant)), "fn_planner_set_schedule")

    PHASES = ("schedule", "sample", "parents", "edge_prep", "probe", "verify", "attach",
              "prune", "output")

    def phase_ms(self):
        ms = (C.c_float * 9)()
        check(lib().fn_planner_phase_ms(self.h, ms), "fn_planner_phase_ms")
        return dict(zip(self.PHASES, [float(x) for x in ms]))

    def set_refine(self, eps=1e-4, max_rounds=8):
        """fn_planner_set_refine (set before capture)."""
        check(lib().fn_planner_set_refine(self.h, float(eps), int(max_rounds)),
              "fn_planner_set_refine")

    def set_grefine(self, iters=8, eta0=0.05, h=1e-3):
        """fn_planner_set_grefine (set before capture)."""
        check(lib().fn_planner_set_grefine(self.h, int(iters), float(eta0), float(h)),
              "fn_planner_set_grefine")

    def set_sampler(self, w_u=0.25, C=4, n_fit=32, em_iters=8, sd_floor=0.02, sd_init=0.1,
                    w_chord=0.5, chord_sigma=0.1):
        """fn_planner_set_sampler (set before capture)."""
        cfg = FnSamplerCfg(w_u, C, n_fit, em_iters, sd_floor, sd_init, w_chord, chord_sigma)
        self._scfg = cfg
        check(lib().fn_planner_set_sampler(self.h, _ct.byref(cfg)), "fn_planner_set_sampler")

    def set_density(self, p, theta, stream=None):
        """fn_planner_set_density from dict(C, w_u, pi, mu, sd)."""
        d = density_from_dict(theta)
        check(lib().fn_planner_set_density(self.h, int(p), C.byref(d), self._stream(stream)),
              "fn_planner_set_density")

    def get_density(self, p):
        """fn_planner_get_density: (theta dict, archive J [n], archive z [n][9])."""
        d = FnDensity()
        J = np.zeros(FN_ARCHIVE_MAX, np.float32)
        Z = np.zeros((FN_ARCHIVE_MAX, 9), np.float32)
        n = C.c_int()
        check(lib().fn_planner_get_density(self.h, int(p), C.byref(d), J.ctypes.data, Z.ctypes.data,
                                           C.byref(n)), "fn_planner_get_density")
        return density_to_dict(d), J[:n.value].copy(), Z[:n.value].copy()

    def set_candidate_params(self, p, z, stream=None):
        """fn_planner_set_candidate_params: chart parameters [n_goal][9] of the
        external goal candidates."""
        z = np.ascontiguousarray(z, np.float32).reshape(-1, 9)
        check(lib().fn_planner_set_candidate_params(self.h, int(p), z.ctypes.data, int(z.shape[0]),
                                                    self._stream(stream)),
              "fn_planner_set_candidate_params")

    def get_candidate_params(self, p, n):
        """fn_planner_get_candidate_params: chart parameters [n][9] (NaN where
        unknown)."""
        z = np.zeros((n, 9), np.float32)
        check(lib().fn_planner_get_candidate_params(self.h, int(p), z.ctypes.data, int(n)),
              "fn_planner_get_candidate_params")
        return z

    def incumbent_path(self, p, max_edges=64, stream=None):
        """fn_planner_incumbent_path: the incumbent plan of problem p as edges,
        root first.  Returns dict(s0, s1 [max_edges,16], T [max_edges],
        nodes [max_edges+1], n_edges [1]) on the device (stream-ordered; the
        first n_edges rows are valid when 0 < n_edges <= max_edges)."""
        dev = torch.device("cuda")
        m = max(int(max_edges), 1)
        out = dict(s0=torch.zeros(m, 16, device=dev), s1=torch.zeros(m, 16, device=dev),
                   T=torch.full((m,), float("nan"), device=dev),
                   nodes=torch.full((m + 1,), -1, dtype=torch.int32, device=dev),
                   n_edges=torch.zeros(1, dtype=torch.int32, device=dev))
        check(lib().fn_planner_incumbent_path(self.h, int(p), int(max_edges),
                                              C.c_void_p(out["s0"].data_ptr()),
                                              C.c_void_p(out["s1"].data_ptr()),
                                              C.c_void_p(out["T"].data_ptr()),
                                              C.c_void_p(out["nodes"].data_ptr()),
                                              C.c_void_p(out["n_edges"].data_ptr()),
                                              self._stream(stream)), "fn_planner_incumbent_path")
        return out

    def recheck_incumbent(self, arm, p, S=256, S_clear=64, obs=None, margin=0.02, max_edges=64,
                          stream=None):
        """The full-resolution recheck of Sec. IV-E on the incumbent plan of
        problem p: fn_planner_incumbent_path chained into fn_check_edges_full
        on the device (no host synchronisation between them).  Returns the
        path dict with rho3, clearance and ok added."""
        from . import ops
        path = self.incumbent_path(p, max_edges, stream=stream)
        res = ops.check_edges_full(arm, path["s0"], path["s1"], path["T"], S, S_clear, obs,
                                   margin, E_dev=path["n_edges"], stream=stream)
        path.update(res)
        return path

    def set_surrogate(self, mlp, W=16):
        """fn_planner_set_surrogate: route free edges through the duration
        surrogate's window pass (mlp = None turns it off)."""
        self._sur = mlp                      # keep the model alive
        check(_bind().fn_planner_set_surrogate(self.h, mlp.h if mlp is not None else None, int(W)),
              "fn_planner_set_surrogate")

    def kernel_ms(self):
        """fn_planner_kernel_ms: [(kernel name, ms)] of every launch of the
        last fn_plan_iteration, in launch order."""
        cap = 64
        ms = (C.c_float * cap)()
        names = (C.c_char_p * cap)()
        n = C.c_int()
        check(_bind().fn_planner_kernel_ms(self.h, ms, names, cap, C.byref(n)),
              "fn_planner_kernel_ms")
        return [(names[i].decode(), float(ms[i])) for i in range(min(n.value, cap))]

    WORK = ("probe", "verify", "mprobe", "knn_pairs", "ik_starts", "surrogate_edges",
            "surrogate_rescans", "refine", "goal_defined", "goal_speed", "goal_ik", "goal_box",
            "goal_singular", "goal_taper")

    def work_counts(self, reset=False):
        """fn_planner_work_counts: dict of the planner's work counters."""
        n = len(self.WORK)
        c = (C.c_ulonglong * n)()
        check(_bind().fn_planner_work_counts(self.h, c, n, int(bool(reset))),
              "fn_planner_work_counts")
        return dict(zip(self.WORK, [int(x) for x in c]))

    def sample_count(self, reset=False):
        """Torque evaluations of the edge kernels: dict(probe=..., verify=...)."""
        c = (C.c_ulonglong * 2)()
        check(lib().fn_planner_sample_count(self.h, c, int(bool(reset))),
              "fn_planner_sample_count")
        return {"probe": int(c[0]), "verify": int(c[1])}
