"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It binds ``fn_oracle.c`` (plain double-precision
loops over the paper's definitions) through ctypes and adds the plan-level
steps of Algorithm 1 in ``oracle.plan``.  It shares no code with the CUDA
library; the only module both sides use is the seeded input generator.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fn_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

D7 = C.c_double * 7
D73 = (C.c_double * 3) * 7
D3 = C.c_double * 3


class OrArm(C.Structure):
    _fields_ = [
        ("dof", C.c_int),
        ("a", D7), ("alpha", D7), ("d", D7), ("theta0", D7),
        ("mass", D7), ("com", D73), ("inertia", D73),
        ("armature", D7), ("fric", D73),
        ("q_lo", D7), ("q_hi", D7), ("qd_max", D7), ("taper_a", D7),
        ("tau_max", D7), ("w_max", C.c_double),
        ("gravity", D3),
        ("flange_d", C.c_double),
        ("blade_base", D3), ("blade_axis", D3), ("blade_normal", D3), ("blade_len", C.c_double),
        ("link_radius", D7),
    ]


class OrProblem(C.Structure):
    _fields_ = [
        ("x0", D3), ("v0", D3),
        ("t_enter", C.c_double), ("t_fall", C.c_double), ("t_offset", C.c_double),
        ("sig_p", C.c_double), ("sig_v", C.c_double), ("sig_a", C.c_double),
        ("sig_linear", C.c_int), ("sig_lin_a", C.c_double), ("sig_lin_b", C.c_double),
        ("a_min", C.c_double), ("v_min", C.c_double),
        ("w_v", C.c_double), ("v_target", C.c_double), ("w_p", C.c_double), ("w_r", C.c_double),
        ("w_x", C.c_double), ("r_catch", C.c_double), ("nu0", C.c_double), ("lam", C.c_double),
        ("v_tip", C.c_double),
        ("g", D3),
    ]


def build(force: bool = False) -> str:
    """Compile fn_oracle.c into liboracle.so (gcc, OpenMP, portable flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "fn_oracle.h"))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.POINTER
        L.or_time_edges.argtypes = [P(OrArm), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                    C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_time_edges_nary.argtypes = [P(OrArm), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_int, C.c_int, C.c_void_p, C.c_float, C.c_int,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_controller_torque.argtypes = [P(OrArm), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p]
        L.or_check_edges.argtypes = [P(OrArm), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                     C.c_int, C.c_void_p, C.c_int, C.c_double, C.c_void_p,
                                     C.c_void_p, C.c_void_p]
        L.or_density_z.argtypes = [C.c_void_p, C.c_ulonglong, C.c_int, C.c_int, C.c_int, C.c_void_p]
        L.or_sample_goals_density.argtypes = [P(OrArm), P(OrProblem), C.c_void_p, C.c_ulonglong,
                                              C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_sample_chord.argtypes = [P(OrArm), C.c_ulonglong, C.c_int, C.c_int, C.c_int, C.c_int,
                                      C.c_double, C.c_void_p, C.c_void_p, C.c_int, C.c_float,
                                      C.c_double, C.c_void_p]
        L.or_rho_batch.argtypes = [P(OrArm), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                   C.c_void_p]
        L.or_torque_dump.argtypes = [P(OrArm), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_int, C.c_void_p]
        L.or_torque.argtypes = [P(OrArm), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_rnea.argtypes = [P(OrArm), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_friction.argtypes = [C.c_void_p, C.c_double]
        L.or_friction.restype = C.c_double
        L.or_taper.argtypes = [P(OrArm), C.c_int, C.c_double]
        L.or_taper.restype = C.c_double
        L.or_cubic.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_knn.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int,
                             C.c_double, C.c_void_p, C.c_void_p]
        L.or_fk.argtypes = [P(OrArm), C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_blade.argtypes = [P(OrArm), C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_jacobian_point.argtypes = [P(OrArm), C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_philox4x32.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_goal_chart.argtypes = [P(OrArm), P(OrProblem), C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_goal_chart.restype = C.c_int
        L.or_sample_uniform.argtypes = [P(OrArm), C.c_ulonglong, C.c_int, C.c_int, C.c_int,
                                        C.c_int, C.c_double, C.c_void_p]
        L.or_sample_goals.argtypes = [P(OrArm), P(OrProblem), C.c_ulonglong, C.c_int, C.c_int,
                                      C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p]
        L.or_objective.argtypes = [P(OrProblem), C.c_double, C.c_double, C.c_double]
        L.or_objective.restype = C.c_double
        L.or_reach_time.argtypes = [P(OrArm), P(OrProblem), C.c_void_p, C.c_double, C.c_int,
                                    C.c_void_p]
        L.or_reach_time.restype = C.c_int
        L.or_edge_clearance.argtypes = [P(OrArm), C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                        C.c_void_p, C.c_int]
        L.or_edge_clearance.restype = C.c_double
        L.or_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def _d(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size >= n
    return a


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def arm_struct(arm: dict) -> OrArm:
    s = OrArm()
    s.dof = int(arm["dof"])

    def put(field, val, shape=None):
        v = np.asarray(val, np.float64)
        tgt = getattr(s, field)
        if v.ndim == 1:
            for i, x in enumerate(v):
                tgt[i] = float(x)
        else:
            for i in range(v.shape[0]):
                for j in range(v.shape[1]):
                    tgt[i][j] = float(v[i, j])

    put("a", arm["dh_a"]); put("alpha", arm["dh_alpha"]); put("d", arm["dh_d"])
    put("theta0", arm["dh_theta0"]); put("mass", arm["mass"]); put("com", arm["com"])
    put("inertia", arm["inertia"]); put("armature", arm["armature"]); put("fric", arm["fric"])
    put("q_lo", arm["q_lo"]); put("q_hi", arm["q_hi"]); put("qd_max", arm["qd_max"])
    put("taper_a", arm["qd_taper_a"]); put("tau_max", arm["tau_max"])
    s.w_max = float(arm["w_max"])
    put("gravity", arm["gravity"])
    s.flange_d = float(arm["flange_d"])
    put("blade_base", arm["blade_base"]); put("blade_axis", arm["blade_axis"])
    put("blade_normal", arm["blade_normal"])
    s.blade_len = float(arm["blade_len"])
    put("link_radius", arm["link_radius"])
    return s


def problem_struct(pr: dict) -> OrProblem:
    s = OrProblem()
    for f, _ in OrProblem._fields_:
        v = pr[f]
        if f in ("x0", "v0", "g"):
            for i in range(3):
                getattr(s, f)[i] = float(v[i])
        elif f == "sig_linear":
            s.sig_linear = int(v)
        else:
            setattr(s, f, float(v))
    return s


# ----------------------------------------------------------------------------
# thin wrappers
# ----------------------------------------------------------------------------

def time_edges(arm, s0, s1, T_grid, S, mode=0, T_fixed=None, T_cap=None):
    L = lib()
    A = arm_struct(arm)
    s0 = np.ascontiguousarray(s0, np.float32)
    s1 = np.ascontiguousarray(s1, np.float32)
    E = s0.shape[0]
    T_grid = np.ascontiguousarray(T_grid, np.float32)
    Tf = None if T_fixed is None else np.ascontiguousarray(T_fixed, np.float32)
    Tc = None if T_cap is None else np.ascontiguousarray(T_cap, np.float32)
    k = np.zeros(E, np.int32)
    Ts = np.zeros(E, np.float32)
    r3 = np.zeros((E, 3), np.float64)
    ok = np.zeros(E, np.uint8)
    L.or_time_edges(C.byref(A), E, _p(s0), _p(s1), _p(T_grid), len(T_grid), int(S), int(mode),
                    None if Tf is None else _p(Tf), None if Tc is None else _p(Tc),
                    _p(k), _p(Ts), _p(r3), _p(ok))
    return dict(k_star=k, T_star=Ts, rho3=r3, ok=ok)


def time_edges_nary(arm, s0, s1, T_grid, S, eps, max_rounds=8, T_cap=None):
    """Grid scan refined by the N-ary search (N = 32) to a bracket
    (T_lo, T_star] no wider than eps; rho3/ok at the refined T_star."""
    L = lib()
    A = arm_struct(arm)
    s0 = np.ascontiguousarray(s0, np.float32)
    s1 = np.ascontiguousarray(s1, np.float32)
    E = s0.shape[0]
    T_grid = np.ascontiguousarray(T_grid, np.float32)
    Tc = None if T_cap is None else np.ascontiguousarray(T_cap, np.float32)
    k = np.zeros(E, np.int32)
    Ts = np.zeros(E, np.float32)
    Tl = np.zeros(E, np.float32)
    r3 = np.zeros((E, 3), np.float64)
    ok = np.zeros(E, np.uint8)
    rounds = np.zeros(E, np.int32)
    margin = np.zeros(E, np.float64)
    L.or_time_edges_nary(C.byref(A), E, _p(s0), _p(s1), _p(T_grid), len(T_grid), int(S),
                         None if Tc is None else _p(Tc), float(np.float32(eps)), int(max_rounds),
                         _p(k), _p(Ts), _p(Tl), _p(r3), _p(ok), _p(rounds), _p(margin))
    return dict(k_star=k, T_star=Ts, T_lo=Tl, rho3=r3, ok=ok, rounds=rounds, margin=margin)


def controller_torque(arm, state, goal, T, dt, tau_prev=None, rate=None):
    """Eq. (controller) for B instances; returns dict(tau, qdd [B][7] f64,
    flags [B] u8)."""
    A = arm_struct(arm)
    state = np.ascontiguousarray(state, np.float32)
    goal = np.ascontiguousarray(goal, np.float32)
    T = np.ascontiguousarray(T, np.float32)
    B = state.shape[0]
    tp = None if tau_prev is None else np.ascontiguousarray(tau_prev, np.float32)
    rt = None if rate is None else _d(rate)
    tau = np.zeros((B, 7), np.float64)
    qdd = np.zeros((B, 7), np.float64)
    flags = np.zeros(B, np.uint8)
    lib().or_controller_torque(C.byref(A), B, _p(state), _p(goal), _p(T),
                               None if tp is None else _p(tp), float(dt),
                               None if rt is None else _p(rt), _p(tau), _p(qdd), _p(flags))
    return dict(tau=tau, qdd=qdd, flags=flags)


def check_edges(arm, s0, s1, T, S, S_clear, obs, margin):
    """Full-resolution recheck of edges at their own durations; returns
    dict(rho3 [E][3], clearance [E], ok [E])."""
    A = arm_struct(arm)
    s0 = np.ascontiguousarray(s0, np.float32)
    s1 = np.ascontiguousarray(s1, np.float32)
    T = np.ascontiguousarray(T, np.float32)
    E = s0.shape[0]
    ob = np.ascontiguousarray(np.asarray(obs, np.float32).reshape(-1, 4))
    r3 = np.zeros((E, 3), np.float64)
    cl = np.zeros(E, np.float64)
    ok = np.zeros(E, np.uint8)
    lib().or_check_edges(C.byref(A), E, _p(s0), _p(s1), _p(T), int(S), int(S_clear),
                         _p(ob) if len(ob) else None, len(ob), float(margin), _p(r3), _p(cl),
                         _p(ok))
    return dict(rho3=r3, clearance=cl, ok=ok)


class OrDensity(C.Structure):
    _fields_ = [("C", C.c_int), ("w_u", C.c_float), ("pi", C.c_float * 4),
                ("mu", (C.c_float * 9) * 4), ("sd", (C.c_float * 9) * 4)]


def density_struct(theta):
    """OrDensity from dict(C, w_u, pi [C], mu [C][9], sd [C][9])."""
    d = OrDensity()
    d.C = int(theta["C"])
    d.w_u = float(theta["w_u"])
    for c in range(d.C):
        d.pi[c] = float(theta["pi"][c])
        for i in range(9):
            d.mu[c][i] = float(theta["mu"][c][i])
            d.sd[c][i] = float(theta["sd"][c][i])
    return d


def density_z(theta, seed, index, it, problem):
    d = density_struct(theta)
    z = np.zeros(9)
    lib().or_density_z(C.byref(d), seed, index, it, problem, _p(z))
    return z


def sample_goals_density(arm, pr, theta, seed, it, problem, first, n):
    """Goal candidates drawn from p_theta and decoded: (states, T_req, v_rel,
    valid, z)."""
    A = arm_struct(arm)
    Pr = problem_struct(pr)
    d = density_struct(theta)
    st = np.zeros((n, 16))
    Tq = np.zeros(n)
    vr = np.zeros(n)
    valid = np.zeros(n, np.int32)
    zs = np.zeros((n, 9))
    lib().or_sample_goals_density(C.byref(A), C.byref(Pr), C.byref(d), seed, it, problem, first, n,
                                  _p(st), _p(Tq), _p(vr), _p(valid), _p(zs))
    return st, Tq, vr, valid, zs


def sample_chord(arm, seed, it, problem, first, n, vel_frac, q0, goals, w_chord, sigma):
    """Free candidates of the chord sampler; goals [n_goals][16] in candidate
    order."""
    A = arm_struct(arm)
    q0 = _d(q0)
    g = np.ascontiguousarray(np.asarray(goals, np.float64).reshape(-1, 16))
    st = np.zeros((n, 16))
    lib().or_sample_chord(C.byref(A), seed, it, problem, first, n, float(vel_frac), _p(q0),
                          _p(g) if len(g) else None, len(g), float(np.float32(w_chord)),
                          float(sigma), _p(st))
    return st


def rho_batch(arm, s0, s1, T, S):
    A = arm_struct(arm)
    s0 = np.ascontiguousarray(s0, np.float32)
    s1 = np.ascontiguousarray(s1, np.float32)
    T = _d(T)
    out = np.zeros((s0.shape[0], 3), np.float64)
    lib().or_rho_batch(C.byref(A), s0.shape[0], _p(s0), _p(s1), _p(T), int(S), _p(out))
    return out


def torque_dump(arm, s0, s1, T, S):
    A = arm_struct(arm)
    s0 = np.ascontiguousarray(s0, np.float32)
    s1 = np.ascontiguousarray(s1, np.float32)
    T = np.ascontiguousarray(T, np.float32)
    E = s0.shape[0]
    out = np.zeros((E, S, 7), np.float64)
    lib().or_torque_dump(C.byref(A), E, _p(s0), _p(s1), _p(T), int(S), _p(out))
    return out


def torque(arm, q, qd, qdd):
    A = arm_struct(arm)
    q, qd, qdd = _d(q), _d(qd), _d(qdd)
    out = np.zeros(7)
    lib().or_torque(C.byref(A), _p(q), _p(qd), _p(qdd), _p(out))
    return out[: arm["dof"]]


def rnea(arm, q, qd, qdd):
    A = arm_struct(arm)
    q, qd, qdd = _d(q), _d(qd), _d(qdd)
    out = np.zeros(7)
    lib().or_rnea(C.byref(A), _p(q), _p(qd), _p(qdd), _p(out))
    return out[: arm["dof"]]


def friction(psi, qd):
    psi = _d(psi)
    return lib().or_friction(_p(psi), float(qd))


def taper(arm, j, q):
    return lib().or_taper(C.byref(arm_struct(arm)), int(j), float(q))


def cubic(q0, qd0, q1, qd1, T, t):
    q0, qd0, q1, qd1 = _d(q0), _d(qd0), _d(q1), _d(qd1)
    n = q0.size
    s, sd, sdd = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().or_cubic(n, _p(q0), _p(qd0), _p(q1), _p(qd1), float(T), float(t), _p(s), _p(sd), _p(sdd))
    return s, sd, sdd


def knn(tree, queries, k, w_vel, first=1):
    tree = np.ascontiguousarray(tree, np.float32)
    queries = np.ascontiguousarray(queries, np.float32)
    N, B = tree.shape[0], queries.shape[0]
    idx = np.zeros((B, k), np.int32)
    d2 = np.zeros((B, k), np.float64)
    lib().or_knn(_p(tree), N, int(first), _p(queries), B, int(k), float(w_vel), _p(idx), _p(d2))
    return idx, d2


def fk(arm, q):
    A = arm_struct(arm)
    q = _d(np.resize(np.asarray(q, np.float64), 7))
    R = np.zeros((8, 3, 3))
    o = np.zeros((8, 3))
    lib().or_fk(C.byref(A), _p(q), _p(R), _p(o))
    return R, o


def blade(arm, q):
    A = arm_struct(arm)
    q = _d(q)
    b0, b1 = np.zeros(3), np.zeros(3)
    lib().or_blade(C.byref(A), _p(q), _p(b0), _p(b1))
    return b0, b1


def jacobian_point(arm, q, p):
    A = arm_struct(arm)
    q, p = _d(q), _d(p)
    J = np.zeros((6, 7))
    lib().or_jacobian_point(C.byref(A), _p(q), _p(p), _p(J))
    return J


def philox4x32(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, np.uint32))
    k = np.ascontiguousarray(np.asarray(key, np.uint32))
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32(_p(c), _p(k), _p(out))
    return out


def goal_chart(arm, pr, z):
    A = arm_struct(arm)
    P = problem_struct(pr)
    z = _d(z)
    st = np.zeros(16)
    Tq = np.zeros(1)
    vr = np.zeros(1)
    vb = np.zeros(3)
    why = np.zeros(1, np.int32)
    ok = lib().or_goal_chart(C.byref(A), C.byref(P), _p(z), _p(st), _p(Tq), _p(vr), _p(vb),
                             _p(why))
    return bool(ok), st, float(Tq[0]), float(vr[0]), vb


def sample_uniform(arm, seed, it, problem, first_index, n, vel_frac=0.5):
    A = arm_struct(arm)
    out = np.zeros((n, 16))
    lib().or_sample_uniform(C.byref(A), int(seed), int(it), int(problem), int(first_index), int(n),
                            float(vel_frac), _p(out))
    return out


# why a goal draw is undefined (or_goal_chart's reason codes)
CHART_REASONS = ("defined", "speed", "ik", "box", "singular", "taper")


def sample_goals(arm, pr, seed, it, problem, first_index, n, reasons=False):
    """Goal draws decoded by the chart: (states, T_req, v_rel, valid), plus
    the reason code of every draw (CHART_REASONS) when `reasons`."""
    A = arm_struct(arm)
    P = problem_struct(pr)
    st = np.zeros((n, 16))
    Tq = np.zeros(n)
    vr = np.zeros(n)
    valid = np.zeros(n, np.int32)
    why = np.zeros(n, np.int32)
    lib().or_sample_goals(C.byref(A), C.byref(P), int(seed), int(it), int(problem),
                          int(first_index), int(n), _p(st), _p(Tq), _p(vr), _p(valid), _p(why))
    if reasons:
        return st, Tq, vr, valid, why
    return st, Tq, vr, valid


def objective(pr, T, vrel, nu):
    P = problem_struct(pr)
    return lib().or_objective(C.byref(P), float(T), float(vrel), float(nu))


def reach_time(arm, pr, q, t_n, G=256):
    A = arm_struct(arm)
    P = problem_struct(pr)
    q = _d(q)
    Tn = np.zeros(1)
    g = lib().or_reach_time(C.byref(A), C.byref(P), _p(q), float(t_n), int(G), _p(Tn))
    return g, float(Tn[0])


def edge_clearance(arm, s0, s1, T, S, obs):
    A = arm_struct(arm)
    s0 = np.ascontiguousarray(s0, np.float32)
    s1 = np.ascontiguousarray(s1, np.float32)
    obs = np.ascontiguousarray(obs, np.float32)
    return lib().or_edge_clearance(C.byref(A), _p(s0), _p(s1), float(T), int(S), _p(obs),
                                   int(obs.shape[0]))
