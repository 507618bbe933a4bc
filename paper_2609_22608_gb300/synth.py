"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module draws inputs only; it holds none of the planner's arithmetic
(no dynamics, no cubic, no feasibility ratios, no chart decoding).  Every
array it returns is already rounded to float32, so that the GPU path and the
FP64 oracle start from bit-identical values.

Workload shapes follow the paper's setting (Sec. III problem statement, Sec. V
methodology): a 7-DOF revolute arm with an FR3-like modified-DH topology,
per-joint torque / velocity / power limits (Def. 1, W_max = 120 W in Sec. IV-D),
ballistic tosses sweeping the workspace from three launch azimuths (Sec. V-A),
and an arrival window under one second (Sec. III).  The paper's own toss
recordings and FR3 identification are not available, so everything here is
synthetic; the recipe is listed in the project's design notes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

F32 = np.float32
DOF = 7
STATE_STRIDE = 16  # q[7], pad, qd[7], pad  (64 bytes per state)

# FR3-like link twists (modified DH, Craig): alpha_{i-1} for joints 1..7.
FR3_ALPHA = (0.0, -math.pi / 2, math.pi / 2, math.pi / 2, -math.pi / 2, math.pi / 2, math.pi / 2)


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(F32)


def make_arm(seed: int = 0) -> dict:
    """A seeded synthetic 7-DOF arm (all fields float32).

    Geometry is FR3-like (link offsets jittered around a Franka-style chain),
    masses U(0.5, 4) kg, COM offsets U(-0.1, 0.1) m, diagonal inertias
    U(1e-3, 5e-2) kg m^2, armature U(0.01, 0.3) kg m^2, sigmoid friction
    psi1 U(0.05, 0.6), psi2 U(5, 60), psi3 U(-0.1, 0.1), torque limits
    U(60, 87) N m on joints 1-4 and U(12, 30) N m on joints 5-7, velocity
    limits U(2.0, 2.9) rad/s, joint boxes +-U(1.5, 2.9) rad, W_max = 120 W.
    """
    rng = np.random.default_rng([0xA53, seed])
    U = rng.uniform
    a = [0.0, 0.0, 0.0, U(0.07, 0.095), -U(0.07, 0.095), 0.0, U(0.075, 0.10)]
    d = [U(0.30, 0.36), 0.0, U(0.29, 0.34), 0.0, U(0.35, 0.40), 0.0, 0.0]
    mass = U(0.5, 4.0, DOF)
    # distal links of a real arm are lighter; keep the range but scale the wrist
    mass[4:] *= 0.5
    com = U(-0.1, 0.1, (DOF, 3))
    inertia = U(1e-3, 5e-2, (DOF, 3))
    armature = U(0.01, 0.3, DOF)
    fric = np.stack([U(0.05, 0.6, DOF), U(5.0, 60.0, DOF), U(-0.1, 0.1, DOF)], axis=1)
    tau_max = np.concatenate([U(60.0, 87.0, 4), U(12.0, 30.0, 3)])
    qd_max = U(2.0, 2.9, DOF)
    q_hi = U(1.5, 2.9, DOF)
    q_lo = -U(1.5, 2.9, DOF)
    arm = dict(
        dof=DOF,
        dh_a=_f32(a), dh_alpha=_f32(FR3_ALPHA), dh_d=_f32(d), dh_theta0=_f32(np.zeros(DOF)),
        mass=_f32(mass), com=_f32(com), inertia=_f32(inertia),
        armature=_f32(armature), fric=_f32(fric),
        q_lo=_f32(q_lo), q_hi=_f32(q_hi), qd_max=_f32(qd_max),
        qd_taper_a=_f32(np.full(DOF, 10.0)),
        tau_max=_f32(tau_max), w_max=F32(120.0),
        gravity=_f32([0.0, 0.0, -9.81]),
        # end-effector frame = frame 7 shifted by flange_d along z7; the blade
        # edge starts at blade_base and runs blade_len along blade_axis (EE frame)
        flange_d=F32(U(0.10, 0.12)),
        blade_base=_f32([0.0, 0.0, 0.05]),
        blade_axis=_f32([1.0, 0.0, 0.0]),
        blade_normal=_f32([0.0, 1.0, 0.0]),
        blade_len=F32(0.30),
        link_radius=_f32([0.09, 0.09, 0.08, 0.08, 0.07, 0.06, 0.05]),
    )
    return arm


def arm_with_dof(arm: dict, dof: int) -> dict:
    """Copy of `arm` that only uses its first `dof` joints (for 1-3 link pins)."""
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in arm.items()}
    out["dof"] = int(dof)
    return out


def duration_grid(K: int, T_lo: float = 0.05, T_hi: float = 2.0) -> np.ndarray:
    """Log-spaced duration grid T_k = T_lo (T_hi/T_lo)^(k/(K-1)), built in FP64,
    rounded to FP32 (the N-ary slots of Sec. IV-D laid out on one log grid)."""
    if K == 1:
        return _f32([T_lo])
    k = np.arange(K, dtype=np.float64)
    return (T_lo * (T_hi / T_lo) ** (k / (K - 1))).astype(F32)


def pack_states(q: np.ndarray, qd: np.ndarray) -> np.ndarray:
    """[n][7] + [n][7] -> [n][16] float32 rows (q, pad, qd, pad)."""
    q = np.asarray(q, np.float64)
    qd = np.asarray(qd, np.float64)
    n = q.shape[0]
    out = np.zeros((n, STATE_STRIDE), F32)
    out[:, 0:DOF] = q
    out[:, 8:8 + DOF] = qd
    return out


def random_states(arm: dict, n: int, seed: int, vel_frac: float = 0.5) -> np.ndarray:
    """q ~ U(joint box), qd ~ U(+-vel_frac * qd_max) as packed [n][16] f32."""
    rng = np.random.default_rng([0x57A7E, seed])
    lo = arm["q_lo"].astype(np.float64)
    hi = arm["q_hi"].astype(np.float64)
    q = rng.uniform(lo, hi, (n, DOF))
    vm = vel_frac * arm["qd_max"].astype(np.float64)
    qd = rng.uniform(-vm, vm, (n, DOF))
    return pack_states(q, qd)


def random_edges(arm: dict, E: int, seed: int, vel_frac: float = 0.5):
    """E independent edge boundary pairs (s0, s1), each [E][16] f32."""
    s0 = random_states(arm, E, 2 * seed, vel_frac)
    s1 = random_states(arm, E, 2 * seed + 1, vel_frac)
    return s0, s1


def random_tree(arm: dict, N: int, seed: int, root: np.ndarray | None = None,
                t_max: float | None = None):
    """Synthetic tree: random states, parent uniform among earlier nodes,
    t = t_parent + U(0.05, 0.3).  Node 0 is the root with t = 0.

    With `t_max` (a planning tree: every node was attached no later than
    t_best <= t_fall), the parent is uniform among the earlier nodes with
    t <= t_max - 0.05 and the increment is U(0.05, min(0.3, t_max - t_parent)),
    so every node's time lies in [0, t_max]."""
    rng = np.random.default_rng([0x7EE, seed])
    states = random_states(arm, N, 1000 + seed)
    if root is not None:
        states[0] = root
    parent = np.full(N, -1, np.int32)
    t = np.zeros(N, np.float64)
    if t_max is None:
        for i in range(1, N):
            p = int(rng.integers(0, i))
            parent[i] = p
            t[i] = t[p] + rng.uniform(0.05, 0.3)
        return states, parent, t.astype(F32)
    t_max = float(t_max)
    if t_max < 0.1:
        raise ValueError("t_max must leave room for a 0.05 s increment")
    open_nodes = [0]                      # nodes that can still take a child
    for i in range(1, N):
        p = open_nodes[int(rng.integers(0, len(open_nodes)))]
        parent[i] = p
        t[i] = t[p] + rng.uniform(0.05, min(0.3, t_max - t[p]))
        if t[i] <= t_max - 0.05:
            open_nodes.append(i)
    return states, parent, t.astype(F32)


@dataclass
class Toss:
    x0: np.ndarray     # [3] f32, position at measurement time
    v0: np.ndarray     # [3] f32
    t_enter: float
    t_fall: float


# the object counts as within the arm's reach (Sec. III: the window
# [t_enter, t_fall] is when it is) while it is above the base plane and no
# farther than REACH from the shoulder, the common origin of frames 1 and 2
# at height d_1
REACH = 0.7
MIN_WINDOW = 0.1


def reach_window(arm: dict, x0, v0, t_lo: float, t_hi: float, reach: float = REACH):
    """First and last time in [t_lo, t_hi] (1 ms steps) at which the flight
    x0 + v0 t + g t^2 / 2 is within `reach` of the shoulder and above z = 0;
    None if it never is.  The window is taken as one interval."""
    g = arm["gravity"].astype(np.float64)
    ts = np.linspace(t_lo, t_hi, int(round((t_hi - t_lo) / 1e-3)) + 1)
    x = np.asarray(x0, np.float64)[None] + np.asarray(v0, np.float64)[None] * ts[:, None] \
        + 0.5 * g[None] * ts[:, None] ** 2
    sh = np.array([0.0, 0.0, float(arm["dh_d"][0])])
    inside = (np.linalg.norm(x - sh, axis=1) <= reach) & (x[:, 2] > 0.0)
    if not inside.any():
        return None
    i = np.nonzero(inside)[0]
    return float(ts[i[0]]), float(ts[i[-1]])


def random_toss(arm: dict, seed: int, t_enter: float = 0.2, t_fall: float = 0.9,
                target: np.ndarray | None = None, reach: float | None = REACH) -> Toss:
    """A ballistic toss that crosses the arm's workspace inside the window.

    Launch from radius U(1.2, 1.6) m at azimuth in {-30, 0, 30} deg (Sec. V-A)
    and height 1.0 m, with speed ~ N(3, 0.5) m/s aimed so that the flight
    passes `target` (default: a point 0.45-0.65 m from the base at height
    0.35-0.6 m) at a time inside [t_enter + 0.1, t_fall - 0.1].

    With `reach` (default REACH), the toss's window is the part of
    [t_enter, t_fall] during which the object is within the arm's reach
    (reach_window), as the problem statement defines the window; tosses whose
    window is shorter than MIN_WINDOW are redrawn.  reach=None keeps
    [t_enter, t_fall] as given.
    """
    rng = np.random.default_rng([0x7055, seed])
    g = arm["gravity"].astype(np.float64)
    for _ in range(1000):
        r0 = rng.uniform(1.2, 1.6)
        az = math.radians(rng.choice([-30.0, 0.0, 30.0]))
        x0 = np.array([r0 * math.cos(az), r0 * math.sin(az), 1.0])
        if target is None:
            rr = rng.uniform(0.45, 0.65)
            ta = az + rng.uniform(-0.5, 0.5)
            tgt = np.array([rr * math.cos(ta), rr * math.sin(ta), rng.uniform(0.35, 0.6)])
        else:
            tgt = np.asarray(target, np.float64)
        speed = rng.normal(3.0, 0.5)
        # find the crossing time whose launch speed matches `speed`
        ts = np.linspace(t_enter + 0.1, t_fall - 0.1, 400)
        v = (tgt[None, :] - x0[None, :] - 0.5 * g[None, :] * ts[:, None] ** 2) / ts[:, None]
        sp = np.linalg.norm(v, axis=1)
        j = int(np.argmin(np.abs(sp - speed)))
        if abs(sp[j] - speed) < 0.05:
            x0f, v0f = _f32(x0), _f32(v[j])
            if reach is None:
                return Toss(x0f, v0f, float(t_enter), float(t_fall))
            win = reach_window(arm, x0f, v0f, t_enter, t_fall, reach)
            if win is not None and win[1] - win[0] >= MIN_WINDOW:
                return Toss(x0f, v0f, float(F32(win[0])), float(F32(win[1])))
    raise RuntimeError("no toss found")


def uniform_candidates(arm: dict, B: int, seed: int, vel_frac: float = 0.5) -> np.ndarray:
    """Host-drawn free candidates (q uniform in the box, qd in +-vel_frac*qd_max)."""
    return random_states(arm, B, 77_000 + seed, vel_frac)


def obstacles(n: int, seed: int) -> np.ndarray:
    """n obstacle spheres [n][4] = (centre xyz, radius), r ~ U(0.05, 0.15) m,
    centres in the arm's front workspace."""
    rng = np.random.default_rng([0x0B5, seed])
    r = rng.uniform(0.05, 0.15, n)
    rad = rng.uniform(0.35, 0.8, n)
    az = rng.uniform(-1.2, 1.2, n)
    z = rng.uniform(0.1, 0.9, n)
    c = np.stack([rad * np.cos(az), rad * np.sin(az), z, r], axis=1)
    return _f32(c)


def make_problem(toss: Toss, root: np.ndarray | None = None, t_offset: float = 0.0,
                 sigma_linear: tuple[float, float] | None = None, v_tip: float = 3.0) -> dict:
    """Problem constants of one planning cycle.

    Scoring constants are the paper's (Sec. V: w_v = 0.20, v_target = 9 m/s,
    w_p = w_r = 8, w_x = 1, r = 9 cm, nu0 = 0.90, lambda = 1.2; simulation
    covariance sigma_p = 4.8 mm, sigma_v = 18.6 mm/s, sigma_a = 0) and the
    manifold thresholds of Def. 2 (a_min = 0.94, v_min = 3 m/s).  V_tip is not
    given in the paper (3 m/s here).  `sigma_linear` = (a, b) switches the
    uncertainty to sigma(t) = a + b t (the anytime stress workload).
    """
    pr = dict(
        x0=np.asarray(toss.x0, np.float64), v0=np.asarray(toss.v0, np.float64),
        t_enter=float(toss.t_enter), t_fall=float(toss.t_fall), t_offset=float(t_offset),
        sig_p=4.8e-3, sig_v=18.6e-3, sig_a=0.0,
        sig_linear=0, sig_lin_a=0.0, sig_lin_b=0.0,
        a_min=0.94, v_min=3.0,
        w_v=0.20, v_target=9.0, w_p=8.0, w_r=8.0, w_x=1.0, r_catch=0.09, nu0=0.90, lam=1.2,
        v_tip=float(v_tip), g=np.array([0.0, 0.0, -9.81]),
    )
    if sigma_linear is not None:
        pr.update(sig_linear=1, sig_lin_a=float(sigma_linear[0]), sig_lin_b=float(sigma_linear[1]))
    # every float goes through float32 so both sides read identical values
    for k, v in list(pr.items()):
        if k == "sig_linear":
            continue
        pr[k] = np.asarray(v, np.float64).astype(F32).astype(np.float64) if isinstance(v, np.ndarray) \
            else float(F32(v))
    pr["root"] = None if root is None else np.asarray(root, F32)
    return pr
