"""Gradient refinement of a rendezvous node -- TEST INFRASTRUCTURE ONLY.

The paper closes by noting that its checks and chart decoder are smooth in
the trajectory parameters and that gradient-based refinement of tree nodes
is a direct next step; it gives no objective, variables or step rule.
Reading used here and in the library's kernel (restated in the design
notes):
  * variables: the chart parameters z in [0, 1]^9 of a rendezvous node n
    with parent p; the node is phi(z) = (q_g, qd_g, T_req(z)) and its edge
    from p runs for T_p = T_req(z) - t(p) (single precision, as in the
    round);
  * objective: F(z) = J of Eq. (objective) at the node's arrival time
    t(p) + T_p, with its relative speed |v_rel(z)| and nu = max(nu(p),
    rho_v of the edge at T_p), where phi(z) is defined, T_p > 0 and the
    edge passes Def. "Feasibility Check" at T_p and the clearance; -inf
    elsewhere;
  * gradient: central differences of the same J (without the feasibility
    condition) with step h in every coordinate; the angle coordinates
    (z2, z3, z4) wrap modulo 1, the others are clamped to [0, 1] and the
    difference is divided by the clamped span; a coordinate where either
    side is undefined gets 0;
  * step: z' = fold(z + eta_t g / |g|) with eta_t = eta0 2^-t, t = 0..I-1
    (fold: wrap the angle coordinates, clamp the others); z' replaces z when
    F(z') > F(z) (so F never decreases and the result passes the check);
    a zero gradient ends the iterations;
  * defaults: I = 8, eta0 = 0.05, h = 1e-3.
Every step follows this order; the evaluations call the FP64 oracle's
goal chart, fixed-duration check, clearance and objective.
"""
from __future__ import annotations

import numpy as np

import oracle as O

F32 = np.float32
ANGLE = (2, 3, 4)
ITERS, ETA0, H = 8, 0.05, 1e-3


def fold(z):
    """Wrap the angle coordinates, clamp the others to [0, 1]."""
    z = np.array(z, np.float64)
    for i in range(9):
        z[i] = z[i] % 1.0 if i in ANGLE else min(max(z[i], 0.0), 1.0)
    return z


def node_eval(arm, pr, z, parent_state, t_parent, nu_parent, S, obstacles=None, margin=0.02,
              S_clear=8):
    """(J without the feasibility condition, feasible, details) of phi(z)
    attached to the parent; J is -inf where phi is undefined or T_p <= 0."""
    ok, st, Treq, vrel, vb = O.goal_chart(arm, pr, z)
    if not ok:
        return -np.inf, False, None
    Tp = F32(F32(Treq) - F32(t_parent))
    if not Tp > 0:
        return -np.inf, False, None
    s0 = np.asarray(parent_state, F32)[None]
    s1 = st.astype(F32)[None]
    r = O.time_edges(arm, s0, s1, np.array([1.0], F32), S, mode=1,
                     T_fixed=np.array([Tp], F32))
    rho3 = r["rho3"][0]
    nu = max(float(nu_parent), float(rho3[2]))
    T_node = float(F32(F32(t_parent) + Tp))
    J = O.objective(pr, T_node, float(F32(vrel)), nu)
    feasible = bool(r["ok"][0] == 1)
    clear = np.inf
    if feasible and obstacles is not None and len(obstacles):
        clear = O.edge_clearance(arm, s0[0], s1[0], float(Tp), S_clear, obstacles)
        feasible = clear >= margin
    return J, feasible, dict(state=s1[0], T_p=float(Tp), T_node=T_node, rho3=rho3, nu=nu,
                             vrel=vrel, clearance=clear)


def fd_gradient(J_of, z, h=H):
    """Central differences of J_of (a callable on z) in every coordinate."""
    g = np.zeros(9)
    for i in range(9):
        zp, zm = np.array(z, np.float64), np.array(z, np.float64)
        if i in ANGLE:
            zp[i] = (z[i] + h) % 1.0
            zm[i] = (z[i] - h) % 1.0
            d = 2.0 * h
        else:
            zp[i] = min(z[i] + h, 1.0)
            zm[i] = max(z[i] - h, 0.0)
            d = zp[i] - zm[i]
        Jp, Jm = J_of(zp), J_of(zm)
        g[i] = (Jp - Jm) / d if (np.isfinite(Jp) and np.isfinite(Jm) and d > 0) else 0.0
    return g


def refine(F_of, J_of, z0, iters=ITERS, eta0=ETA0, h=H):
    """Projected, normalised gradient ascent with halving steps and
    acceptance on improvement.  F_of: the objective with the feasibility
    condition (-inf where infeasible); J_of: the same J without it (the
    gradient's function).  Returns (z, F, accepted steps)."""
    z = fold(z0)
    F = F_of(z)
    acc = 0
    for t in range(iters):
        g = fd_gradient(J_of, z, h)
        n = float(np.sqrt(np.sum(g * g)))
        if not n > 0:
            break
        zn = fold(z + (eta0 * 0.5 ** t) * g / n)
        Fn = F_of(zn)
        if Fn > F:
            z, F = zn, Fn
            acc += 1
    return z, F, acc


def refine_node(arm, pr, z0, parent_state, t_parent, nu_parent, S, obstacles=None, margin=0.02,
                S_clear=8, iters=ITERS, eta0=ETA0, h=H):
    """refine() on the objective of a rendezvous node with its parent."""
    def J_of(z):
        return node_eval(arm, pr, z, parent_state, t_parent, nu_parent, S, obstacles, margin,
                         S_clear)[0]

    def F_of(z):
        J, feas, _ = node_eval(arm, pr, z, parent_state, t_parent, nu_parent, S, obstacles,
                               margin, S_clear)
        return J if feas else -np.inf

    z, F, acc = refine(F_of, J_of, z0, iters, eta0, h)
    _, feas, det = node_eval(arm, pr, z, parent_state, t_parent, nu_parent, S, obstacles, margin,
                             S_clear)
    return dict(z=z, J=F, accepted=acc, feasible=feas, detail=det)
