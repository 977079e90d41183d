"""FP64 oracle of the gradient of a force objective over a window of time steps
(TEST INFRASTRUCTURE ONLY: only tests, smoke() and the bench's CPU leg use it).

Objective over steps n = 1..N (fixed time steps dt_n, times t_n = t_0 + sum):
    J = sum_n w . F_n  (+ <lu, u_N> + <le, ue_N> when final cotangents are given)
with F_n the pressure force on the body after step n (orc_forces: the BDIM
kernel-weighted integral of the step's pressure, body at t_n). The mean thrust
of a flapping foil over the window is w = (-1/N, 0, 0).

The gradient is the discrete adjoint (reverse sweep over the stored states):
per step the oracle's vector-Jacobian product of the step (orc_step_vjp_fields)
gives the cotangents of the start state and of the body's face fields; the
face fields depend on a body parameter (heave amplitude A, pitch amplitude)
only through the measure, whose parameter derivative is taken here by central
differences of orc_measure (the measured fields are smooth in the parameters;
step h = 1e-6 in FP64 leaves an error near 1e-10, far below every test bar),
and likewise the force's direct dependence on the parameters at fixed
pressure. All arithmetic is the oracle's; this file only sequences it.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import force_dp, forces, grid_from_case, make_body, measure, step_fields_fn, step_vjp_fields


def _fields(g, body, t):
    if body.kind == "none":
        return None
    return measure(g, make_body(body), t)


def _with(body, name, value):
    return dataclasses.replace(body, **{name: value})


def dfields_dparam(g, body, t, name, h=1e-6):
    """Central difference of the measured face fields (mu0, mu1n, V) at time t
    with respect to the body parameter `name` (e.g. heave_amp, pitch_amp).
    The measure cuts mu0 below 1e-5 to 0 (a solid face), so mu0 is a step
    function there: its derivative is 0 on a face cut at the parameter value
    itself and mu0'(d) elsewhere. A face within h of the cut on one side only
    takes the one-sided difference from the side that is not cut, so that no
    step of the cut enters the derivative."""
    v = getattr(body, name)
    fp = _fields(g, _with(body, name, v + h), t)
    fm = _fields(g, _with(body, name, v - h), t)
    out = [(a - b) / (2 * h) for a, b in zip(fp, fm)]
    f0 = _fields(g, body, t)
    m0, mp, mm = f0[0], fp[0], fm[0]
    d = out[0]
    d[m0 == 0.0] = 0.0
    up = (m0 > 0.0) & (mm == 0.0) & (mp > 0.0)
    dn = (m0 > 0.0) & (mp == 0.0) & (mm > 0.0)
    d[up] = (mp[up] - m0[up]) / h
    d[dn] = (m0[dn] - mm[dn]) / h
    return out


def dforce_dparam(g, body, t, P, name, h=1e-6):
    v = getattr(body, name)
    return (forces(g, make_body(_with(body, name, v + h)), t, P)
            - forces(g, make_body(_with(body, name, v - h)), t, P)) / (2 * h)


def window_forward(case, u0, ue0, P0, t0, dts, w, body=None, tol=1e-13):
    """Run the steps with fixed dts; returns (J, states) with states[n] =
    (u, ue, P, t) at the start of step n (and the final state appended)."""
    body = case.body if body is None else body
    g = grid_from_case(case)
    u, ue, P, t = np.array(u0, float), np.array(ue0, float), np.array(P0, float), float(t0)
    states = [(u, ue, P, t)]
    J = 0.0
    for dt in dts:
        u, ue, P = step_fields_fn(g, _fields(g, body, t + dt), dt, u, ue, P, tol=tol)
        t = t + dt
        if body.kind != "none":
            J += float(np.dot(w, forces(g, make_body(body), t, P)[: len(w)]))
        states.append((u, ue, P, t))
    return J, states


def window_gradient(case, u0, ue0, P0, t0, dts, w, params=(), body=None, lu=None, le=None):
    """Discrete adjoint of window_forward. Returns (J, dJ/du0, dJ/due0,
    {param: dJ/dparam})."""
    body = case.body if body is None else body
    g = grid_from_case(case)
    J, states = window_forward(case, u0, ue0, P0, t0, dts, w, body)
    lam = np.zeros_like(states[0][0]) if lu is None else np.array(lu, float)
    lame = np.zeros_like(states[0][1]) if le is None else np.array(le, float)
    grads = {p: 0.0 for p in params}
    for n in range(len(dts) - 1, -1, -1):
        u, ue, P, t = states[n]
        dt = dts[n]
        t1 = t + dt
        Pn = states[n + 1][2]
        if body.kind == "none":
            from . import step_vjp
            lam, lame = step_vjp(g, make_body(body), t, dt, u, ue, P, lam, lame, None)
            continue
        B = make_body(body)
        lP = sum(w[a] * force_dp(g, B, t1, a) for a in range(len(w)))
        fields = _fields(g, body, t1)
        ub, ueb, mu0b, mu1nb, Vb = step_vjp_fields(g, fields, dt, u, ue, P, lam, lame, lP)
        for p in params:
            d0, d1, dV = dfields_dparam(g, body, t1, p)
            grads[p] += float(np.sum(mu0b * d0) + np.sum(mu1nb * d1) + np.sum(Vb * dV))
            grads[p] += float(np.dot(w, dforce_dparam(g, body, t1, Pn, p)[: len(w)]))
        lam, lame = ub, ueb
    return J, lam, lame, grads


# ------------------------------------------------------------- sampled bodies
def window_forward_sampled(case, fields, centre, u0, ue0, P0, dts, w, step_w=None, tol=1e-13, viscous=False):
    """window_forward for a body given by samples: fixed face fields (mu0,
    mu1n, V) of orc_measure_sampled and centre samples (d_cell, n_cell) for
    the force; J = sum_n step_w[n] w . F_n (step_w None = all 1), F_n the
    pressure force plus, with viscous, the viscous force."""
    from . import forces_sampled, forces_viscous_sampled
    g = grid_from_case(case)
    u, ue, P = np.array(u0, float), np.array(ue0, float), np.array(P0, float)
    states = [(u, ue, P)]
    J = 0.0
    for n, dt in enumerate(dts):
        u, ue, P = step_fields_fn(g, fields, dt, u, ue, P, tol=tol)
        sw = 1.0 if step_w is None else float(step_w[n])
        F = forces_sampled(g, centre[0], centre[1], P)
        if viscous:
            F = F + forces_viscous_sampled(g, centre[0], centre[1], u, ue)
        J += sw * float(np.dot(w, F[: len(w)]))
        states.append((u, ue, P))
    return J, states


def window_gradient_sampled(case, fields, centre, dV, u0, ue0, P0, dts, w, step_w=None, viscous=False):
    """Discrete adjoint of window_forward_sampled (viscous: J includes the
    viscous force, linear in the state after each step): returns (J, dJ/du0, dJ/due0,
    dJ/dtheta) for a parameter theta that moves the body velocity only, along
    the face tangent dV (layout of V): dJ/dtheta = sum_n <Vbar_n, dV>, Vbar_n
    the cotangent of the face velocity from step n's vector-Jacobian product."""
    from . import force_dp_sampled, forces_viscous_sampled_vjp
    g = grid_from_case(case)
    J, states = window_forward_sampled(case, fields, centre, u0, ue0, P0, dts, w, step_w, viscous=viscous)
    if viscous:
        gv, gve = forces_viscous_sampled_vjp(g, centre[0], centre[1], w)
    lam = np.zeros_like(states[0][0])
    lame = np.zeros_like(states[0][1])
    dtheta = 0.0
    for n in range(len(dts) - 1, -1, -1):
        u, ue, P = states[n]
        sw = 1.0 if step_w is None else float(step_w[n])
        if viscous:
            # the viscous force of step n reads the state after it
            lam = lam + sw * gv
            lame = lame + sw * gve[: lame.size]
        lP = sw * sum(w[a] * force_dp_sampled(g, centre[0], centre[1], a) for a in range(len(w)))
        ub, ueb, mu0b, mu1nb, Vb = step_vjp_fields(g, fields, dts[n], u, ue, P, lam, lame, lP)
        dtheta += float(np.sum(Vb * dV))
        lam, lame = ub, ueb
    return J, lam, lame, dtheta
