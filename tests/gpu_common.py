"""Helpers shared by the GPU parity tests: run the CUDA path (through the C ABI
binding) and the FP64 oracle on the same seeded inputs."""
import numpy as np

import oracle
import synth


def gpu_sim(case, precision="f32", **kw):
    from paper_2407_16032_b300 import sim_from_case
    return sim_from_case(case, precision, **kw)


def start_fields(case, precision):
    u, ue = synth.initial_velocity(case)
    if precision == "f32":
        u = u.astype(np.float32).astype(np.float64)
        ue = ue.astype(np.float32).astype(np.float64)
    return u, ue


def run_pair(case, steps, precision="f32", dt=None, gpu_tol=5e-9, oracle_tol=1e-11, smooth_iters=4, on_step=None,
             setup=None):
    """Advance the oracle and the GPU path `steps` steps with the oracle's
    time steps; returns (oracle Sim, gpu Sim, per-step GPU stats). on_step(k,
    orc, sim), if given, runs after step k (1-based) of both; setup(sim), if
    given, runs on the new GPU sim before its first step."""
    import torch
    u, ue = start_fields(case, precision)
    orc = oracle.Sim(case, tol=oracle_tol, u=u, ue=ue)
    sim = gpu_sim(case, precision, tol=gpu_tol, itmax=60, smooth_iters=smooth_iters)
    if setup:
        setup(sim)
    tdt = torch.float32 if precision == "f32" else torch.float64
    sim.set_velocity(torch.tensor(orc.u, dtype=tdt).cuda(), torch.tensor(orc.ue, dtype=tdt).cuda())
    stats = []
    orc.dts = []
    for _ in range(steps):
        d = orc.dt if dt is None else dt
        orc.dts.append(d)
        orc.step(d)
        st, rc = sim.mom_step(d, allow_unconverged=True)
        stats.append((st.proj[0].vcycles, st.proj[0].rel_resid, st.proj[1].vcycles, st.proj[1].rel_resid, rc))
        if on_step:
            on_step(len(stats), orc, sim)
    return orc, sim, stats


def rel_max(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def gpu_fields(sim):
    u, ue = sim.get_velocity()
    p = sim.get_pressure()
    return u.double().cpu().numpy(), (ue.double().cpu().numpy() if ue is not None else None), p.cpu().numpy()


def well_determined(c, ndim):
    """Cells whose 2n faces all have Poisson coefficient >= 1/2 (the pressure of
    cells with nearly solid faces is not determined to working precision)."""
    m = np.ones(c.shape[1:], bool)
    for a in range(ndim):
        ax = ndim - 1 - a
        m &= (c[a] >= 0.5) & (np.roll(c[a], -1, axis=ax) >= 0.5)
    return m


def p_err(p, P, c, ndim):
    """Relative max error of the mean-free pressure on well-determined cells."""
    m = well_determined(c, ndim)
    pm, Pm = p - p[m].mean(), P - P[m].mean()
    return float(np.abs(pm - Pm)[m].max() / np.abs(Pm[m]).max())


def near_body_p_err(p, P, c, ndim):
    """Relative max error of the mean-free pressure on the cells that p_err
    leaves out: active cells (a face with c > 0) with a face of c < 1/2, the
    band where the pressure force is integrated. Means and scale are those of
    the well-determined cells, as in p_err."""
    m = well_determined(c, ndim)
    act = np.zeros(c.shape[1:], bool)
    for a in range(ndim):
        ax = ndim - 1 - a
        act |= (c[a] > 0) | (np.roll(c[a], -1, axis=ax) > 0)
    band = act & ~m
    if not band.any():
        return 0.0
    pm, Pm = p - p[m].mean(), P - P[m].mean()
    return float(np.abs(pm - Pm)[band].max() / np.abs(Pm[m]).max())


def flux_err(p, P, c, ndim):
    """Relative max error of the projection face fluxes c_a (p[I] - p[I - e_a])."""
    e, ref = 0.0, 0.0
    for a in range(ndim):
        ax = ndim - 1 - a
        fg = c[a] * (p - np.roll(p, 1, axis=ax))
        fo = c[a] * (P - np.roll(P, 1, axis=ax))
        e = max(e, float(np.abs(fg - fo).max()))
        ref = max(ref, float(np.abs(fo).max()))
    return e / ref


def oracle_start_response(case, ref, amp=1e-7, seed=9):
    """The oracle's own response to an absolute perturbation `amp` of the
    initial velocity (FP64 both runs): a second oracle run from the perturbed
    start, with the time steps and tolerance of the reference run `ref` (an
    oracle Sim that ran from the unperturbed start), compared after the same
    number of steps. This is the amplification that an FP32 implementation's
    rounding meets on this input. Returns (u change, p change): relative
    max-norm of u and p_err of p."""
    u, ue = start_fields(case, "f32")
    rng = np.random.default_rng(seed)
    b = oracle.Sim(case, tol=ref.S.tol, u=u + amp * rng.uniform(-1, 1, size=u.shape), ue=ue)
    for d in ref.dts:
        b.step(d)
    c = oracle.coeffs(ref.g, oracle.measure(ref.g, ref.b, ref.t)[0] if case.body.kind != "none" else None)
    return float(np.abs(ref.u - b.u).max() / np.abs(ref.u).max()), p_err(b.P, ref.P, c, case.ndim)


def calibrated_bars(case, ref, floor=1e-5):
    """Parity bars (u, p) for inputs whose discrete step amplifies rounding:
    five times the oracle's own response to a 1e-7 perturbation of the start
    (oracle_start_response), and at least `floor`. Computed from the oracle
    only."""
    su, sp = oracle_start_response(case, ref)
    return max(floor, 5.0 * su), max(floor, 5.0 * sp)


def report(name, **vals):
    """Append the measured errors of a parity case to the JSON-lines file named
    by WL_PARITY_REPORT (nothing when it is unset)."""
    import json
    import os
    path = os.environ.get("WL_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"case": name, **{k: float(v) for k, v in vals.items()}}) + "\n")
