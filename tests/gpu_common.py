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


def run_pair(case, steps, precision="f32", dt=None, gpu_tol=5e-9, oracle_tol=1e-11, smooth_iters=4):
    """Advance the oracle and the GPU path `steps` steps with the oracle's
    time steps; returns (oracle Sim, gpu Sim, per-step GPU stats)."""
    import torch
    u, ue = start_fields(case, precision)
    orc = oracle.Sim(case, tol=oracle_tol, u=u, ue=ue)
    sim = gpu_sim(case, precision, tol=gpu_tol, itmax=60, smooth_iters=smooth_iters)
    tdt = torch.float32 if precision == "f32" else torch.float64
    sim.set_velocity(torch.tensor(orc.u, dtype=tdt).cuda(), torch.tensor(orc.ue, dtype=tdt).cuda())
    stats = []
    for _ in range(steps):
        d = orc.dt if dt is None else dt
        orc.step(d)
        st, rc = sim.mom_step(d, allow_unconverged=True)
        stats.append((st.proj[0].vcycles, st.proj[0].rel_resid, st.proj[1].vcycles, st.proj[1].rel_resid, rc))
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


def oracle_rounding_response(case, steps, amp=1e-7, seed=9):
    """The oracle's own response after `steps` steps (FP64 throughout) to
    (i) an absolute perturbation `amp` of the initial velocity, and (ii) its
    velocity and exit plane rounded to FP32 after every step (the storage
    rounding an FP32 implementation cannot avoid). Returns (u_start, p_start,
    u_store, p_store): relative max-norm change of u and p_err change of p."""
    u, ue = start_fields(case, "f32")
    rng = np.random.default_rng(seed)
    a = oracle.Sim(case, tol=1e-11, u=u, ue=ue)
    b = oracle.Sim(case, tol=1e-11, u=u + amp * rng.uniform(-1, 1, size=u.shape), ue=ue)
    r = oracle.Sim(case, tol=1e-11, u=u, ue=ue)
    for _ in range(steps):
        d = a.dt
        a.step(d)
        b.step(d)
        r.step(d)
        r.u[...] = r.u.astype(np.float32).astype(np.float64)
        r.ue[...] = r.ue.astype(np.float32).astype(np.float64)
    c = oracle.coeffs(a.g, oracle.measure(a.g, a.b, a.t)[0] if case.body.kind != "none" else None)
    un = np.abs(a.u).max()
    return (float(np.abs(a.u - b.u).max() / un), p_err(b.P, a.P, c, case.ndim),
            float(np.abs(a.u - r.u).max() / un), p_err(r.P, a.P, c, case.ndim))
