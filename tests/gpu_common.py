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


def run_pair(case, steps, precision="f32", dt=None, gpu_tol=1e-9, oracle_tol=1e-11, smooth_iters=4):
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
