"""torch.autograd.Function wrappers of the hand-written adjoint (libwl.so).

Argument marshalling only: the forward passes run wl_mom_step /
wl_window_forward and the backward passes wl_step_vjp / wl_window_backward,
whose kernels do all the arithmetic.

    Step.apply(sim, u, dt)                     -> u after one step (dt fixed)
    WindowForce.apply(u0, params, sim, nsteps, ckpt_every, dts, w, tol)
        -> J = sum_n w . F_n over the window, differentiable in the start
           velocity u0 and params = (heave_amp, pitch_amp) of the body.
"""
from __future__ import annotations

import dataclasses

import torch


class Step(torch.autograd.Function):
    """One time step with a fixed dt as a differentiable map u -> u'."""

    @staticmethod
    def forward(ctx, sim, u, dt, tol=1e-7):
        sim.set_velocity(u.detach().contiguous())
        u0, ue0 = sim.get_velocity()
        t0, _ = sim.get_time()
        sim.mom_step(float(dt))
        u1, _ = sim.get_velocity()
        ctx.sim, ctx.t0, ctx.dt, ctx.tol = sim, t0, float(dt), tol
        ctx.save_for_backward(u0)
        ctx.ue0 = ue0
        return u1

    @staticmethod
    def backward(ctx, gu):
        (u0,) = ctx.saved_tensors
        ub, _, _ = ctx.sim.step_vjp(ctx.t0, ctx.dt, u0, ctx.ue0, None, gu.contiguous().to(u0.dtype), None, None,
                                    tol=ctx.tol)
        return None, ub, None, None


class WindowForce(torch.autograd.Function):
    """J = sum_n w . F_n over nsteps steps from the start velocity u0, with the
    body's heave and pitch amplitudes params[0], params[1]; the backward pass is
    the checkpointed adjoint sweep (checkpoint every ckpt_every steps)."""

    @staticmethod
    def forward(ctx, u0, params, sim, nsteps, ckpt_every=20, dts=None, w=(-1.0, 0.0, 0.0), tol=1e-7):
        p = params.detach().double().cpu().tolist()
        sim.set_body(dataclasses.replace(sim.body, heave_amp=p[0], pitch_amp=p[1]))
        sim.set_velocity(u0.detach().contiguous())
        J, taken = sim.window_forward(nsteps, ckpt_every, dts, w)
        ctx.sim, ctx.tol = sim, tol
        ctx.dts = taken
        ctx.pdtype, ctx.pdevice = params.dtype, params.device
        return torch.tensor(J, dtype=torch.float64, device=u0.device)

    @staticmethod
    def backward(ctx, gJ):
        du0, _, dp = ctx.sim.window_backward(float(gJ), None, None, ctx.tol, params=True)
        gp = torch.tensor(dp, dtype=ctx.pdtype, device=ctx.pdevice)
        return du0, gp, None, None, None, None, None, None
