"""Spin-rate control of the flow past a circle (Sec. 6.1, the optimised control
cylinders): a fixed circle of diameter D and a small control circle that
spins with surface speed xi U, joined by the union of their distance
functions and handed to the library as samples (WL_BODY_USER_FACE_FIELDS).

The objective is the scaled propulsive power at time t* = t U / D,
    C_P = F U / (rho d c^3),  c = xi U,  d = d_D D  (rho = 1),
with F the net thrust, read here as minus the x component of the total
force on the bodies (wl_forces + wl_forces_viscous; viscous = False keeps the
pressure part alone) after the last step; the half domain (a symmetry plane at y = 0)
carries half the system, which scales C_P but not its maximiser. dC_P/dxi
comes from the window adjoint: the geometry does not depend on xi and the
body velocity is linear in it, so dF/dxi is the gradient along the control
circle's velocity per unit xi (wl_set_body_velocity_tangent), and
    dC_P/dxi = (dJ/dxi) / (d xi^3 U^2) - 3 C_P / xi,  J = -F_x.
The time steps are the adaptive CFL steps of a plain run until it passes t*,
all scaled by one factor (at most 1, so within the CFL bound) to land on t*,
then held fixed for the window and its gradient. (A last step shortened to
land on t* can be tiny, and the pressure of a tiny step carries the start
velocity's residual divergence divided by that step.)
"""
from __future__ import annotations

import math
import os
import sys
from dataclasses import dataclass, field

import numpy as np

from .davidon import davidon_maximize
from .wl import sim_from_case

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _synth():
    if _ROOT not in sys.path:
        sys.path.insert(0, _ROOT)
    import synth
    return synth


@dataclass
class SpinControl:
    D: int = 96
    Re: float = 500.0
    d_D: float = 0.15
    g_D: float = 0.05
    t_star: float = 2.0
    precision: str = "f32"
    tol: float = 1e-6           # forward Poisson tolerance
    adj_tol: float = 1e-6       # adjoint Poisson tolerance
    ckpt_every: int = 32
    viscous: bool = True        # F includes the viscous force
    seed: int = 0
    log: list = field(default_factory=list)

    def _setup(self, xi):
        synth = _synth()
        case, shape, tangent = synth.spinning_cylinders(self.D, self.Re, self.d_D, self.g_D, xi)
        case = case.with_(seed=self.seed)
        npt = np.float32 if self.precision == "f32" else np.float64
        sim = sim_from_case(case, self.precision, tol=self.tol, itmax=64)
        sim.set_body_fields(*synth.sample_body(shape, 2, case.n, npt))
        sim.set_body_velocity_tangent(synth.sample_body(tangent, 2, case.n, npt)[2])
        u0, ue0 = synth.initial_velocity(case)
        T = sim.torch
        u0 = T.tensor(u0, dtype=sim.dtype, device=sim.device)
        ue0 = T.tensor(ue0, dtype=sim.dtype, device=sim.device)
        return case, sim, u0, ue0

    def _restart(self, sim, case, u0, ue0):
        sim.set_velocity(u0, ue0)
        sim.set_pressure(sim.torch.zeros(sim._shape(), dtype=sim.torch.float64, device=sim.device))
        sim.set_time(0.0, case.dt0)

    def cp(self, xi, grad=True, dts=None):
        """C_P at t* for spin xi and, with grad, dC_P/dxi (else None).
        Returns (C_P, dC_P/dxi, info dict with J, steps, dts)."""
        case, sim, u0, ue0 = self._setup(xi)
        U = case.U[0]
        t_end = self.t_star * self.D / U
        hist = None
        if dts is None:
            dts, hist = [], []
            self._restart(sim, case, u0, ue0)
            t = 0.0
            while t < t_end - 1e-9:
                st, _ = sim.mom_step()
                dts.append(st.dt)
                t += st.dt
                hist.append((t, -sim.forces()[0], -sim.forces_viscous()[0]))
            dts = [d * t_end / t for d in dts]
        self._restart(sim, case, u0, ue0)
        n = len(dts)
        step_w = np.zeros(n)
        step_w[-1] = 1.0
        J, _ = sim.window_forward(n, self.ckpt_every, dts, (-1.0, 0.0), step_w=step_w, viscous=self.viscous)
        d = self.d_D * self.D
        scale = 1.0 / (d * xi ** 3 * U ** 2)
        Cp = J * scale
        dCp = None
        if grad:
            _, _, dp = sim.window_backward(1.0, tol=self.adj_tol)
            dCp = dp[0] * scale - 3.0 * Cp / xi
        sim.close()
        info = {"J": J, "steps": n, "dts": dts, "thrust_history": hist}
        self.log.append((xi, Cp, dCp, n))
        return Cp, dCp, info

    def optimize(self, a=3.0, b=8.0, xtol=0.02, maxit=8):
        """Davidon's search for the spin that maximises C_P on [a, b]."""
        return davidon_maximize(lambda x: self.cp(x)[:2], a, b, xtol=xtol, maxit=maxit)
