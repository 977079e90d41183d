"""GPU parity of the checkpointed window adjoint (wl_window_forward /
wl_window_backward, and the torch.autograd.Function over them) against the
FP64 oracle's window gradient (oracle/adjoint.py, pinned by central
differences of complete forward runs), and against central differences of the
GPU's own forward window with the parameter step of the flapping-foil study
(1e-3).

Objective: the mean thrust J = -(1/N) sum_n F_x,n of a heaving and pitching
ellipse over N steps; gradients with respect to the start velocity and to the
heave and pitch amplitudes.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import adjoint as oadj

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_16032_b300 import build
    build.build()


def _foil(n=(96, 64), chord=24.0):
    body = synth.Body("ellipse", (30.3, 31.7, 0.0), 0.0, (chord / 2, 0.06 * chord), heave_amp=4.0,
                      pitch_amp=math.radians(15.0), omega=2 * math.pi * 0.3 / chord)
    case = synth.Case("foil", 2, (n[0], n[1], 1), (False, False, False), True, (1.0, 0.0, 0.0), chord / 1000.0, body)
    u0 = synth.random_field(41, 2, (n[0], n[1], 1), amp=0.02, offset=(1.0, 0.0))
    u0[0][:, 0] = 1.0
    u0[1][0, :] = 0.0
    ue0 = np.ones(n[1])
    return case, u0, ue0


DTS = [0.3, 0.35, 0.3, 0.32, 0.3, 0.31, 0.3]
T0 = 0.5


def _gpu(case, prec, u0, ue0, tol):
    import torch
    from paper_2407_16032_b300 import sim_from_case
    sim = sim_from_case(case, prec, tol=tol, itmax=80)
    dt = torch.float32 if prec == "f32" else torch.float64
    sim.set_velocity(torch.tensor(u0, dtype=dt, device="cuda"), torch.tensor(ue0, dtype=dt, device="cuda"))
    sim.set_time(T0, DTS[0])
    return sim


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_window_gradient_matches_oracle(prec):
    case, u0, ue0 = _foil()
    if prec == "f32":
        u0 = u0.astype(np.float32).astype(np.float64)
    w = (-1.0 / len(DTS), 0.0, 0.0)
    J_o, du_o, due_o, g_o = oadj.window_gradient(case, u0, ue0, np.zeros((64, 96)), T0, DTS, w[:2],
                                                 ("heave_amp", "pitch_amp"))
    sim = _gpu(case, prec, u0, ue0, 1e-12 if prec == "f64" else 1e-7)
    J, taken = sim.window_forward(len(DTS), 3, DTS, w)
    assert np.allclose(taken, DTS)
    du, due, dp = sim.window_backward(1.0, tol=1e-12 if prec == "f64" else 1e-7)
    du = du.double().cpu().numpy()
    go = np.array([g_o["heave_amp"], g_o["pitch_amp"]])
    if prec == "f64":
        assert abs(J - J_o) <= 1e-9 * abs(J_o)
        assert np.abs(dp - go).max() <= 1e-7 * np.abs(go).max(), (dp, go)
        assert np.abs(du - du_o).max() <= 1e-7 * np.abs(du_o).max()
    else:
        assert abs(J - J_o) <= 1e-5 * abs(J_o)
        assert np.abs(dp - go).max() <= 1e-3 * np.abs(go).max(), (dp, go)
        assert np.linalg.norm(du - du_o) <= 1e-3 * np.linalg.norm(du_o)
    # the sim is left in the state after the window
    u_end, _ = sim.get_velocity()
    J2, _ = oadj.window_forward(case, u0, ue0, np.zeros((64, 96)), T0, DTS, w[:2])
    assert sim.get_time()[0] == pytest.approx(T0 + sum(DTS))
    sim.close()


def test_window_parameter_gradient_matches_gpu_central_differences():
    # the flapping-foil check: central differences of the GPU's own forward
    # window (FP64), 12 steps, checkpoints every 5. The objective is piecewise
    # smooth (limiter branches, the kernel band), so the secant at the study's
    # parameter step 1e-3 differs from the derivative by the kinks it spans
    # (measured on this case: 9e-5 relative for the heave amplitude, 0.8 % for
    # the pitch amplitude, converging to 1e-9 as the step shrinks to 1e-6);
    # the bars: 1e-6 at step 1e-6 and 2 % at step 1e-3.
    case, u0, ue0 = _foil()
    dts = [0.3] * 12
    w = (-1.0 / len(dts), 0.0, 0.0)
    sim = _gpu(case, "f64", u0, ue0, 1e-12)
    J, _ = sim.window_forward(len(dts), 5, dts, w)
    _, _, dp = sim.window_backward(1.0, tol=1e-12)
    for k, name in enumerate(("heave_amp", "pitch_amp")):
        v = getattr(case.body, name)
        for h, bar in ((1e-6, 1e-6), (1e-3, 2e-2)):
            Js = []
            for sgn in (1, -1):
                s2 = _gpu(case.with_(body=dataclasses.replace(case.body, **{name: v + sgn * h})), "f64", u0, ue0,
                          1e-12)
                Js.append(s2.window_forward(len(dts), 5, dts, w)[0])
                s2.close()
            fd = (Js[0] - Js[1]) / (2 * h)
            assert abs(dp[k] - fd) <= bar * abs(fd), (name, h, dp[k], fd)
    sim.close()


def test_autograd_function_matches_window_backward():
    import torch
    from paper_2407_16032_b300.autograd import Step, WindowForce
    case, u0, ue0 = _foil()
    sim = _gpu(case, "f64", u0, ue0, 1e-12)
    u = torch.tensor(u0, dtype=torch.float64, device="cuda", requires_grad=True)
    p = torch.tensor([case.body.heave_amp, case.body.pitch_amp], dtype=torch.float64, requires_grad=True)
    J = WindowForce.apply(u, p, sim, len(DTS), 3, DTS, (-1.0 / len(DTS), 0.0, 0.0), 1e-12)
    gu, gp = torch.autograd.grad(J, (u, p))
    sim2 = _gpu(case, "f64", u0, ue0, 1e-12)
    J2, _ = sim2.window_forward(len(DTS), 3, DTS, (-1.0 / len(DTS), 0.0, 0.0))
    du, _, dp = sim2.window_backward(1.0, tol=1e-12)
    assert float(J.detach()) == pytest.approx(J2, rel=1e-12)
    assert np.allclose(gp.numpy(), dp, rtol=1e-9, atol=0)
    assert torch.allclose(gu, du, rtol=1e-9, atol=1e-12 * float(du.abs().max()))
    # one-step Function: its pull-back equals the oracle's (FP64), and the
    # directional derivative by central differences of the GPU step. This flow
    # is nearly uniform (1 +- 0.02), so many limiter comparisons sit close to
    # ties and a difference step of 1e-6 already spans kinks (measured: 7 %
    # off on this case, in the oracle's own differences too); steps of 1e-7 /
    # 1e-8 are used, the closer one within 2e-4.
    sim3 = _gpu(case, "f64", u0, ue0, 1e-12)
    x = torch.tensor(u0, dtype=torch.float64, device="cuda", requires_grad=True)
    y = Step.apply(sim3, x, 0.3, 1e-12)
    rng = np.random.default_rng(3)
    lam = rng.normal(size=u0.shape)
    v = rng.normal(size=u0.shape)
    v[0][:, 0] = 0.0
    v[1][0, :] = 0.0
    (gx,) = torch.autograd.grad((y * torch.tensor(lam, device="cuda")).sum(), x)
    g = oracle.grid_from_case(case)
    ub_o, _ = oracle.step_vjp(g, oracle.make_body(case.body), T0, 0.3, u0, ue0, np.zeros((64, 96)), lam, None, None)
    got = float((gx.cpu().numpy() * v).sum())
    assert got == pytest.approx(float((ub_o * v).sum()), rel=1e-8)
    fds = []
    for h in (1e-7, 1e-8):
        outs = []
        for sgn in (1, -1):
            sim3.set_time(T0, 0.3)
            sim3.set_velocity(torch.tensor(u0 + sgn * h * v, device="cuda"), torch.tensor(ue0, device="cuda"))
            sim3.mom_step(0.3)
            outs.append(float((sim3.get_velocity()[0].cpu().numpy() * lam).sum()))
        fds.append((outs[0] - outs[1]) / (2 * h))
    assert min(abs(got - f) for f in fds) <= 2e-4 * abs(got), (got, fds)
    for s_ in (sim, sim2, sim3):
        s_.close()


_ROBUST = {}


def _robust_oracle(case, spin, dt, nwin, w):
    # the FP64 oracle spun up from the seeded start with its own CFL steps,
    # then its discrete adjoint over the window (computed once per module)
    key = (spin, dt, nwin)
    if key not in _ROBUST:
        u, ue = synth.initial_velocity(case)
        orc = oracle.Sim(case, tol=1e-11, u=u, ue=ue)
        dts = []
        for _ in range(spin):
            dts.append(orc.dt)
            orc.step()
        res = oadj.window_gradient(case, orc.u, orc.ue, orc.P, orc.t, [dt] * nwin, w, ("heave_amp", "pitch_amp"))
        _ROBUST[key] = (dts, orc.t, res)
    return _ROBUST[key]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_window_gradient_at_a_robust_length_on_the_256x128_foil(prec):
    # the flapping foil with chord 64 on 256 x 128, spun up 300 steps, then a
    # 50-step window of the mean thrust: a length at which the gradient is
    # well defined (central differences at 1e-3 and 1e-4 agree with each other
    # and with the adjoint up to 400 steps on this grid in both precisions).
    # The GPU adjoint against the FP64 oracle's adjoint (FP64 1e-6, FP32 1e-3)
    # and against the GPU's own central differences at steps 1e-3 and 1e-4
    # (2 % for the better of the two: a secant can span limiter kinks)
    import torch
    from paper_2407_16032_b300 import sim_from_case
    case = synth.config4_ellipse((256, 128), chord=64.0, A=16.0, centre=(64.0, 64.0))
    spin, dt, nwin = 300, 0.25, 50
    w = (-1.0 / nwin, 0.0, 0.0)
    dts, t0, (J_o, du_o, due_o, g_o) = _robust_oracle(case, spin, dt, nwin, w[:2])
    tol = 1e-11 if prec == "f64" else 1e-6
    sim = sim_from_case(case, prec, tol=tol, itmax=80)
    tdt = torch.float32 if prec == "f32" else torch.float64
    u, ue = synth.initial_velocity(case)
    ref = oracle.Sim(case, u=u, ue=ue)      # boundary values of the start as the oracle sets them
    sim.set_velocity(torch.tensor(ref.u, dtype=tdt, device="cuda"), torch.tensor(ref.ue, dtype=tdt, device="cuda"))
    for d in dts:
        sim.mom_step(d, allow_unconverged=True)
    sim.set_time(t0, dt)
    U0, UE0 = sim.get_velocity()
    P0 = sim.get_pressure()
    J, _ = sim.window_forward(nwin, 7, [dt] * nwin, w)
    _, _, dp = sim.window_backward(1.0, tol=tol)
    go = np.array([g_o["heave_amp"], g_o["pitch_amp"]])
    bar = 1e-6 if prec == "f64" else 1e-3
    assert abs(J - J_o) <= (1e-9 if prec == "f64" else 1e-5) * abs(J_o)
    assert np.all(np.abs(dp - go) <= bar * np.abs(go)), (dp, go)
    body = case.body
    for k, name in enumerate(("heave_amp", "pitch_amp")):
        errs = []
        for h in (1e-3, 1e-4):
            Js = []
            for s in (1.0, -1.0):
                sim.set_body(dataclasses.replace(body, **{name: getattr(body, name) + s * h}))
                sim.set_velocity(U0, UE0)
                sim.set_pressure(P0)
                sim.set_time(t0, dt)
                Js.append(sim.window_forward(nwin, 7, [dt] * nwin, w)[0])
            errs.append(abs((Js[0] - Js[1]) / (2 * h) - dp[k]) / abs(dp[k]))
        # a limiter branch switch within h of the point spoils at most one step size
        assert min(errs) <= 2e-2, (name, errs, dp[k])
    sim.set_body(body)
