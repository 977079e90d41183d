"""GPU parity of bodies given by samples (WL_BODY_USER_FACE_FIELDS): the
distance function and motion of any shape evaluated by the caller (Sec. 3),
moments formed on the device (Sec. 2), against the oracle fed the same
samples."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import gpu_fields, gpu_sim, near_body_p_err, p_err, rel_max, report, start_fields

pytestmark = pytest.mark.gpu

NPT = {"f32": np.float32, "f64": np.float64}


def _user(case):
    return case.with_(body=synth.Body("user"))


def _sim_with(case, shape, prec, **kw):
    sim = gpu_sim(_user(case), prec, **kw)
    samples = synth.sample_body(shape, case.ndim, case.n, NPT[prec])
    sim.set_body_fields(*samples)
    return sim, [s.astype(np.float64) for s in samples]


def _fields(sim):
    c, m, V = sim.get_body_fields()
    return c.double().cpu().numpy(), m.double().cpu().numpy(), V.double().cpu().numpy()


@pytest.mark.parametrize("prec,ndim", [("f32", 3), ("f64", 2), ("f32", 2)])
def test_sampled_sphere_fields_match_the_analytic_sphere(prec, ndim):
    # the sphere as samples and as the analytic primitive: the same Poisson
    # coefficients, mu1 n and velocity on every face (FP64: to rounding; FP32:
    # the samples carry the distance rounded to FP32, one ulp of d moves mu0
    # by at most |d| 2^-24 / eps), and the oracle fed the same samples
    if ndim == 3:
        case = synth.config3_sphere((64, 40, 32), D=14.0, centre=(22.3, 19.6, 15.1))
    else:
        case = synth.config1_circle((96, 48)).with_(body=synth.Body("sphere", (30.3, 23.9, 0.0), 8.0))
    b = case.body
    shape = synth.Circle(b.centre, b.radius)
    su, samples = _sim_with(case, shape, prec)
    sa = gpu_sim(case, prec)
    cu, mu, Vu = _fields(su)
    ca, ma, Va = _fields(sa)
    bar = 2e-6 if prec == "f32" else 1e-13
    assert np.abs(cu - ca).max() <= bar and np.abs(mu - ma).max() <= bar and np.abs(Vu - Va).max() <= bar
    g = oracle.grid_from_case(case)
    mu0o, mu1o, Vo = oracle.measure_sampled(g, *samples[:3])
    co = oracle.coeffs(g, mu0o)
    ulp = 2.0 ** -24 if prec == "f32" else 2.0 ** -53
    assert np.abs(cu - co).max() <= 8 * ulp
    assert np.abs(mu - mu1o).max() <= 8 * ulp
    assert np.array_equal(Vu, Vo)
    assert (cu < 1).sum() > 100


def test_user_body_before_its_fields_is_all_fluid():
    case = _user(synth.config1_circle((64, 32)))
    sim = gpu_sim(case, "f64")
    c, m, V = _fields(sim)
    g = oracle.grid_from_case(case)
    assert np.array_equal(c, oracle.coeffs(g, None))
    assert not m.any()


def _shapes(name):
    if name == "union2d":
        case = synth.config1_circle((128, 64))
        shape = synth.Circle((30.3, 31.6), 7.0) + synth.Circle((39.1, 27.2), 5.0)
    elif name == "spin2d":
        case, shape, _ = synth.spinning_cylinders(D=24, Re=200.0, xi=2.0)
    elif name == "bowl3d":
        # a sphere minus the half-space above a tilted plane through it, plus a
        # smaller sphere behind it: three surfaces, two kinds of corners
        case = synth.config3_sphere((96, 48, 48), D=16.0, centre=(24.0, 24.0, 24.0))
        shape = (synth.Circle((24.3, 23.8, 24.1), 8.0) - synth.HalfSpace((24.3, 25.0, 24.1), (0.3, 1.0, 0.2))
                 + synth.Circle((36.2, 21.7, 23.4), 4.0))
    return case, shape


def _run_pair(case, shape, steps, prec, gpu_tol, oracle_tol=1e-11, perturb=0.0):
    """Oracle (orc_step_fields with the sampled moments) and GPU, the same
    samples and start, the oracle's CFL steps; with perturb, the oracle alone
    from a start perturbed by that absolute amount (its own response)."""
    import torch
    g = oracle.grid_from_case(case)
    sim, samples = _sim_with(case, shape, prec, tol=gpu_tol, itmax=60)
    fields = oracle.measure_sampled(g, *samples[:3])
    u, ue = start_fields(case, prec)
    # the start's boundary values as the oracle's stepping loop sets them
    ref = oracle.Sim(case.with_(body=synth.Body()), u=u, ue=ue)
    u, ue = ref.u.copy(), ref.ue.copy()
    if perturb:
        u = u + perturb * np.random.default_rng(9).uniform(-1, 1, size=u.shape)
    tdt = torch.float32 if prec == "f32" else torch.float64
    sim.set_velocity(torch.tensor(u, dtype=tdt).cuda(), torch.tensor(ue, dtype=tdt).cuda())
    P = np.zeros(u.shape[1:])
    dt, dts = case.dt0, []
    for _ in range(steps):
        dts.append(dt)
        u, ue, P = oracle.step_fields_fn(g, fields, dt, u, ue, P, tol=oracle_tol)
        if not perturb:
            sim.mom_step(dt, allow_unconverged=True)
        dt = oracle.cfl(g, u, ue, case.cfl, case.dt_max)
    return sim, samples, fields, (u, ue, P), dts


@pytest.mark.parametrize("name,prec", [("union2d", "f64"), ("union2d", "f32"), ("spin2d", "f32"), ("bowl3d", "f32")])
def test_sampled_shape_steps_match_the_oracle(name, prec):
    # ten steps past a non-primitive body (a union, a spinning control
    # cylinder beside a fixed one, a cut sphere plus a sphere): velocity and
    # pressure against the oracle's. FP64: 1e-9. FP32: the bars of the
    # analytic bodies' step parity, five times the oracle's own response to a
    # 1e-7 perturbation of the start, at least 1e-5
    case, shape = _shapes(name)
    steps = 10
    sim, samples, fields, (u_o, ue_o, P_o), dts = _run_pair(case, shape, steps, prec,
                                                          5e-9 if prec == "f32" else 1e-11)
    u, ue, p = gpu_fields(sim)
    g = oracle.grid_from_case(case)
    c = oracle.coeffs(g, fields[0])
    if prec == "f64":
        bu = bp = 1e-9
    else:
        _, _, _, (u_p, _, P_p), _ = _run_pair(case, shape, steps, prec, 5e-9, perturb=1e-7)
        bu = max(1e-5, 5 * float(np.abs(u_p - u_o).max() / np.abs(u_o).max()))
        bp = max(1e-5, 5 * p_err(P_p, P_o, c, case.ndim))
    eu, ep = rel_max(u, u_o), p_err(p, P_o, c, case.ndim)
    F = sim.forces()
    F_o = oracle.forces_sampled(g, samples[3], samples[4], P_o)
    ef = float(np.abs(F - F_o).max() / np.abs(F_o).max())
    report(f"sampled {name} {prec}", u=eu, p=ep, bar_u=bu, bar_p=bp, force_rel=ef,
           p_near_body=near_body_p_err(p, P_o, c, case.ndim))
    assert eu < bu, (eu, bu)
    assert ep < bp, (ep, bp)
    assert ef < bp, (F, F_o)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_sampled_viscous_force_and_force_dp_match_the_oracle(prec):
    # the same velocity on both sides: the viscous force of the sampled union
    # (bar of the analytic bodies' viscous-force test) and dF/dp per cell
    import torch
    case, shape = _shapes("union2d")
    case = case.with_(nu=0.05)
    sim, samples = _sim_with(case, shape, prec)
    g = oracle.grid_from_case(case)
    u = synth.random_field(5, 2, case.n).astype(NPT[prec]).astype(np.float64)
    tdt = torch.float32 if prec == "f32" else torch.float64
    sim.set_velocity(torch.tensor(u, dtype=tdt).cuda())
    u_s, ue_s = sim.get_velocity()
    u = u_s.double().cpu().numpy()
    ue = ue_s.double().cpu().numpy() if ue_s is not None else None
    F = sim.forces_viscous()
    F_o = oracle.forces_viscous_sampled(g, samples[3], samples[4], u, ue)
    eps = 2.0 ** -24 if prec == "f32" else 2.0 ** -53
    surf = 2 * np.pi * 12.0
    bar = 16 * 2 * eps * case.nu * np.abs(u).max() * surf
    assert np.abs(F_o).max() > 100 * bar
    assert np.abs(F - F_o).max() <= bar, (F, F_o, bar)
    for axis in range(2):
        gd = sim.force_dp(axis).cpu().numpy()
        go = oracle.force_dp_sampled(g, samples[3], samples[4], axis)
        act = gd != 0      # the library leaves out inactive cells (all faces solid)
        assert act.sum() > 50
        assert np.abs(gd - go)[act].max() <= 1e-15 * np.abs(go).max()


def test_set_body_fields_rejects_an_analytic_body():
    from paper_2407_16032_b300.wl import WLError, WL_ERR_ARG
    case = synth.config1_circle((64, 32))
    sim = gpu_sim(case, "f64")
    d = synth.sample_body(synth.Circle((20.0, 16.0), 5.0), 2, case.n)
    with pytest.raises(WLError) as e:
        sim.set_body_fields(*d)
    assert e.value.code == WL_ERR_ARG


@pytest.mark.parametrize("viscous", [False, True])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_spin_rate_window_gradient_matches_the_oracle(prec, viscous):
    # Sec. 6.1's controlled cylinder (coarse): J = thrust (pressure, or pressure
    # plus viscous force) weighted towards the window's last steps; its gradient along the spin rate's velocity tangent
    # (wl_set_body_velocity_tangent) and along the start velocity, against the
    # FP64 oracle's discrete adjoint on the same samples (the bars of the
    # analytic bodies' window test)
    import torch
    from oracle import adjoint as oadj
    case, shape, tangent = synth.spinning_cylinders(D=16, Re=100.0, xi=3.0)
    g = oracle.grid_from_case(case)
    sim, samples = _sim_with(case, shape, prec, tol=1e-12 if prec == "f64" else 1e-7, itmax=80)
    dV = synth.sample_body(tangent, 2, case.n, NPT[prec])[2]
    sim.set_body_velocity_tangent(dV)
    u0 = synth.random_field(31, 2, case.n, amp=0.05, offset=(1.0, 0.0)).astype(NPT[prec]).astype(np.float64)
    u0[0][:, 0] = 1.0
    u0[1][0, :] = 0.0
    ue0 = np.ones(case.n[1])
    tdt = torch.float32 if prec == "f32" else torch.float64
    sim.set_velocity(torch.tensor(u0, dtype=tdt).cuda(), torch.tensor(ue0, dtype=tdt).cuda())
    dts = [0.2, 0.22, 0.2, 0.21, 0.2, 0.2]
    w, sw = (-1.0, 0.0), [0.0, 0.0, 0.0, 0.25, 0.5, 1.0]
    J, taken = sim.window_forward(len(dts), 2, dts, w, step_w=sw, viscous=viscous)
    du, due, dp = sim.window_backward(1.0, tol=1e-12 if prec == "f64" else 1e-7)
    fields = oracle.measure_sampled(g, *samples[:3])
    J_o, du_o, due_o, dth_o = oadj.window_gradient_sampled(case, fields, (samples[3], samples[4]),
                                                           dV.astype(np.float64), u0, ue0, np.zeros(u0.shape[1:]),
                                                           dts, w, sw, viscous=viscous)
    du = du.double().cpu().numpy()
    assert abs(dth_o) > 1e-3 and dp[1] == 0.0
    if prec == "f64":
        assert abs(J - J_o) <= 1e-9 * abs(J_o)
        assert abs(dp[0] - dth_o) <= 1e-7 * abs(dth_o), (dp, dth_o)
        assert np.abs(du - du_o).max() <= 1e-7 * np.abs(du_o).max()
    else:
        assert abs(J - J_o) <= 1e-5 * abs(J_o)
        assert abs(dp[0] - dth_o) <= 1e-3 * abs(dth_o), (dp, dth_o)
        assert np.linalg.norm(du - du_o) <= 1e-3 * np.linalg.norm(du_o)
    # without a tangent the parameter gradient is zero
    sim.set_body_velocity_tangent(None)
    sim.set_velocity(torch.tensor(u0, dtype=tdt).cuda(), torch.tensor(ue0, dtype=tdt).cuda())
    sim.window_forward(len(dts), 2, dts, w, step_w=sw)
    assert not sim.window_backward(1.0, tol=1e-7)[2].any()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_a_sampled_body_moved_every_step_matches_the_oracle(prec):
    # the caller's map moves the body: a circle heaving as c_y + A sin(w t),
    # with velocity A w cos(w t), sampled at t + dt and set before every step
    # (the library does not re-measure a sampled body itself); the oracle steps
    # with the moments of the same samples. 10 steps; FP64 1e-9, FP32 1e-5
    import math
    import torch
    case = synth.config1_circle((128, 64))
    g = oracle.grid_from_case(case)
    cx, cy, R, A, w = 30.3, 31.6, 6.0, 3.0, 2 * math.pi / 40.0

    def shape(t):
        return synth.Circle((cx, cy + A * math.sin(w * t)), R, velocity=(0.0, A * w * math.cos(w * t)))

    sim = gpu_sim(_user(case), prec, tol=1e-11 if prec == "f64" else 5e-9, itmax=60)
    u, ue = start_fields(case, prec)
    ref = oracle.Sim(case.with_(body=synth.Body()), u=u, ue=ue)
    u, ue = ref.u.copy(), ref.ue.copy()
    tdt = torch.float32 if prec == "f32" else torch.float64
    sim.set_velocity(torch.tensor(u, dtype=tdt).cuda(), torch.tensor(ue, dtype=tdt).cuda())
    P = np.zeros(u.shape[1:])
    t, dt = 0.0, case.dt0
    for _ in range(10):
        samples = synth.sample_body(shape(t + dt), 2, case.n, NPT[prec])
        sim.set_body_fields(*samples)
        fields = oracle.measure_sampled(g, *[s.astype(np.float64) for s in samples[:3]])
        u, ue, P = oracle.step_fields_fn(g, fields, dt, u, ue, P, tol=1e-11)
        sim.mom_step(dt, allow_unconverged=True)
        t += dt
        dt = oracle.cfl(g, u, ue, case.cfl, case.dt_max)
    ug, ueg, pg = gpu_fields(sim)
    c = oracle.coeffs(g, fields[0])
    bar = 1e-9 if prec == "f64" else 1e-5
    eu, ep = rel_max(ug, u), p_err(pg, P, c, 2)
    report(f"sampled heaving circle {prec}", u=eu, p=ep, bar_u=bar, bar_p=bar,
           p_near_body=near_body_p_err(pg, P, c, 2))
    assert eu < bar and ep < bar, (eu, ep)


def _heave3d_run(case, steps, shape, with_gpu, perturb=0.0):
    """Oracle (and GPU) steps with a sphere re-sampled before every step; the
    oracle's own CFL steps; perturb: the oracle alone from a start perturbed
    by that absolute amount."""
    import torch
    g = oracle.grid_from_case(case)
    u, ue = start_fields(case, "f32")
    ref = oracle.Sim(case.with_(body=synth.Body()), u=u, ue=ue)
    u, ue = ref.u.copy(), ref.ue.copy()
    if perturb:
        u = u + perturb * np.random.default_rng(9).uniform(-1, 1, size=u.shape)
    sim = None
    if with_gpu:
        sim = gpu_sim(_user(case), "f32", tol=5e-9, itmax=60)
        sim.set_velocity(torch.tensor(u, dtype=torch.float32).cuda(), torch.tensor(ue, dtype=torch.float32).cuda())
    P = np.zeros(u.shape[1:])
    t, dt = 0.0, case.dt0
    for _ in range(steps):
        samples = synth.sample_body(shape(t + dt), 3, case.n, np.float32)
        fields = oracle.measure_sampled(g, *[x.astype(np.float64) for x in samples[:3]])
        u, ue, P = oracle.step_fields_fn(g, fields, dt, u, ue, P, tol=1e-11)
        if sim is not None:
            sim.set_body_fields(*samples)
            sim.mom_step(dt, allow_unconverged=True)
        t += dt
        dt = oracle.cfl(g, u, ue, case.cfl, case.dt_max)
    return sim, (u, ue, P), oracle.coeffs(g, fields[0])


@pytest.mark.parametrize("steps", [1, 10])
def test_a_sampled_sphere_moved_every_step_in_3d_matches_the_oracle(steps):
    # the 3D FP32 path of a moving sampled body: plane-marching flux, the band
    # blend over the tile list rebuilt after every wl_set_body_fields, the
    # coefficients of every level rebuilt on the device; a heaving sphere
    # re-sampled before each step against the oracle on the same samples, with
    # the bars of the analytic 3D sphere cases: 1e-6 after one step; after ten,
    # five times the oracle's own response to a 1e-7 perturbation of the start
    # (at least 1e-5)
    import math
    case = synth.config5_moving_sphere((96, 48, 48), D=10.0, centre=(24.0, 24.0, 24.0))
    c0, R, A, w = (24.3, 23.8, 24.1), 5.0, 2.5, 2 * math.pi / 30.0

    def shape(t):
        return synth.Circle((c0[0], c0[1] + A * math.sin(w * t), c0[2]), R,
                            velocity=(0.0, A * w * math.cos(w * t), 0.0))

    sim, (u, ue, P), c = _heave3d_run(case, steps, shape, True)
    ug, ueg, pg = gpu_fields(sim)
    eu, ep = rel_max(ug, u), p_err(pg, P, c, 3)
    if steps == 1:
        bu = bp = 1e-6
    else:
        _, (up, _, Pp), _ = _heave3d_run(case, steps, shape, False, perturb=1e-7)
        bu = max(1e-5, 5 * float(np.abs(up - u).max() / np.abs(u).max()))
        bp = max(1e-5, 5 * p_err(Pp, P, c, 3))
    report(f"sampled heaving sphere 3D f32 ({steps} steps)", u=eu, p=ep, bar_u=bu, bar_p=bp,
           p_near_body=near_body_p_err(pg, P, c, 3))
    assert eu < bu and ep < bp, (eu, ep, bu, bp)
