"""Pins of the FP64 oracle's discrete adjoint of one step (the vector-Jacobian
product with respect to the start velocity and exit plane, fixed dt and body).

Expected values come from central finite differences of the oracle's forward
step (an independent computation: the forward code never calls the adjoint)
and from a structural property of the projection, not from the adjoint's own
formulas.
"""
import numpy as np
import pytest

import oracle
import synth

RNG = np.random.default_rng(99)


def _case(kind):
    B = synth.Body()
    if kind == "periodic2d":
        g = oracle.make_grid(2, (24, 16), (True, True), False, (0.0, 0.0), 0.01)
        u0 = synth.random_field(11, 2, (24, 16), amp=0.5)
    elif kind == "channel_exit":
        g = oracle.make_grid(2, (20, 12), (False, True), True, (1.0, 0.0), 0.005)
        u0 = synth.random_field(12, 2, (20, 12), amp=0.2, offset=(1.0, 0.0))
    elif kind == "circle":
        g = oracle.make_grid(2, (28, 20), (False, False), True, (1.0, 0.0), 0.01)
        u0 = synth.random_field(13, 2, (28, 20), amp=0.2, offset=(1.0, 0.0))
        B = synth.Body(kind="sphere", centre=(10.0, 10.3, 0.0), radius=4.2)
    elif kind == "walled3d":
        g = oracle.make_grid(3, (12, 10, 8), (True, True, False), False, (0.0, 0.0, 0.0), 0.02)
        u0 = synth.random_field(14, 3, (12, 10, 8), amp=0.4)
    elif kind == "sphere3d_exit":
        # a 3D body with an exit plane: the sphere's kernel band crosses the
        # periodic z boundary and reaches both y walls, and the free stream is
        # 1.6 so that terms scaled by the exit plane's mean velocity count
        g = oracle.make_grid(3, (14, 10, 12), (False, False, True), True, (1.6, 0.0, 0.0), 0.02)
        u0 = synth.random_field(15, 3, (14, 10, 12), amp=0.2, offset=(1.6, 0.0, 0.0))
        B = synth.Body(kind="sphere", centre=(7.0, 4.9, 1.2), radius=4.3)
    elif kind == "walled3d_body":
        # walls on every face and a sphere whose band reaches the lower z wall
        g = oracle.make_grid(3, (12, 10, 8), (False, False, False), False, (0.0, 0.0, 0.0), 0.02)
        u0 = synth.random_field(18, 3, (12, 10, 8), amp=0.3)
        B = synth.Body(kind="sphere", centre=(6.2, 5.1, 2.3), radius=2.5)
    elif kind == "square_wave2d":
        # a square wave in x with small noise: the limiter clips many faces
        g = oracle.make_grid(2, (24, 16), (True, True), False, (0.0, 0.0), 0.01)
        u0 = synth.random_field(16, 2, (24, 16), amp=0.01, offset=(1.0, 0.0))
        x = np.arange(24)
        u0[0] += 0.5 * np.where((x // 4) % 2 == 0, 1.0, -1.0)[None, :]
        u0[1] += 0.3 * np.where((x // 4) % 2 == 0, -1.0, 1.0)[None, :]
    else:
        raise KeyError(kind)
    ue0 = np.zeros(max(oracle.plane_size(g), 1))
    if g.exit_hi_x:
        ue0 = g.U[0] * (1.0 + 0.1 * (2 * synth.uniform01(21, 0, ue0.size) - 1))
    return g, oracle.make_body(B), u0, ue0


def _dot(a, b):
    return float(np.sum(np.asarray(a) * np.asarray(b)))


def _fd_step(g, B, t, dt, u0, ue0, P0, lu, le, v, ve, lP=None):
    """Central differences of <(lu, le, lP), step(u0 + h v, ue0 + h ve)> at two
    small h. A limiter branch switch (a kink of the piecewise-smooth step) within
    h of the point spoils one of them; both are returned."""
    out = []
    for h in (1e-6, 1e-7):
        up, uep, Pp = oracle.step_fn(g, B, t, dt, u0 + h * v, ue0 + h * ve, P0)
        um, uem, Pm = oracle.step_fn(g, B, t, dt, u0 - h * v, ue0 - h * ve, P0)
        d = _dot(lu, up - um) + _dot(le[: uep.size], uep - uem)
        if lP is not None:
            d += _dot(lP, Pp - Pm)
        out.append(d / (2 * h))
    return out


def _close_to_one(got, fds, rel, abs_):
    return any(abs(got - f) <= rel * abs(f) + abs_ for f in fds)


@pytest.mark.parametrize("kind", ["periodic2d", "channel_exit", "circle", "walled3d", "sphere3d_exit",
                                  "square_wave2d"])
def test_conv_diff_vjp_matches_central_differences(kind):
    g, _, u0, ue0 = _case(kind)
    lam = RNG.normal(size=u0.shape)
    ub, ueb = oracle.conv_diff_vjp(g, u0, ue0, lam)
    for _ in range(3):
        v = RNG.normal(size=u0.shape)
        ve = RNG.normal(size=ue0.shape) if g.exit_hi_x else np.zeros_like(ue0)
        # the flux is piecewise quadratic: a central difference is exact up to
        # rounding unless a limiter kink lies within h of the point (the square
        # wave puts kinks near many faces), so three step sizes are tried
        fds = []
        for h in (1e-6, 1e-7, 1e-8):
            rp = oracle.conv_diff(g, u0 + h * v, ue0 + h * ve)
            rm = oracle.conv_diff(g, u0 - h * v, ue0 - h * ve)
            fds.append(_dot(lam, (rp - rm) / (2 * h)))
        got = _dot(ub, v) + _dot(ueb, ve)
        assert _close_to_one(got, fds, 1e-7, 1e-9), (got, fds)


@pytest.mark.parametrize("kind", ["periodic2d", "channel_exit", "circle", "walled3d", "sphere3d_exit",
                                  "walled3d_body", "square_wave2d"])
def test_step_vjp_matches_central_differences(kind):
    g, B, u0, ue0 = _case(kind)
    dt, t = 0.3, 0.0
    P0 = np.zeros(u0.shape[1:])
    lu = RNG.normal(size=u0.shape)
    le = RNG.normal(size=ue0.shape) if g.exit_hi_x else np.zeros_like(ue0)
    ub, ueb = oracle.step_vjp(g, B, t, dt, u0, ue0, P0, lu, le)
    assert np.all(np.isfinite(ub)) and np.all(np.isfinite(ueb))
    for _ in range(2):
        v = RNG.normal(size=u0.shape)
        ve = RNG.normal(size=ue0.shape) if g.exit_hi_x else np.zeros_like(ue0)
        fds = _fd_step(g, B, t, dt, u0, ue0, P0, lu, le, v, ve)
        got = _dot(ub, v) + _dot(ueb, ve)
        assert _close_to_one(got, fds, 1e-6, 1e-6), (got, fds)


def test_step_vjp_single_entries_match_finite_differences():
    # unit directions on a few faces, including the lower wall face and exit plane
    g, B, u0, ue0 = _case("channel_exit")
    dt, P0 = 0.25, np.zeros(u0.shape[1:])
    lu = RNG.normal(size=u0.shape)
    le = RNG.normal(size=ue0.shape)
    ub, ueb = oracle.step_vjp(g, B, 0.0, dt, u0, ue0, P0, lu, le)
    zu, ze = np.zeros_like(u0), np.zeros_like(ue0)
    for idx in [(0, 5, 0), (0, 3, 19), (1, 7, 10), (0, 0, 1)]:
        v = zu.copy()
        v[idx] = 1.0
        fds = _fd_step(g, B, 0.0, dt, u0, ue0, P0, lu, le, v, ze)
        assert _close_to_one(ub[idx], fds, 1e-5, 1e-7), (idx, ub[idx], fds)
    for p in (0, 5, 11):
        ve = ze.copy()
        ve[p] = 1.0
        fds = _fd_step(g, B, 0.0, dt, u0, ue0, P0, lu, le, zu, ve)
        assert _close_to_one(ueb[p], fds, 1e-5, 1e-7), (p, ueb[p], fds)


def test_step_vjp_annihilates_gradients_on_periodic_grid():
    # Body-free periodic grid: the corrector ends with the orthogonal projector
    # onto divergence-free fields, which maps every discrete gradient to zero,
    # so a cotangent that is a gradient has a zero pull-back.
    g, B, u0, ue0 = _case("periodic2d")
    phi = RNG.normal(size=u0.shape[1:])
    lu = np.stack([phi - np.roll(phi, 1, axis=-1), phi - np.roll(phi, 1, axis=-2)])
    ub, _ = oracle.step_vjp(g, B, 0.0, 0.3, u0, ue0, np.zeros(u0.shape[1:]), lu, None)
    assert np.max(np.abs(ub)) < 1e-10 * np.max(np.abs(lu))


@pytest.mark.parametrize("kind", ["circle", "channel_exit", "walled3d", "sphere3d_exit"])
def test_step_vjp_with_pressure_cotangent_matches_central_differences(kind):
    # the reported pressure (mean-free over active cells) enters force
    # objectives; its cotangent joins the corrector projection's adjoint solve
    g, B, u0, ue0 = _case(kind)
    dt, t = 0.3, 0.0
    P0 = np.zeros(u0.shape[1:])
    lu = np.zeros(u0.shape)
    le = np.zeros_like(ue0)
    lP = RNG.normal(size=u0.shape[1:])
    ub, ueb = oracle.step_vjp(g, B, t, dt, u0, ue0, P0, lu, le, lP)
    assert np.max(np.abs(ub)) > 0
    for _ in range(2):
        v = RNG.normal(size=u0.shape)
        ve = RNG.normal(size=ue0.shape) if g.exit_hi_x else np.zeros_like(ue0)
        fds = _fd_step(g, B, t, dt, u0, ue0, P0, lu, le, v, ve, lP)
        got = _dot(ub, v) + _dot(ueb, ve)
        assert _close_to_one(got, fds, 1e-6, 1e-6), (got, fds)


def _fields_case(kind):
    if kind == "circle":
        g, B, u0, ue0 = _case("circle")
        body = synth.Body(kind="sphere", centre=(10.0, 10.3, 0.0), radius=4.2)
    elif kind == "periodic_circle":
        # periodic in y with the circle's kernel band across the periodic seam
        g = oracle.make_grid(2, (28, 20), (False, True), True, (1.0, 0.0), 0.01)
        u0 = synth.random_field(19, 2, (28, 20), amp=0.2, offset=(1.0, 0.0))
        ue0 = 1.0 + 0.1 * (2 * synth.uniform01(24, 0, 20) - 1)
        body = synth.Body(kind="sphere", centre=(10.0, 1.1, 0.0), radius=4.2)
        B = oracle.make_body(body)
    elif kind == "wall_circle":
        # the circle's kernel band reaches the upper y wall
        g = oracle.make_grid(2, (28, 20), (False, False), True, (1.0, 0.0), 0.01)
        u0 = synth.random_field(20, 2, (28, 20), amp=0.2, offset=(1.0, 0.0))
        ue0 = 1.0 + 0.1 * (2 * synth.uniform01(25, 0, 20) - 1)
        body = synth.Body(kind="sphere", centre=(10.0, 17.2, 0.0), radius=3.5)
        B = oracle.make_body(body)
    else:
        g = oracle.make_grid(2, (40, 28), (False, False), True, (1.0, 0.0), 0.02)
        u0 = synth.random_field(17, 2, (40, 28), amp=0.1, offset=(1.0, 0.0))
        ue0 = 1.0 + 0.1 * (2 * synth.uniform01(23, 0, 28) - 1)
        body = synth.Body("ellipse", (15.2, 14.1, 0.0), 0.0, (8.0, 1.6), heave_amp=2.0, pitch_amp=0.3, omega=0.05)
        B = oracle.make_body(body)
    return g, B, body, u0, ue0


@pytest.mark.parametrize("kind", ["circle", "ellipse", "periodic_circle", "wall_circle"])
def test_field_cotangents_match_central_differences(kind):
    # the step's dependence on the measured face fields (mu0 in the blend and
    # in the Poisson coefficients, mu1 n and V in the blend), checked against
    # central differences of the step run with perturbed explicit fields
    g, B, body, u0, ue0 = _fields_case(kind)
    dt, t = 0.3, 1.0
    fields = oracle.measure(g, B, t + dt)
    P0 = np.zeros(u0.shape[1:])
    lu = RNG.normal(size=u0.shape)
    le = RNG.normal(size=ue0.shape)
    lP = RNG.normal(size=u0.shape[1:])
    ub, ueb, mu0b, mu1nb, Vb = oracle.step_vjp_fields(g, fields, dt, u0, ue0, P0, lu, le, lP)
    ub2, ueb2 = oracle.step_vjp(g, B, t, dt, u0, ue0, P0, lu, le, lP)
    assert np.array_equal(ub, ub2) and np.array_equal(ueb, ueb2)
    mu0, mu1n, V = fields
    band = (mu0 > 0.05) & (mu0 < 1.0)          # keep the active set of the solve fixed
    assert band.sum() > 10
    for _ in range(2):
        d0 = np.where(band, RNG.normal(size=mu0.shape), 0.0)
        d1 = np.zeros_like(mu1n)
        d1[:, : g.ndim] = np.where(band[:, None], RNG.normal(size=mu1n[:, : g.ndim].shape), 0.0)
        dV = np.where(band, RNG.normal(size=V.shape), 0.0)
        got = _dot(mu0b, d0) + _dot(mu1nb, d1) + _dot(Vb, dV)
        fds = []
        for h in (1e-6, 1e-7):
            outs = []
            for sgn in (1, -1):
                f = (mu0 + sgn * h * d0, mu1n + sgn * h * d1, V + sgn * h * dV)
                u, ue, P = oracle.step_fields_fn(g, f, dt, u0, ue0, P0)
                outs.append(_dot(lu, u) + _dot(le, ue) + _dot(lP, P))
            fds.append((outs[0] - outs[1]) / (2 * h))
        assert _close_to_one(got, fds, 1e-6, 1e-6), (got, fds)


def test_window_parameter_gradient_matches_central_differences():
    # mean thrust of a heaving and pitching ellipse over a few steps: the
    # adjoint gradient with respect to the heave and pitch amplitudes against
    # central differences of complete forward runs
    from oracle import adjoint
    case = synth.Case("el", 2, (48, 32, 1), (False, False, False), True, (1.0, 0.0, 0.0), 0.02,
                      synth.Body("ellipse", (16.3, 15.8, 0.0), 0.0, (8.0, 1.6), heave_amp=2.0, pitch_amp=0.3,
                                 omega=0.06))
    g = oracle.grid_from_case(case)
    u0 = synth.random_field(31, 2, (48, 32, 1), amp=0.05, offset=(1.0, 0.0))
    u0[0][:, 0] = 1.0
    u0[1][0, :] = 0.0
    ue0 = np.ones(32)
    P0 = np.zeros((32, 48))
    dts = [0.25, 0.3, 0.3, 0.3]
    w = (-1.0 / len(dts), 0.0)
    J, du0, due0, grads = adjoint.window_gradient(case, u0, ue0, P0, 0.5, dts, w, ("heave_amp", "pitch_amp"))
    assert np.isfinite(J) and J != 0.0
    for name in ("heave_amp", "pitch_amp"):
        fds = []
        for h in (1e-4, 1e-5):
            v = getattr(case.body, name)
            Jp, _ = adjoint.window_forward(case, u0, ue0, P0, 0.5, dts, w, adjoint._with(case.body, name, v + h))
            Jm, _ = adjoint.window_forward(case, u0, ue0, P0, 0.5, dts, w, adjoint._with(case.body, name, v - h))
            fds.append((Jp - Jm) / (2 * h))
        assert _close_to_one(grads[name], fds, 1e-5, 1e-8), (name, grads[name], fds)
    # and the initial-velocity gradient along a random direction
    v = RNG.normal(size=u0.shape)
    v[0][:, 0] = 0.0
    v[1][0, :] = 0.0
    fds = []
    for h in (1e-6, 1e-7):
        Jp, _ = adjoint.window_forward(case, u0 + h * v, ue0, P0, 0.5, dts, w)
        Jm, _ = adjoint.window_forward(case, u0 - h * v, ue0, P0, 0.5, dts, w)
        fds.append((Jp - Jm) / (2 * h))
    assert _close_to_one(_dot(du0, v), fds, 1e-5, 1e-9), (_dot(du0, v), fds)


@pytest.mark.parametrize("viscous", [False, True])
def test_sampled_body_velocity_gradient_matches_central_differences(viscous):
    # a spinning control cylinder beside a fixed one (Sec. 6.1's controlled
    # flow, coarse): the window gradient of the final step's thrust along the
    # spin rate's velocity tangent against central differences of complete
    # forward windows with the face velocity moved by +-h dV
    from oracle import adjoint as oadj
    case, shape, tangent = synth.spinning_cylinders(D=12, Re=100.0, xi=3.0)
    g = oracle.grid_from_case(case)
    d, nf, V, dc, nc = synth.sample_body(shape, 2, case.n)
    dV = synth.sample_body(tangent, 2, case.n)[2]
    fields = oracle.measure_sampled(g, d, nf, V)
    u0 = synth.random_field(31, 2, case.n, amp=0.05, offset=(1.0, 0.0))
    u0[0][:, 0] = 1.0
    u0[1][0, :] = 0.0
    ue0 = np.ones(case.n[1])
    P0 = np.zeros(u0.shape[1:])
    dts = [0.2, 0.22, 0.2, 0.21]
    w, sw = (-1.0, 0.0), [0.0, 0.0, 0.5, 1.0]
    J, du, due, dth = oadj.window_gradient_sampled(case, fields, (dc, nc), dV, u0, ue0, P0, dts, w, sw, viscous)
    assert abs(dth) > 1e-3
    for h in (1e-4, 1e-5):
        Jp = oadj.window_forward_sampled(case, (fields[0], fields[1], fields[2] + h * dV), (dc, nc), u0, ue0, P0,
                                         dts, w, sw, viscous=viscous)[0]
        Jm = oadj.window_forward_sampled(case, (fields[0], fields[1], fields[2] - h * dV), (dc, nc), u0, ue0, P0,
                                         dts, w, sw, viscous=viscous)[0]
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - dth) <= 1e-5 * abs(dth), (fd, dth, h)
