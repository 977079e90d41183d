"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Each test names what fixes the expected value: a closed form of the scheme, an
invariant of the discretisation, or an independent computation (quadrature,
a dense direct solve). None of them retypes the oracle's own formula.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from synth import face_coords

RNG = np.random.default_rng(1234)


# --------------------------------------------------------------- QUICK ------
def test_quick_exact_on_linear_data():
    # On equally spaced linear samples both the interpolant and the limiter
    # return the face midpoint value (c+d)/2 (third-order scheme, any slope).
    for _ in range(200):
        c, h = RNG.normal(), RNG.normal()
        assert oracle.quick(c - h, c, c + h) == pytest.approx(c + 0.5 * h, abs=1e-14)


def test_quick_exact_for_cell_averages_of_monotone_quadratic():
    # The kappa=1/3 upwind-biased interpolant reproduces the point value at the
    # face from the three upstream/downstream cell AVERAGES of a quadratic.
    for _ in range(50):
        a, b, c0 = RNG.normal(size=3)
        b = 10.0 * abs(b) + 5.0 * abs(a) + 1.0  # monotone on [-2, 1]
        avg = lambda lo, hi: (a * (hi**3 - lo**3) / 3 + b * (hi**2 - lo**2) / 2 + c0 * (hi - lo)) / (hi - lo)
        got = oracle.quick(avg(-2, -1), avg(-1, 0), avg(0, 1))
        assert got == pytest.approx(c0, abs=1e-12)


def test_quick_is_bounded_by_neighbours():
    # Flux limiter: the face value never leaves [min(c,d), max(c,d)] (no new extrema).
    for _ in range(2000):
        u, c, d = RNG.normal(size=3)
        f = oracle.quick(u, c, d)
        assert min(c, d) - 1e-15 <= f <= max(c, d) + 1e-15


def _advect_u_y(n, profile, courant, steps):
    """Pure advection through the whole step: a 2D periodic box with u_x = 1
    everywhere and u_y = profile(x). Every term but the x-transport of u_y
    vanishes (u_x uniform, u_y constant along y, so the field stays divergence
    free and the projection does nothing): the oracle's step reduces to the
    limited-QUICK advection of u_y with the Heun scheme at Courant number
    `courant` (nu = 0). Returns the start and final u_y on one row."""
    case = synth.Case("adv", 2, (n, 4, 1), (True, True, False), False, (0.0, 0.0, 0.0), 0.0)
    u = np.zeros((2, 4, n))
    u[0] = 1.0
    u[1][:] = profile(np.arange(n) + 0.5)   # u_y sits at its face's x = i + 1/2
    s = oracle.Sim(case, tol=1e-13, u=u, ue=np.zeros(4))
    for _ in range(steps):
        s.step(courant)
    assert np.abs(s.u[0] - 1.0).max() == 0.0      # the transporting velocity is untouched
    return u[1][0], s.u[1][0]


@pytest.mark.parametrize("courant", [0.1, 0.2])
def test_limited_advection_of_a_square_wave_makes_no_new_extrema(courant):
    # The limiter's purpose: a discontinuity advected for many steps stays
    # within the range of its start values (no overshoot, no undershoot) while
    # its integral is conserved. The step bound median(10c - 9u, c, d) is what
    # keeps the foot of a step from going negative: without it the face value
    # ahead of a rising step is (5c + 2d - u)/6 > c and the cell undershoots at
    # once (a mutated oracle without that bound overshoots by 0.15 here).
    # Courant <= 0.2: the slope bound 10 is the normalised-variable TVD bound
    # 1/Courant of a forward-Euler stage at Courant 0.1 (the Heun scheme is a
    # convex combination of such stages); larger Courant numbers make small
    # new extrema by design of that bound.
    start, end = _advect_u_y(64, lambda x: ((x >= 16) & (x < 32)).astype(float), courant, 200)
    assert end.min() >= -1e-13 and end.max() <= 1.0 + 1e-13, (end.min(), end.max())
    assert end.sum() == pytest.approx(start.sum(), abs=1e-11)
    assert end.max() - end.min() > 0.9                  # still a wave, not smeared flat


def test_limited_advection_of_a_smooth_wave_is_second_order():
    # One period of a sine at Courant 0.2 on 32, 64, 128 cells: the RMS error
    # against the exactly translated sine falls at least 4x per halving of h
    # (measured 2.15 in log2; the limiter clips only at the two extrema, and a
    # tighter slope bound there would drop the order, e.g. to 1.8 without the
    # inner bound's 10c - 9u term).
    errs = []
    for n in (32, 64, 128):
        f = lambda x: np.sin(2 * np.pi * x / n)
        steps = 5 * n
        start, end = _advect_u_y(n, f, 0.2, steps)
        x = np.arange(n) + 0.5
        errs.append(float(np.sqrt(((end - f(x - 0.2 * steps)) ** 2).mean())))
    orders = [math.log2(errs[q] / errs[q + 1]) for q in range(2)]
    assert min(orders) >= 2.0, (errs, orders)


# --------------------------------------------------------- BDIM moments ------
def test_kernel_moments_match_quadrature():
    # 48-point Gauss-Legendre quadrature: the integrands are entire functions
    # on intervals of length <= 2 eps, where it is exact to rounding
    x, w = np.polynomial.legendre.leggauss(48)

    def quad(f, a, b):
        t = 0.5 * (b - a) * x + 0.5 * (b + a)
        return 0.5 * (b - a) * float(np.dot(w, f(t)))

    for eps in (1.0, 1.5, 2.0):
        K = lambda s: (1 + np.cos(np.pi * s / eps)) / (2 * eps)
        for d in np.linspace(-1.2 * eps, 1.2 * eps, 23):
            # mu0 = int_{-eps}^{d} K(s) ds: kernel mass on the fluid side of the face
            lo = -eps
            hi = min(max(d, -eps), eps)
            m0 = quad(K, lo, hi) if hi > lo else 0.0
            if d >= eps:
                m0 = 1.0
            assert oracle.mu0(d, eps) == pytest.approx(m0, abs=1e-13)
            # mu1 = first moment of K over the fluid side, measured from the face:
            # int_{s' > 0} (s' - d) K(s' - d) ds'   (distance d of the face)
            t_lo = max(-d, -eps)
            m1 = quad(lambda t: t * K(t), t_lo, eps) if t_lo < eps else 0.0
            assert oracle.mu1(d, eps) == pytest.approx(m1, abs=1e-13)
            kk = K(d) if abs(d) < eps else 0.0
            assert oracle.kernel(d, eps) == pytest.approx(kk, abs=1e-15)


def test_kernel_moment_symmetries():
    for d in np.linspace(-1.5, 1.5, 31):
        assert oracle.mu0(d) + oracle.mu0(-d) == pytest.approx(1.0, abs=1e-15)
        assert oracle.mu1(d) == pytest.approx(oracle.mu1(-d), abs=1e-15)
    assert oracle.mu1(1.0) == 0.0 and oracle.mu1(-1.0) == 0.0
    assert oracle.mu1(0.0) == pytest.approx(0.25 - 1 / math.pi**2, abs=1e-15)
    assert oracle.mu0(-3.0) == 0.0 and oracle.mu0(3.0) == 1.0


# --------------------------------------------------- convection-diffusion ----
def _linear_field(ndim, n, A, B):
    u = np.zeros((ndim,) + tuple(n[:ndim][::-1]))
    for a in range(ndim):
        X = face_coords(ndim, n, a)
        u[a] = A[a] + sum(B[a][c] * X[c] for c in range(ndim))
    return u


@pytest.mark.parametrize("ndim,n", [(2, (20, 18, 1)), (3, (12, 11, 10))])
def test_conv_diff_exact_for_linear_fields(ndim, n):
    # For linear u the QUICK face value and the advecting-velocity average are
    # exact point values at the face, and the flux difference of the quadratic
    # product is exact: r_a = -sum_b d_b(u_a u_b) = -sum_b (B_ab u_b + u_a B_bb)
    # at the a-face position; diffusion of a linear field is zero.
    A = RNG.normal(size=3)
    B = RNG.normal(size=(3, 3)) * 0.1
    g = oracle.make_grid(ndim, n, (False,) * 3, False, (0, 0, 0), nu=0.37)
    u = _linear_field(ndim, n, A, B)
    r = oracle.conv_diff(g, u, np.zeros(n[1] * n[2]))
    for a in range(ndim):
        X = face_coords(ndim, n, a)
        ua = A[a] + sum(B[a][c] * X[c] for c in range(ndim))
        ub = [A[b] + sum(B[b][c] * X[c] for c in range(ndim)) for b in range(ndim)]
        exact = -sum(B[a][b] * ub[b] + ua * B[b][b] for b in range(ndim))
        sl = tuple(slice(3, -3) for _ in range(ndim))
        np.testing.assert_allclose(r[a][sl], exact[sl], atol=1e-12)


@pytest.mark.parametrize("ndim,n", [(2, (24, 16, 1)), (3, (12, 10, 8))])
def test_conv_diff_conserves_momentum_on_periodic_box(ndim, n):
    g = oracle.make_grid(ndim, n, (True,) * 3, False, (0, 0, 0), nu=0.05)
    u = synth.random_field(3, ndim, n)
    r = oracle.conv_diff(g, u, np.zeros(1))
    for a in range(ndim):
        assert abs(r[a].sum()) <= 1e-13 * np.abs(r[a]).sum()
        assert np.abs(r[a]).max() > 0.1


def test_conv_diff_uniform_field_is_zero():
    n = (10, 9, 8)
    g = oracle.make_grid(3, n, (True,) * 3, False, (0, 0, 0), nu=0.2)
    u = np.zeros((3, 8, 9, 10))
    for a in range(3):
        u[a] = 0.3 + a
    assert np.abs(oracle.conv_diff(g, u, np.zeros(1))).max() == 0.0


def test_conv_diff_shear_mode_diffuses_exactly():
    # u_x = sin(k y), u_y = 0 on a periodic box: convection cancels and the
    # diffusion stencil gives exactly nu (2 cos k - 2) u_x.
    N = 32
    k = 2 * math.pi * 3 / N
    g = oracle.make_grid(2, (N, N, 1), (True, True, False), False, (0, 0, 0), nu=0.11)
    x, y = face_coords(2, (N, N, 1), 0)
    u = np.zeros((2, N, N))
    u[0] = np.sin(k * y)
    r = oracle.conv_diff(g, u, np.zeros(1))
    np.testing.assert_allclose(r[0], 0.11 * (2 * math.cos(k) - 2) * u[0], atol=1e-15)
    assert np.abs(r[1]).max() == 0.0


# ------------------------------------------------------------- BDIM blend ----
def test_bdim_blend_closed_form_for_linear_f():
    ndim, n = 3, (9, 8, 7)
    g = oracle.make_grid(ndim, n, (False,) * 3, False, (0.5, 0, 0), nu=0.0)
    A = RNG.normal(size=3)
    Bm = RNG.normal(size=(3, 3))
    f = _linear_field(ndim, n, A, Bm)
    sh = (7, 8, 9)
    mu0 = RNG.uniform(0, 1, size=(3,) + sh)
    mu1n = RNG.normal(size=(3, 3) + sh)
    V = np.zeros((3,) + sh)
    V[0], V[1], V[2] = 0.2, -0.3, 0.7  # uniform body velocity: grad V = 0
    dt = 0.3
    r = RNG.normal(size=(3,) + sh)
    u0 = f - dt * r
    out = oracle.bdim(g, u0, r, dt, mu0, mu1n, V)
    for a in range(3):
        exact = V[a] + mu0[a] * (f[a] - V[a]) + sum(mu1n[a, b] * Bm[a][b] for b in range(3))
        np.testing.assert_allclose(out[a][1:-1, 1:-1, 1:-1], exact[1:-1, 1:-1, 1:-1], atol=1e-12)
    # lower boundary faces of the non-periodic axes carry U_a
    assert np.all(out[0][:, :, 0] == 0.5) and np.all(out[1][:, 0, :] == 0) and np.all(out[2][0] == 0)


def test_bdim_blend_limits_and_corrector_average():
    ndim, n = 2, (12, 10, 1)
    g = oracle.make_grid(ndim, n, (True, True, False), False, (0, 0, 0), nu=0.0)
    sh = (10, 12)
    u0 = RNG.normal(size=(2,) + sh)
    r = RNG.normal(size=(2,) + sh)
    dt = 0.17
    f = u0 + dt * r
    V = RNG.normal(size=(2,) + sh)
    z = np.zeros((2, 3) + sh)
    # fluid everywhere: f (V + 1*(f - V) is f up to one rounding)
    np.testing.assert_allclose(oracle.bdim(g, u0, r, dt, np.ones((2,) + sh), z, V), f, rtol=0, atol=1e-15 * 8)
    # solid everywhere: exactly V
    assert np.array_equal(oracle.bdim(g, u0, r, dt, np.zeros((2,) + sh), z, V), V)
    # no body at all: f; corrector stage: (u* + f)/2
    us = RNG.normal(size=(2,) + sh)
    np.testing.assert_allclose(oracle.bdim(g, u0, r, dt, ustar=us), 0.5 * (us + f), atol=1e-15)


# --------------------------------------------------------------- bodies ------
def test_sphere_distance_normal_velocity():
    b = synth.Body("sphere", (5.0, 6.0, 7.0), 3.0, heave_amp=2.0, omega=0.3, phase=0.1, heave_axis=1)
    bs = oracle.make_body(b)
    for _ in range(20):
        x = RNG.uniform(0, 12, size=3)
        t = RNG.uniform(0, 10)
        d, nrm, V = oracle.body_eval(bs, 3, x, t)
        c = np.array([5.0, 6.0 + 2.0 * math.sin(0.3 * t + 0.1), 7.0])
        assert d == pytest.approx(np.linalg.norm(x - c) - 3.0, abs=1e-13)
        np.testing.assert_allclose(nrm, (x - c) / np.linalg.norm(x - c), atol=1e-13)
        # velocity = time derivative of the centre (central difference)
        h = 1e-5
        cp = 2.0 * math.sin(0.3 * (t + h) + 0.1)
        cm = 2.0 * math.sin(0.3 * (t - h) + 0.1)
        np.testing.assert_allclose(V, [0, (cp - cm) / (2 * h), 0], atol=1e-9)
        # normal = gradient of the distance (central difference, O(h^2))
        gd = []
        for a in range(3):
            e = np.zeros(3)
            e[a] = 1e-4
            gd.append((oracle.body_eval(bs, 3, x + e, t)[0] - oracle.body_eval(bs, 3, x - e, t)[0]) / 2e-4)
        np.testing.assert_allclose(nrm, gd, atol=1e-7)


def test_cylinder_distance_is_planar_and_its_normal_is_the_gradient():
    # a z-axis cylinder: the distance to the axis minus the radius, the same
    # in every z plane, normal = grad d (central differences) with no z part,
    # velocity = d(centre)/dt of the heave map
    B = synth.Body("cylinder", (20.3, 15.7, 0.0), 4.5, heave_amp=2.0, omega=0.3, phase=0.4, heave_axis=1)
    bs = oracle.make_body(B)
    for _ in range(20):
        x = RNG.uniform(5, 35, size=3)
        t = RNG.uniform(0, 10)
        d, nrm, V = oracle.body_eval(bs, 3, x, t)
        cy = 15.7 + 2.0 * np.sin(0.3 * t + 0.4)
        assert d == pytest.approx(np.hypot(x[0] - 20.3, x[1] - cy) - 4.5, abs=1e-12)
        for z in (0.0, 17.0):
            assert oracle.body_eval(bs, 3, (x[0], x[1], z), t)[0] == pytest.approx(d, abs=1e-12)
        gd = []
        for a in range(3):
            e = np.zeros(3)
            e[a] = 1e-4
            gd.append((oracle.body_eval(bs, 3, x + e, t)[0] - oracle.body_eval(bs, 3, x - e, t)[0]) / 2e-4)
        assert np.allclose(nrm, gd, atol=1e-7) and nrm[2] == 0.0
        h = 1e-5
        vy = (2.0 * np.sin(0.3 * (t + h) + 0.4) - 2.0 * np.sin(0.3 * (t - h) + 0.4)) / (2 * h)
        assert V[1] == pytest.approx(vy, abs=1e-8) and V[0] == 0.0 and V[2] == 0.0


def test_ellipse_reduces_to_circle_and_normal_is_distance_gradient_on_surface():
    circ = oracle.make_body(synth.Body("ellipse", (10.0, 9.0, 0.0), 0.0, (4.0, 4.0), pitch_amp=0.4, omega=0.2))
    for _ in range(20):
        x = np.array(list(RNG.uniform(0, 20, size=2)) + [0.0])
        d, nrm, V = oracle.body_eval(circ, 2, x, RNG.uniform(0, 5))
        r = x[:2] - np.array([10.0, 9.0])
        assert d == pytest.approx(np.linalg.norm(r) - 4.0, abs=1e-12)
        np.testing.assert_allclose(nrm[:2], r / np.linalg.norm(r), atol=1e-12)
    # thin pitched, heaving ellipse: on the surface the normal equals grad d,
    # and the velocity is the rigid motion of the surface point.
    b = synth.Body("ellipse", (10.0, 9.0, 0.0), 0.0, (8.0, 1.5), heave_amp=1.0, pitch_amp=0.3, omega=0.4)
    bs = oracle.make_body(b)
    t = 0.7
    th = 0.3 * math.sin(0.4 * t + math.pi / 2)
    yc = 9.0 + math.sin(0.4 * t)
    for phi in np.linspace(0, 2 * math.pi, 13)[:-1]:
        p_body = np.array([8.0 * math.cos(phi), 1.5 * math.sin(phi)])
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        x = np.array(list(R @ p_body + [10.0, yc]) + [0.0])
        d, nrm, V = oracle.body_eval(bs, 2, x, t)
        assert abs(d) < 1e-12
        gd = []
        for a in range(2):
            e = np.zeros(3)
            e[a] = 1e-5
            gd.append((oracle.body_eval(bs, 2, x + e, t)[0] - oracle.body_eval(bs, 2, x - e, t)[0]) / 2e-5)
        np.testing.assert_allclose(nrm[:2], gd, atol=1e-6)
        # rigid-body velocity: finite difference of the material point's position
        h = 1e-6
        def pos(tt):
            tht = 0.3 * math.sin(0.4 * tt + math.pi / 2)
            Rt = np.array([[math.cos(tht), -math.sin(tht)], [math.sin(tht), math.cos(tht)]])
            return Rt @ p_body + [10.0, 9.0 + math.sin(0.4 * tt)]
        np.testing.assert_allclose(V[:2], (pos(t + h) - pos(t - h)) / (2 * h), atol=1e-7)


def test_measure_places_bodies_on_face_centres():
    n = (16, 12, 1)
    g = oracle.make_grid(2, n, (False,) * 3, True, (1, 0, 0), nu=0.01)
    b = synth.Body("sphere", (7.3, 5.9, 0.0), 3.1)
    mu0, mu1n, V = oracle.measure(g, oracle.make_body(b), 0.0)
    for a in range(2):
        X = face_coords(2, n, a)
        d = np.sqrt((X[0] - 7.3) ** 2 + (X[1] - 5.9) ** 2) - 3.1
        exp0 = np.vectorize(oracle.mu0)(d)
        # reading: a face whose mu0 is below 1e-5 is solid (mu0 = 0)
        exp0 = np.where(exp0 < 1e-5, 0.0, exp0)
        np.testing.assert_allclose(mu0[a], exp0, atol=1e-15)
        m1 = np.vectorize(oracle.mu1)(d)
        nb = [(X[0] - 7.3) / (d + 3.1), (X[1] - 5.9) / (d + 3.1)]
        for bb in range(2):
            np.testing.assert_allclose(mu1n[a, bb], m1 * nb[bb], atol=1e-14)
        assert np.abs(mu1n[a, 2]).max() == 0.0


# --------------------------------------------------------------- Poisson -----
def test_poisson_operator_on_quadratic_and_constants():
    n = (14, 12, 10)
    g = oracle.make_grid(3, n, (False,) * 3)
    c = oracle.coeffs(g)
    z, y, x = np.meshgrid(*[np.arange(m) + 0.5 for m in n[::-1]], indexing="ij")
    p = 0.5 * x**2 - 1.5 * y**2 + 2.0 * z**2 + 3 * x * y
    Ap = oracle.poisson_apply(g, c, p)
    np.testing.assert_allclose(Ap[1:-1, 1:-1, 1:-1], 1.0 - 3.0 + 4.0, atol=1e-10)
    gp = oracle.make_grid(3, n, (True,) * 3)
    for gg in (g, gp):
        cc = oracle.coeffs(gg) * RNG.uniform(0.1, 1.0, size=(3,) + n[::-1])
        assert np.abs(oracle.poisson_apply(gg, cc, np.full(n[::-1], 3.3))).max() < 1e-14


def test_poisson_operator_symmetric_and_semidefinite():
    for per in ((True, False, False), (False, True, True)):
        n = (9, 8, 6)
        g = oracle.make_grid(3, n, per)
        c = oracle.coeffs(g) * RNG.uniform(0.0, 1.0, size=(3,) + n[::-1])
        p, q = RNG.normal(size=n[::-1]), RNG.normal(size=n[::-1])
        Ap, Aq = oracle.poisson_apply(g, c, p), oracle.poisson_apply(g, c, q)
        assert np.vdot(Ap, q) == pytest.approx(np.vdot(p, Aq), rel=1e-12)
        assert np.vdot(Ap, p) < 0


def test_poisson_operator_is_divergence_of_weighted_gradient():
    # The operator must be exactly div(c grad p) built from the projection's
    # own gradient update and divergence: that is what makes the projected
    # velocity discretely divergence-free.
    for per, ex in (((True, True, True), False), ((False, False, False), True)):
        n = (10, 9, 8)
        g = oracle.make_grid(3, n, per, ex, (1.0, 0, 0))
        c = oracle.coeffs(g) * RNG.uniform(0.2, 1.0, size=(3,) + n[::-1])
        p = RNG.normal(size=n[::-1])
        u0 = np.zeros((3,) + n[::-1])
        ue = np.zeros(n[1] * n[2])
        g2 = oracle.make_grid(3, n, per, ex, (0, 0, 0))
        u1 = oracle.grad_update(g2, c, p, 0.7, u0)
        div = oracle.divergence(g2, u1, ue)
        np.testing.assert_allclose(-div / 0.7, oracle.poisson_apply(g2, c, p), atol=1e-12)


def _dense_matrix(g, c):
    n = g.n[0] * g.n[1] * g.n[2]
    sh = oracle._shape(g)
    M = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        M[:, q] = oracle.poisson_apply(g, c, e.reshape(sh)).ravel()
    return M


@pytest.mark.parametrize("per,body", [((True, True, False), False), ((False, False, False), False),
                                      ((False, False, False), True), ((True, False, False), True)])
def test_multigrid_matches_dense_solve(per, body):
    N = 16
    g = oracle.make_grid(2, (N, N, 1), per, False, (0, 0, 0), nu=0.0)
    mu0 = None
    if body:
        mu0, _, _ = oracle.measure(g, oracle.make_body(synth.Body("sphere", (7.7, 8.2, 0), 3.3)), 0.0)
    c = oracle.coeffs(g, mu0)
    b = synth.random_scalar(5, 2, (N, N, 1))
    p, rc, st = oracle.poisson_solve(g, c, b, tol=1e-13, itmax=100)
    assert rc == 0 and oracle.mg_levels(g) == 3
    M = _dense_matrix(g, c)
    D = np.diag(M)
    act = D != 0
    bb = b.ravel().copy()
    bb[act] -= bb[act].mean()
    bb[~act] = 0
    x = np.linalg.lstsq(M[np.ix_(act, act)], bb[act], rcond=None)[0]
    x -= x.mean()
    np.testing.assert_allclose(p.ravel()[act], x, atol=1e-11 * np.abs(x).max())
    assert np.all(p.ravel()[~act] == 0)


def test_multigrid_level_rule():
    assert oracle.mg_levels(oracle.make_grid(2, (128, 64, 1))) == 5          # ... 8x4
    assert oracle.mg_levels(oracle.make_grid(3, (256, 128, 128))) == 6       # ... 8x4x4
    assert oracle.mg_levels(oracle.make_grid(3, (64, 64, 64))) == 5          # ... 4^3
    assert oracle.mg_levels(oracle.make_grid(2, (70, 36, 1))) == 2           # 35x18, then odd: stop
    assert oracle.mg_levels(oracle.make_grid(2, (35, 18, 1))) == 1           # odd side: single level
    assert oracle.mg_levels(oracle.make_grid(2, (40, 24, 1))) == 3           # 20x12, 10x6


def test_multigrid_convergence_is_grid_independent():
    # the textbook property of multigrid: the V-cycles needed for a fixed
    # residual reduction do not grow with the grid (a single-level smoother
    # would need O(N) times more), for periodic and walled boxes in 2D and 3D
    counts = []
    for nd, sizes in ((2, (32, 64, 128, 256)), (3, (16, 32, 64))):
        for N in sizes:
            n = (N, N, N if nd == 3 else 1)
            for per in ((True,) * 3, (False,) * 3):
                g = oracle.make_grid(nd, n, per)
                p, rc, st = oracle.poisson_solve(g, oracle.coeffs(g, None), synth.random_scalar(5, nd, n),
                                                 tol=1e-10, itmax=100)
                assert rc == 0 and st.rel_resid <= 1e-10
                counts.append(st.vcycles)
    assert max(counts) <= 14 and max(counts) - min(counts) <= 2, counts


def test_projection_leaves_discretely_divergence_free_field():
    case = synth.config1_circle((48, 32)).with_(body=synth.Body("sphere", (14.0, 15.5, 0.0), 5.0))
    g = oracle.grid_from_case(case)
    mu0, _, _ = oracle.measure(g, oracle.make_body(case.body), 0.0)
    c = oracle.coeffs(g, mu0)
    u = synth.random_field(9, 2, case.n, 0.5, (1.0, 0.0, 0.0))
    u *= mu0  # inside the solid the blended velocity is the body's (here at rest)
    u[0][:, 0] = 1.0
    u[1][0, :] = 0.0
    ue = np.full(case.n[1], 1.0) + 0.1 * synth.random_scalar(3, 2, (case.n[1], 1, 1)).ravel()
    ue += (u[0][:, 0].sum() - ue.sum()) / ue.size  # zero net boundary flux
    u1, P, rc, st = oracle.project(g, c, u, ue, np.zeros((32, 48)), 1.0, 0.3, tol=1e-13)
    assert rc == 0
    div = oracle.divergence(g, u1, ue)
    assert np.abs(div).max() < 1e-10
    assert np.abs(oracle.divergence(g, u, ue)).max() > 0.1
    # a projection is idempotent: projecting the result again changes nothing
    u2, P2, rc, st = oracle.project(g, c, u1, ue, np.zeros((32, 48)), 1.0, 0.3, tol=1e-13)
    assert rc == 0
    assert np.abs(u2 - u1).max() < 1e-10 * np.abs(u1).max()
    assert np.abs(P2).max() < 1e-8 * np.abs(P).max()


# ----------------------------------------------------- exit, CFL, forces -----
def test_exit_condition_zeroes_net_flux_and_keeps_uniform_flow():
    n = (20, 10, 6)
    g = oracle.make_grid(3, n, (False,) * 3, True, (1.0, 0, 0), nu=0.01)
    u = synth.random_field(2, 3, n, 0.2, (1.0, 0, 0))
    u[0][:, :, 0] = 1.0
    u[1][:, 0, :] = 0.0
    u[2][0] = 0.0
    ue0 = 1.0 + 0.1 * RNG.normal(size=n[1] * n[2])
    ue = oracle.exit_bc(g, ue0, u, ue0, 0.4, 0, None, u, ue0)
    div = oracle.divergence(g, u, ue)
    assert abs(div.sum()) < 1e-11
    # uniform flow: the exit condition changes nothing
    uu = np.zeros((3,) + n[::-1])
    uu[0] = 1.0
    e1 = np.ones(n[1] * n[2])
    assert np.allclose(oracle.exit_bc(g, e1, uu, e1, 0.4, 0, None, uu, e1), 1.0, atol=1e-15)


def test_exit_update_is_first_order_upwind_up_to_a_uniform_shift():
    # du/dt + U du/dx = 0 on the exit plane, upwind against the last interior
    # u_x face, one Heun stage at a time; the mass correction only adds the
    # same constant to every exit face, so the mean-free part of the result is
    # the closed form of the upwind update
    n = (12, 7, 5)
    Ux, dt = 1.3, 0.4
    g = oracle.make_grid(3, n, (False,) * 3, True, (Ux, 0, 0), nu=0.01)
    u = synth.random_field(4, 3, n, 0.3, (1.0, 0, 0))
    last = u[0][:, :, n[0] - 1].ravel()          # plane index j + n1 k
    ue0 = 1.0 + 0.1 * RNG.normal(size=n[1] * n[2])
    ueG = 1.0 + 0.1 * RNG.normal(size=n[1] * n[2])
    ue = oracle.exit_bc(g, ue0, u, ueG, dt, 0, None, u, ue0)
    want = ue0 - dt * Ux * (ueG - last)
    np.testing.assert_allclose(ue - ue.mean(), want - want.mean(), atol=1e-13)
    us = 1.0 + 0.1 * RNG.normal(size=n[1] * n[2])  # predictor's exit plane
    ue = oracle.exit_bc(g, ue0, u, ueG, dt, 1, us, u, ue0)
    want = 0.5 * (us + ue0 - dt * Ux * (ueG - last))
    np.testing.assert_allclose(ue - ue.mean(), want - want.mean(), atol=1e-13)


def test_cfl_closed_form_on_uniform_field():
    n = (8, 7, 6)
    g = oracle.make_grid(3, n, (True,) * 3, False, (0, 0, 0), nu=0.05)
    u = np.zeros((3,) + n[::-1])
    u[0], u[1], u[2] = 0.7, -0.4, 0.2
    assert oracle.cfl(g, u, np.zeros(1), 1.0, 10.0) == pytest.approx(1 / (1.3 + 0.25), rel=1e-15)
    assert oracle.cfl(g, u, np.zeros(1), 1.0, 0.1) == 0.1


def test_pressure_force_invariants():
    # uniform pressure: no net force; linear hydrostatic pressure p = g y:
    # F = -integral(grad p) over the body = -g * area e_y (Archimedes), O(h^2).
    n = (64, 64, 1)
    g = oracle.make_grid(2, n, (False,) * 3)
    R = 10.0
    bs = oracle.make_body(synth.Body("sphere", (31.3, 32.6, 0), R))
    F = oracle.forces(g, bs, 0.0, np.full((64, 64), 2.5))
    assert np.abs(F).max() < 1e-3 * 2.5 * 2 * math.pi * R
    y = np.arange(64)[:, None] + 0.5 + 0 * np.arange(64)[None, :]
    F = oracle.forces(g, bs, 0.0, 0.8 * y)
    assert F[1] == pytest.approx(-0.8 * math.pi * R * R, rel=5e-3)
    assert abs(F[0]) < 1e-2 * abs(F[1])
    n3 = (40, 40, 40)
    g3 = oracle.make_grid(3, n3, (False,) * 3)
    bs3 = oracle.make_body(synth.Body("sphere", (19.6, 20.3, 20.1), 8.0))
    z = np.arange(40)[:, None, None] + 0.5 + 0 * np.ones(n3)
    F3 = oracle.forces(g3, bs3, 0.0, 1.3 * z)
    assert F3[2] == pytest.approx(-1.3 * 4 / 3 * math.pi * 8.0**3, rel=5e-3)


def test_viscous_force_closed_forms():
    # the viscous traction nu (grad u + grad u^T) . n over the body:
    # * rigid motion (translation + rotation) has no strain: F = 0 to rounding;
    # * a linear field u = M x has constant strain, so F = nu (M + M^T) sum K n,
    #   and sum K n vanishes over a closed surface (O(h^2));
    # * u_x = gam y^2 has strain 2 gam y in the xy pair, so by the divergence
    #   theorem F_x = 2 nu gam * area (the body's volume in 3D), F_y ~ 0;
    #   u_x = gam x^2 has normal strain 4 gam x, F_x = 4 nu gam * area.
    nu, R = 0.05, 10.0
    g = oracle.make_grid(2, (64, 64, 1), (False,) * 3, nu=nu)
    bs = oracle.make_body(synth.Body("sphere", (31.3, 32.6, 0), R))
    ue = np.zeros(64)
    X = [face_coords(2, (64, 64), a) for a in range(2)]
    om, x0, y0 = 0.37, 20.0, 41.0
    u = np.stack([1.3 - om * (X[0][1] - y0), -0.4 + om * (X[1][0] - x0)])
    assert np.abs(oracle.forces_viscous(g, bs, 0.0, u, ue)).max() < 1e-12
    M = np.array([[0.2, 0.5], [-0.1, -0.2]])
    u = np.stack([M[0, 0] * X[0][0] + M[0, 1] * X[0][1], M[1, 0] * X[1][0] + M[1, 1] * X[1][1]])
    F = oracle.forces_viscous(g, bs, 0.0, u, ue)
    assert np.abs(F).max() < 1e-3 * nu * np.abs(M + M.T).max() * 2 * math.pi * R
    gam = 0.02
    u = np.stack([gam * X[0][1] ** 2, np.zeros((64, 64))])
    F = oracle.forces_viscous(g, bs, 0.0, u, ue)
    assert F[0] == pytest.approx(2 * nu * gam * math.pi * R * R, rel=5e-3)
    assert abs(F[1]) < 1e-2 * abs(F[0])
    # u_x = gam x^2: the normal strain 2 d_x u_x = 4 gam x -> F_x = 4 nu gam * area
    u = np.stack([gam * X[0][0] ** 2, np.zeros((64, 64))])
    F = oracle.forces_viscous(g, bs, 0.0, u, ue)
    assert F[0] == pytest.approx(4 * nu * gam * math.pi * R * R, rel=5e-3)
    assert abs(F[1]) < 1e-2 * abs(F[0])
    # 3D sphere: u_x = gam z^2 -> F_x = 2 nu gam (4/3) pi R^3; a rotation -> 0
    n3 = (40, 40, 40)
    g3 = oracle.make_grid(3, n3, (False,) * 3, nu=nu)
    bs3 = oracle.make_body(synth.Body("sphere", (19.6, 20.3, 20.1), 8.0))
    X3 = [face_coords(3, n3, a) for a in range(3)]
    u3 = np.stack([gam * X3[0][2] ** 2, np.zeros(n3), np.zeros(n3)])
    F3 = oracle.forces_viscous(g3, bs3, 0.0, u3, np.zeros(40 * 40))
    assert F3[0] == pytest.approx(2 * nu * gam * 4 / 3 * math.pi * 8.0**3, rel=5e-3)
    assert np.abs(F3[1:]).max() < 1e-2 * abs(F3[0])
    w = np.array([0.1, -0.3, 0.2])   # u = w x (x - c)
    c = np.array([15.0, 22.0, 18.0])
    r = [[X3[a][b] - c[b] for b in range(3)] for a in range(3)]
    u3 = np.stack([w[1] * r[0][2] - w[2] * r[0][1], w[2] * r[1][0] - w[0] * r[1][2], w[0] * r[2][1] - w[1] * r[2][0]])
    assert np.abs(oracle.forces_viscous(g3, bs3, 0.0, u3, np.zeros(40 * 40))).max() < 1e-12


def test_diagnostics_closed_form_on_2d_tgv():
    N = 24
    case = synth.Case("t", 2, (N, N, 1), (True, True, False), False, (0, 0, 0), 0.01, init="tgv2d")
    u, ue = synth.initial_velocity(case)
    ke, ens = oracle.diagnostics(oracle.grid_from_case(case), u, ue)
    k = 2 * math.pi / N
    assert ke == pytest.approx(math.cos(k / 2) ** 2 / 4, rel=1e-13)
    assert ens == pytest.approx(4 * math.sin(k / 2) ** 2, rel=1e-13)


# ------------------------------------------------------------------- step ----
def test_step_keeps_uniform_flow():
    case = synth.Case("u", 3, (8, 8, 8), (True,) * 3, False, (0, 0, 0), 0.05, init="uniform+noise",
                      noise_amp=0.0)
    s = oracle.Sim(case, u=np.stack([np.full((8, 8, 8), v) for v in (0.3, -0.2, 0.1)]), ue=np.zeros(64))
    u0 = s.u.copy()
    for _ in range(3):
        s.step(0.5)
    np.testing.assert_allclose(s.u, u0, atol=1e-14)


def test_step_keeps_uniform_channel_flow_with_exit():
    case = synth.Case("ch", 2, (24, 12, 1), (False, False, False), True, (1.0, 0, 0), 0.02,
                      init="uniform+noise", noise_amp=0.0)
    s = oracle.Sim(case)
    u0 = s.u.copy()
    for _ in range(3):
        s.step(0.5)
    np.testing.assert_allclose(s.u, u0, atol=1e-13)
    np.testing.assert_allclose(s.ue, 1.0, atol=1e-13)


def test_step_conserves_momentum_on_periodic_box():
    n = (16, 12, 10)
    case = synth.Case("p", 3, n, (True,) * 3, False, (0, 0, 0), 0.03, init="noise", noise_amp=0.3, seed=11)
    s = oracle.Sim(case)
    # project the random start so the step starts from a divergence-free field
    g = s.g
    c = oracle.coeffs(g)
    s.u, _, _, _ = oracle.project(g, c, s.u, s.ue, np.zeros(n[::-1]), 1.0, 1.0, tol=1e-13)
    m0 = s.u.sum(axis=(1, 2, 3))
    for _ in range(3):
        s.step(0.6)
    m1 = s.u.sum(axis=(1, 2, 3))
    np.testing.assert_allclose(m1, m0, atol=1e-12)
    assert max(st[1] for st in s.stats) < 1e-10 and max(st[3] for st in s.stats) < 1e-10


def test_tgv3d_keeps_reflection_symmetries():
    # The TGV start is odd in x for u and even in z for (u, v), with w = 0;
    # the Navier-Stokes equations keep both reflection symmetries, and so must
    # the discrete step (staggered reflection maps faces i -> -i, cells i -> N-1-i).
    N = 16
    case = synth.config2_tgv(N)
    s = oracle.Sim(case)
    for _ in range(3):
        s.step(0.5)
    u, v, w = s.u
    fi = (-np.arange(N)) % N
    ci = N - 1 - np.arange(N)
    # x reflection: u odd about faces, v and w even about cells (x is the last axis)
    np.testing.assert_allclose(u, -u[:, :, fi], atol=1e-9)
    np.testing.assert_allclose(v, v[:, :, ci], atol=1e-9)
    np.testing.assert_allclose(w, w[:, :, ci], atol=1e-9)
    # z reflection: w odd about faces, u and v even about cells (z is the first axis)
    np.testing.assert_allclose(u, u[ci], atol=1e-9)
    np.testing.assert_allclose(v, v[ci], atol=1e-9)
    np.testing.assert_allclose(w, -w[fi], atol=1e-9)
    assert np.abs(w).max() > 1e-4


def test_tgv_octant_start_is_the_full_field_on_its_mirror_planes():
    # the octant start equals the full-period field on the first octant, and
    # the normal velocity vanishes on every wall (the field's mirror planes)
    N = 24
    uo, _ = synth.initial_velocity(synth.tgv_octant(N))
    uf, _ = synth.initial_velocity(synth.config2_tgv(N))
    h = N // 2
    assert np.abs(uo - uf[:, :h, :h, :h]).max() < 1e-14
    assert np.abs(uo[0][:, :, 0]).max() == 0.0 and np.abs(uo[1][:, 0, :]).max() == 0.0
    assert np.abs(uf[0][:h, :h, h]).max() < 1e-12 and np.abs(uf[1][:h, h, :h]).max() < 1e-12


def test_heun_step_is_second_order_in_time():
    # on a fixed grid, the step's error against a small-dt run falls 4x per
    # halving of dt (Heun is second order; a forward-Euler slip, e.g. a lost
    # corrector average, would give 2x)
    N = 32
    case = synth.Case("tgv2d", 2, (N, N, 1), (True, True, False), False, (0.0, 0.0, 0.0), 0.02,
                      synth.Body("none", (0, 0, 0), 0.0), init="tgv2d")

    def run(dt, T=2.0):
        u, ue = synth.initial_velocity(case)
        s = oracle.Sim(case, tol=1e-13, u=u, ue=ue)
        for _ in range(int(round(T / dt))):
            s.step(dt)
        return s.u.copy()

    ref = run(0.0125)
    e = [np.abs(run(dt) - ref).max() for dt in (0.2, 0.1, 0.05)]
    assert e[0] / e[1] > 3.5 and e[1] / e[2] > 3.5, e


def test_tgv2d_decay_converges_at_second_order_or_better():
    # 2D Taylor-Green: exact Navier-Stokes solution whose kinetic energy decays
    # as exp(-4 nu k^2 t). The discrete decay rate error must fall by >= 4x per
    # grid halving (second order) at fixed Reynolds and Courant numbers.
    errs = []
    for N in (16, 32, 64):
        k = 2 * math.pi / N
        nu = 1.0 / (50.0 * k)
        case = synth.Case("t", 2, (N, N, 1), (True, True, False), False, (0, 0, 0), nu, init="tgv2d")
        s = oracle.Sim(case, tol=1e-10)
        ke0, _ = oracle.diagnostics(s.g, s.u, s.ue)
        t_end = 0.1 / (nu * k * k)
        steps = int(round(t_end / 0.4))
        for _ in range(steps):
            s.step(t_end / steps)
        ke, _ = oracle.diagnostics(s.g, s.u, s.ue)
        lam = -math.log(ke / ke0) / (4 * t_end)
        errs.append(abs(lam / (nu * k * k) - 1))
    assert errs[0] < 0.15
    assert errs[1] < errs[0] / 4 and errs[2] < errs[1] / 4, errs


def test_paper_benchmark_grid_sizes():
    # Sec. 4 lists the benchmark grids in millions of cells (golden file).
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_benchmark_dof.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for case, L, dofM in rows:
        L = int(L)
        shape = {"tgv": (L, L, L), "sphere": (16 * L, 6 * L, 6 * L), "cylinder": (9 * L, 6 * L, 2 * L)}[case]
        assert round(np.prod(shape) / 1e6, 2) == float(dofM)


# ----------------------------------------------------------------- threads ---
def test_results_do_not_depend_on_the_thread_count():
    # The per-cell loops run on OpenMP threads and every sum over cells uses a
    # fixed blocked order, so one thread and all host cores give bitwise the
    # same velocity, exit plane, pressure and solver statistics (a sphere in a
    # walled channel with an exit: measure, blend, exit condition and a
    # multigrid whose level sums span several reduction blocks).
    case = synth.config3_sphere((48, 24, 24), D=8.0, centre=(14.3, 11.7, 12.2))
    runs = []
    cores = max(oracle.host_cores(), 4)
    try:
        for th in (1, cores):
            oracle.set_threads(th)
            s = oracle.Sim(case, tol=1e-9)
            for _ in range(2):
                s.step()
            runs.append((s.u.copy(), s.ue.copy(), s.P.copy(), list(s.stats), s.dt))
    finally:
        oracle.set_threads(oracle.host_cores())
    (u1, e1, p1, st1, dt1), (u2, e2, p2, st2, dt2) = runs
    assert np.array_equal(u1, u2) and np.array_equal(e1, e2) and np.array_equal(p1, p2)
    assert st1 == st2 and dt1 == dt2


def test_measure_cuts_the_kernel_tail_so_no_cell_is_nearly_solid():
    # reading: faces with mu0 below 1e-5 count as solid, so every cell's face
    # coefficients sum to 0 or to at least 1e-5 (a cell with a tiny nonzero sum
    # has a pressure fixed only by rounding / that sum); faces in the cut band
    # exist for this body and are zeroed, the others keep mu0(d)
    n = (48, 40, 1)
    g = oracle.make_grid(2, n, (False,) * 3, True, (1, 0, 0), nu=0.01)
    b = synth.Body("sphere", (21.37, 19.61, 0.0), 9.3)
    mu0, _, _ = oracle.measure(g, oracle.make_body(b), 0.0)
    raw = []
    for a in range(2):
        X = face_coords(2, n, a)
        d = np.sqrt((X[0] - 21.37) ** 2 + (X[1] - 19.61) ** 2) - 9.3
        raw.append(np.vectorize(oracle.mu0)(d))
    raw = np.stack(raw)
    tiny = (raw > 0) & (raw < 1e-5)
    assert tiny.any()
    assert (mu0[tiny] == 0).all() and np.array_equal(mu0[~tiny], raw[~tiny])
    c = oracle.coeffs(g, mu0)
    csum = c[0] + np.roll(c[0], -1, axis=1) + c[1] + np.roll(c[1], -1, axis=0)
    assert not ((csum > 0) & (csum < 1e-5)).any()


def test_sim_takes_the_first_then_the_cfl_time_step():
    # reading 10: the first step is dt0, the next min(dt_max, cfl / (max
    # outflux + 5 nu)); a uniform stream U = 1 along x has outflux 1 per cell
    case = synth.Case("u", 2, (32, 16), (False, False), True, (1.0, 0.0), 0.05, init="uniform+noise",
                      noise_amp=0.0)
    s = oracle.Sim(case, tol=1e-12)
    assert s.dt == case.dt0 == 0.25
    s.step()
    assert s.dt == pytest.approx(min(case.dt_max, case.cfl / (1.0 + 5.0 * case.nu)), rel=1e-12)


def test_sim_moves_a_body_on_its_own_clock():
    # two steps of a heaving circle through Sim equal two explicit steps with
    # the body measured at t = 0.2 and t = 0.5, and its clock reads 0.5
    body = synth.Body("sphere", (12.0, 12.0, 0.0), 4.0, heave_amp=2.0, omega=0.3, heave_axis=1)
    case = synth.Case("m", 2, (40, 24), (False, False), True, (1.0, 0.0), 0.02, body, init="noise", seed=2)
    s = oracle.Sim(case, tol=1e-12)
    u0, ue0, P0 = s.u.copy(), s.ue.copy(), s.P.copy()
    s.step(0.2)
    s.step(0.3)
    assert s.t == pytest.approx(0.5, abs=1e-15)
    u1, ue1, P1 = oracle.step_fn(s.g, s.b, 0.0, 0.2, u0, ue0, P0, tol=1e-12)
    u2, _, _ = oracle.step_fn(s.g, s.b, 0.2, 0.3, u1, ue1, P1, tol=1e-12)
    assert np.abs(s.u - u2).max() < 1e-9


def test_sim_starts_with_the_free_stream_on_inflow_and_wall_faces():
    # config 1: noise everywhere, then the lower normal faces of the
    # non-periodic axes carry U (inflow u_x = 1 at x = 0, wall u_y = 0 at y = 0)
    case = synth.config1_circle()
    s = oracle.Sim(case)
    u, v = s.u[0], s.u[1]                       # [y, x]
    assert np.all(u[:, 0] == 1.0) and np.all(v[0, :] == 0.0)
    assert np.abs(u[:, 1:] - 0.0).max() <= case.noise_amp and np.abs(u[:, 1:]).max() > 0
