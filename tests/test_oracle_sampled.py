"""Pins of the oracle's sampled-body functions (a body given by samples of its
distance function and motion, Sec. 3): they must reproduce the analytic
bodies exactly where the samples come from the same shape, and the solid they
describe must have the area of the shape, composite shapes included (the body
arithmetic of Sec. 6)."""
import math

import numpy as np
import pytest

import oracle
import synth


def _grid(ndim, n, eps=1.0, nu=0.0):
    return oracle.make_grid(ndim, n[:ndim], eps=eps, nu=nu)


@pytest.mark.parametrize("ndim", [2, 3])
def test_sampled_sphere_reproduces_the_analytic_measure(ndim):
    # the same sphere given as a formula (orc_measure) and as face samples
    # (orc_measure_sampled): identical moments and velocities, bit for bit
    n = (40, 28, 22) if ndim == 3 else (48, 36, 1)
    centre = (17.3, 13.6, 10.9)
    body = synth.Body("sphere", centre, 7.5)
    g = _grid(ndim, n, eps=1.5)
    mu0a, mu1a, Va = oracle.measure(g, oracle.make_body(body), 0.0)
    d, nf, V, dc, nc = synth.sample_body(synth.Circle(centre, 7.5), ndim, n)
    mu0s, mu1s, Vs = oracle.measure_sampled(g, d, nf, V)
    assert np.array_equal(mu0s, mu0a)
    assert np.array_equal(mu1s, mu1a)
    assert np.array_equal(Vs, Va)
    assert (mu0a < 1).sum() > 100        # the body crosses many faces


def test_sampled_forces_reproduce_the_analytic_forces():
    # pressure force, viscous force and dF/dp from centre samples of a circle
    # equal the analytic body's on arbitrary fields
    n = (48, 40, 1)
    centre = (21.2, 19.7, 0.0)
    g = _grid(2, n, eps=2.0, nu=0.01)
    b = oracle.make_body(synth.Body("sphere", centre, 8.0))
    _, _, _, dc, nc = synth.sample_body(synth.Circle(centre, 8.0), 2, n)
    p = synth.random_scalar(3, 2, n)
    u = synth.random_field(4, 2, n)
    ue = np.zeros(oracle.plane_size(g))
    assert np.array_equal(oracle.forces_sampled(g, dc, nc, p), oracle.forces(g, b, 0.0, p))
    assert np.array_equal(oracle.forces_viscous_sampled(g, dc, nc, u, ue), oracle.forces_viscous(g, b, 0.0, u, ue))
    for axis in range(2):
        assert np.array_equal(oracle.force_dp_sampled(g, dc, nc, axis), oracle.force_dp(g, b, 0.0, axis))


def _solid_area(shape, n, eps):
    # sum over the x-faces of 1 - mu0: each face stands for a unit cell of
    # area, and the smoothed Heaviside integrates the solid to O(eps^2) at
    # corners (exact for a straight edge, O(eps^2 curvature) on a smooth one)
    g = _grid(2, n, eps=eps)
    d, nf, V, _, _ = synth.sample_body(shape, 2, n)
    mu0, _, _ = oracle.measure_sampled(g, d, nf, V)
    return float((1.0 - mu0[0]).sum()), float((1.0 - mu0[1]).sum())


@pytest.mark.parametrize("eps", [1.0, 2.0])
def test_union_of_overlapping_circles_has_the_lens_area(eps):
    # two circles of radius R whose centres are s apart: area 2 pi R^2 minus
    # the lens 2 R^2 acos(s / 2R) - (s / 2) sqrt(4 R^2 - s^2); the two concave
    # corners where the circles meet are smoothed by at most ~eps^2 / 2 each
    R, s = 10.0, 12.0
    shape = synth.Circle((25.3, 23.7), R) + synth.Circle((25.3 + s, 23.7), R)
    lens = 2 * R * R * math.acos(s / (2 * R)) - 0.5 * s * math.sqrt(4 * R * R - s * s)
    A = 2 * math.pi * R * R - lens
    for area in _solid_area(shape, (64, 48, 1), eps):
        assert abs(area - A) <= 1.0 * eps * eps, (area, A)


@pytest.mark.parametrize("eps", [1.0, 2.0])
def test_circle_minus_half_plane_has_the_half_disc_area(eps):
    # a circle minus the half-plane above its centre line: a half disc of area
    # pi R^2 / 2 with two convex corners
    R = 10.0
    shape = synth.Circle((25.3, 23.7), R) - synth.HalfSpace((25.3, 23.7), (0.0, 1.0))
    for area in _solid_area(shape, (64, 48, 1), eps):
        assert abs(area - math.pi * R * R / 2) <= 1.0 * eps * eps, area


@pytest.mark.parametrize("eps", [1.0, 2.0])
@pytest.mark.parametrize("R", [9.0, 14.0])
def test_circle_area_has_the_closed_form_smoothing_term(R, eps):
    # with the exact distance of a circle the area element is (R + d) dd dtheta,
    # and 1 - mu0(d) minus the sharp indicator is odd in d, so the smoothed area
    # is pi R^2 + 4 pi int_0^eps (1 - mu0(d)) d dd = pi R^2 + 2 pi eps^2 (1/6 -
    # 1/pi^2), independent of R; the face sum is a midpoint rule of it
    extra = 2 * math.pi * eps * eps * (1.0 / 6.0 - 1.0 / math.pi ** 2)
    for area in _solid_area(synth.Circle((40.4, 20.2), R), (96, 40, 1), eps):
        assert abs(area - math.pi * R * R - extra) < 0.02, (area, math.pi * R * R + extra)


def test_far_apart_union_measures_as_each_circle():
    # a union of two circles far apart measures, around each, exactly as that
    # circle alone
    R = 9.0
    n = (96, 40, 1)
    a, b = synth.Circle((20.4, 20.2), R), synth.Circle((70.6, 19.1), R)
    g = _grid(2, n, eps=1.0)
    mu = [oracle.measure_sampled(g, *synth.sample_body(s, 2, n)[:3]) for s in (a + b, a, b)]
    left = (slice(None), slice(0, 45))
    right = (slice(None), slice(45, None))
    for k in range(3):   # mu0, mu1n, V
        assert np.array_equal(mu[0][k][..., left[1]], mu[1][k][..., left[1]])
        assert np.array_equal(mu[0][k][..., right[1]], mu[2][k][..., right[1]])


def test_spinning_circle_velocity_is_a_rigid_rotation():
    # the spinning circle's face velocity (the map rot(w t)(x - c)) is
    # w (y - c_y, -(x - c_x)): perpendicular to x - c with |V| = w |x - c|
    w, c = 0.3, (20.5, 18.25)
    n = (40, 36, 1)
    d, nf, V, _, _ = synth.sample_body(synth.Circle(c, 6.0, spin=w), 2, n)
    for a in range(2):
        x = synth.face_coords(2, n, a)
        r = (x[0] - c[0], x[1] - c[1])
        expect = w * r[1] if a == 0 else -w * r[0]
        assert np.allclose(V[a], expect, rtol=0, atol=1e-12)


def test_sampled_fields_step_equals_the_analytic_step():
    # one oracle step with the sampled circle's face fields equals the step of
    # the analytic circle (the fields are bitwise equal, so is the step)
    case = synth.config1_circle((64, 32)).with_(body=synth.Body("sphere", (20.3, 15.8, 0.0), 5.0))
    g = oracle.grid_from_case(case)
    u, ue = synth.initial_velocity(case)
    P = np.zeros((32, 64))
    ua, uea, Pa = oracle.step_fn(g, oracle.make_body(case.body), 0.0, 0.2, u, ue, P)
    d, nf, V, _, _ = synth.sample_body(synth.Circle((20.3, 15.8), 5.0), 2, case.n)
    fields = oracle.measure_sampled(g, d, nf, V)
    us, ues, Ps = oracle.step_fields_fn(g, fields, 0.2, u, ue, P)
    assert np.array_equal(us, ua) and np.array_equal(Ps, Pa)


def test_viscous_force_transpose_is_its_linear_part_3d():
    # the same identity on a sampled sphere in a 3D channel with an exit plane
    case = synth.Case("v3", 3, (20, 14, 12), (False, False, True), True, (1.0, 0.0, 0.0), 0.02)
    g = oracle.grid_from_case(case)
    _, _, _, dc, nc = synth.sample_body(synth.Circle((8.3, 7.1, 5.6), 3.7), 3, case.n)
    u = synth.random_field(7, 3, case.n, amp=0.3, offset=(1.0, 0.0, 0.0))
    v = synth.random_field(8, 3, case.n, amp=1.0)
    ue = 1.0 + 0.1 * synth.random_scalar(9, 2, (case.n[1], case.n[2], 1)).ravel()
    ve = synth.random_scalar(10, 2, (case.n[1], case.n[2], 1)).ravel()
    w = (0.7, -1.3, 0.4)
    ub, ueb = oracle.forces_viscous_sampled_vjp(g, dc, nc, w)
    F1 = oracle.forces_viscous_sampled(g, dc, nc, u + v, ue + ve)
    F0 = oracle.forces_viscous_sampled(g, dc, nc, u, ue)
    lhs = float(np.sum(ub * v) + np.dot(ueb[: ve.size], ve))
    rhs = float(np.dot(w, (F1 - F0)[:3]))
    assert abs(rhs) > 1e-3
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs))


def test_viscous_force_transpose_is_its_linear_part():
    # the viscous force is affine in (u, ue) (boundary constants aside), so its
    # transpose contracted with (v, ve) is w . (F(u + v, ue + ve) - F(u, ue))
    case, shape, _ = synth.spinning_cylinders(D=16, Re=50.0, xi=2.0)
    g = oracle.grid_from_case(case)
    _, _, _, dc, nc = synth.sample_body(shape, 2, case.n)
    u = synth.random_field(7, 2, case.n, amp=0.3, offset=(1.0, 0.0))
    v = synth.random_field(8, 2, case.n, amp=1.0)
    ue = 1.0 + 0.1 * synth.random_scalar(9, 1, (case.n[1], 1, 1)).ravel()
    ve = synth.random_scalar(10, 1, (case.n[1], 1, 1)).ravel()
    w = (0.7, -1.3)
    ub, ueb = oracle.forces_viscous_sampled_vjp(g, dc, nc, w)
    F1 = oracle.forces_viscous_sampled(g, dc, nc, u + v, ue + ve)
    F0 = oracle.forces_viscous_sampled(g, dc, nc, u, ue)
    lhs = float(np.sum(ub * v) + np.dot(ueb[: ve.size], ve))
    rhs = float(np.dot(w, (F1 - F0)[:2]))
    assert abs(rhs) > 1e-3
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs))
