"""GPU parity of the adjoint of one time step (wl_step_vjp) against the FP64
oracle's discrete adjoint (itself pinned by central differences of the
oracle's forward step).

Bars. FP64 on the GPU: the limiter branches are decided in the same precision
on both sides, so the pull-backs agree to the solver tolerances (1e-8 relative
max-norm). FP32 on the GPU: the branch decisions are taken on FP32 values of
u*, which differ from the oracle's by ~1e-7, so a face whose limiter sits
within that distance of a kink may take the other (equally valid) one-sided
derivative; each such flux moves up to six entries of the pull-back by a small
amount (measured: 9 of 69,120 entries, 1.6e-4 of the max-norm, on the 3D
sphere case, unchanged when the solves are tightened from 1e-7 to 1e-8). The
bar is 1e-4 relative in the L2 norm, 1e-5 relative max-norm on all entries but
at most max(12, 2e-4 of the entries), and 1e-3 on those.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_16032_b300 import build
    build.build()


def _case(kind):
    B = synth.Body()
    if kind == "periodic2d":
        case = synth.Case("p2", 2, (40, 36, 1), (True, True, False), False, (0.0, 0.0, 0.0), 0.01)
        u0 = synth.random_field(11, 2, (40, 36, 1), amp=0.5)
    elif kind == "channel_exit":
        case = synth.Case("ch", 2, (70, 34, 1), (False, True, False), True, (1.0, 0.0, 0.0), 0.005)
        u0 = synth.random_field(12, 2, (70, 34, 1), amp=0.2, offset=(1.0, 0.0))
    elif kind == "circle":
        B = synth.Body("sphere", (30.0, 20.3, 0.0), 6.2)
        case = synth.Case("ci", 2, (72, 40, 1), (False, False, False), True, (1.0, 0.0, 0.0), 0.01, B)
        u0 = synth.random_field(13, 2, (72, 40, 1), amp=0.2, offset=(1.0, 0.0))
    elif kind == "ellipse_moving":
        B = synth.Body("ellipse", (40.2, 32.7, 0.0), 0.0, (16.0, 3.84), heave_amp=4.0, pitch_amp=0.26, omega=0.05)
        case = synth.Case("el", 2, (96, 64, 1), (False, False, False), True, (1.0, 0.0, 0.0), 0.02, B)
        u0 = synth.random_field(15, 2, (96, 64, 1), amp=0.1, offset=(1.0, 0.0))
    elif kind == "walled3d":
        case = synth.Case("w3", 3, (36, 20, 18), (True, True, False), False, (0.0, 0.0, 0.0), 0.02)
        u0 = synth.random_field(14, 3, (36, 20, 18), amp=0.4)
    elif kind == "sphere3d":
        B = synth.Body("sphere", (14.2, 12.1, 11.7), 4.6)
        case = synth.Case("s3", 3, (40, 24, 24), (False, False, False), True, (1.0, 0.0, 0.0), 0.02, B)
        u0 = synth.random_field(16, 3, (40, 24, 24), amp=0.1, offset=(1.0, 0.0, 0.0))
    else:
        raise KeyError(kind)
    g = oracle.grid_from_case(case)
    ue0 = np.zeros(max(oracle.plane_size(g), 1))
    if case.exit_hi_x:
        ue0 = 1.0 + 0.1 * (2 * synth.uniform01(21, 0, ue0.size) - 1)
    # lower boundary faces carry U (the state the step starts from)
    for a in range(case.ndim):
        if not case.periodic[a]:
            idx = [slice(None)] * case.ndim
            idx[case.ndim - 1 - a] = 0
            u0[(a,) + tuple(idx)] = case.U[a]
    return case, g, oracle.make_body(B), u0, ue0


def _round32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def _gpu_vjp(case, prec, t, dt, u0, ue0, lu, le, lP, tol):
    import torch
    from paper_2407_16032_b300 import sim_from_case
    tdt = torch.float32 if prec == "f32" else torch.float64
    sim = sim_from_case(case, prec, tol=1e-6, itmax=80)
    T = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=tdt, device="cuda")
    P0 = torch.zeros(u0.shape[1:], dtype=torch.float64, device="cuda")
    lPd = None if lP is None else torch.tensor(lP, dtype=torch.float64, device="cuda")
    ub, ueb, st = sim.step_vjp(t, dt, T(u0), T(ue0) if case.exit_hi_x else None, P0, T(lu),
                               T(le) if case.exit_hi_x else None, lPd, tol=tol)
    out = ub.double().cpu().numpy(), (ueb.double().cpu().numpy() if ueb is not None else None)
    sim.close()
    return out, st


KINDS = ["periodic2d", "channel_exit", "circle", "ellipse_moving", "walled3d", "sphere3d"]


@pytest.mark.parametrize("kind", KINDS)
def test_step_vjp_fp64_matches_oracle(kind):
    case, g, B, u0, ue0 = _case(kind)
    rng = np.random.default_rng(5)
    t, dt = 1.5, 0.3
    lu = rng.normal(size=u0.shape)
    le = rng.normal(size=ue0.shape) if case.exit_hi_x else np.zeros_like(ue0)
    lP = rng.normal(size=u0.shape[1:]) if case.body.kind != "none" else None
    P0 = np.zeros(u0.shape[1:])
    ub_o, ueb_o = oracle.step_vjp(g, B, t, dt, u0, ue0, P0, lu, le, lP)
    (ub, ueb), st = _gpu_vjp(case, "f64", t, dt, u0, ue0, lu, le, lP, tol=1e-12)
    assert all(s.rel_resid <= 1e-12 for s in st)
    scale = np.abs(ub_o).max()
    assert np.abs(ub - ub_o).max() <= 1e-8 * scale
    if case.exit_hi_x:
        assert np.abs(ueb - ueb_o).max() <= 1e-8 * scale


@pytest.mark.parametrize("kind", KINDS)
def test_step_vjp_fp32_matches_oracle(kind):
    case, g, B, u0, ue0 = _case(kind)
    u0, ue0 = _round32(u0), _round32(ue0)
    rng = np.random.default_rng(6)
    t, dt = 1.5, 0.3
    lu = _round32(rng.normal(size=u0.shape))
    le = _round32(rng.normal(size=ue0.shape)) if case.exit_hi_x else np.zeros_like(ue0)
    lP = rng.normal(size=u0.shape[1:]) if case.body.kind != "none" else None
    P0 = np.zeros(u0.shape[1:])
    ub_o, ueb_o = oracle.step_vjp(g, B, t, dt, u0, ue0, P0, lu, le, lP)
    (ub, ueb), st = _gpu_vjp(case, "f32", t, dt, u0, ue0, lu, le, lP, tol=1e-7)
    assert all(s.rel_resid <= 1e-7 for s in st)
    e = np.abs(ub - ub_o)
    scale = np.abs(ub_o).max()
    assert np.linalg.norm(ub - ub_o) <= 1e-4 * np.linalg.norm(ub_o)
    bad = e > 1e-5 * scale
    assert bad.sum() <= max(12, int(2e-4 * e.size)), (bad.sum(), e.max() / scale)
    assert e.max() <= 1e-3 * scale
    if case.exit_hi_x:
        assert np.linalg.norm(ueb - ueb_o) <= 1e-4 * np.linalg.norm(ueb_o)


def test_step_vjp_leaves_the_state_unchanged():
    import torch
    from paper_2407_16032_b300 import sim_from_case
    case, g, B, u0, ue0 = _case("circle")
    sim = sim_from_case(case, "f32", tol=1e-6, itmax=60)
    for _ in range(3):
        sim.mom_step()
    u1, ue1 = sim.get_velocity()
    p1 = sim.get_pressure()
    t1 = sim.get_time()
    T = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float32, device="cuda")
    sim.step_vjp(0.2, 0.25, T(u0), T(ue0), None, T(np.ones_like(u0)), T(np.ones_like(ue0)), None, tol=1e-6)
    u2, ue2 = sim.get_velocity()
    assert torch.equal(u1, u2) and torch.equal(ue1, ue2)
    assert torch.equal(p1, sim.get_pressure())
    assert sim.get_time() == t1
    st, rc = sim.mom_step()
    assert rc == 0
    sim.close()
