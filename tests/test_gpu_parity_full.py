"""GPU parity at the workloads' full sizes: the CUDA path (through the C ABI,
in the launch configuration the bench times) against the FP64 oracle, run on
all host cores, after 10 steps with the oracle's time steps.

Bars: 1e-5 relative max-norm on u and on the mean-free pressure of
well-determined cells (all faces with c >= 1/2) where the input does not
amplify rounding (the body-free Taylor-Green vortex, the flapping foil). The
impulsively started spheres amplify a 1e-7 perturbation of their start to
~1e-5 within 10 steps in the FP64 oracle itself; for them the bar after 10
steps is five times that measured response (and at least 1e-5), and after one
step 1e-6. The near-body pressure and the pressure force are reported
(WL_PARITY_REPORT) as well as asserted where stated.

Sizes: Taylor-Green vortex 256^3 and the fixed sphere 256x128x128 (full
size), the flapping foil 1024x512 with chord 64 (full size), the oscillating
sphere at its oracle size 128x64x64 (D = 12; the full 512x256x256 runs in the
bench, where the solver's residual is checked every projection)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import (calibrated_bars, gpu_fields, near_body_p_err, p_err, rel_max, report, run_pair)

pytestmark = [pytest.mark.gpu, pytest.mark.full_size]

ORACLE_TOL = 1e-9   # the oracle's Poisson tolerance: four orders below the bars


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_16032_b300 import build
    build.build()
    oracle.set_threads(oracle.host_cores())


def _errors(orc, sim):
    u, ue, p = gpu_fields(sim)
    g = orc.g
    body = orc.case.body.kind != "none"
    c = oracle.coeffs(g, oracle.measure(g, orc.b, orc.t)[0] if body else None)
    e = {"u": rel_max(u, orc.u), "p": p_err(p, orc.P, c, orc.case.ndim)}
    if orc.case.exit_hi_x:
        e["ue"] = rel_max(ue, orc.ue)
    if body:
        F_or = oracle.forces(g, orc.b, orc.t, orc.P)
        e["p_near_body"] = near_body_p_err(p, orc.P, c, orc.case.ndim)
        e["force_rel"] = float(np.abs(sim.forces() - F_or).max() / np.abs(F_or).max())
    return e


def _check(name, e, bar_u, bar_p, bar_force=None):
    report(name, **e, bar_u=bar_u, bar_p=bar_p)
    assert e["u"] < bar_u and e.get("ue", 0.0) < bar_u, (name, e, bar_u)
    assert e["p"] < bar_p, (name, e, bar_p)
    if bar_force is not None:
        assert e["force_rel"] < bar_force, (name, e, bar_force)


def test_config2_tgv256_full_size_fp32_10_steps():
    case = synth.config2_tgv(256)
    orc, sim, st = run_pair(case, 10, "f32", oracle_tol=ORACLE_TOL)
    _check("tgv256 full", _errors(orc, sim), 1e-5, 1e-5)
    ke_or, en_or = oracle.diagnostics(orc.g, orc.u, orc.ue)
    ke, en, md = sim.diagnostics()
    assert abs(ke / ke_or - 1) < 1e-5 and abs(en / en_or - 1) < 1e-4
    assert md < 1e-4


def _sphere_case(case, name):
    first = {}
    orc, sim, st = run_pair(case, 10, "f32", oracle_tol=ORACLE_TOL,
                            on_step=lambda k, o, s: first.update(_errors(o, s)) if k == 1 else None)
    _check(name + " step 1", first, 1e-6, 1e-6)
    bu, bp = calibrated_bars(case, orc)
    _check(name, _errors(orc, sim), bu, bp, bar_force=bp)


def test_config3_sphere_full_size_fp32_1_and_10_steps():
    _sphere_case(synth.config3_sphere(), "sphere3d 256x128x128 full")


def test_config5_moving_sphere_oracle_size_fp32_1_and_10_steps():
    _sphere_case(synth.scaled(synth.config5_moving_sphere(), 0.25), "msphere3d 128x64x64 oracle size")


def test_config4_flapping_foil_full_size_fp32_10_steps():
    case = synth.config4_ellipse()
    orc, sim, st = run_pair(case, 10, "f32", oracle_tol=ORACLE_TOL)
    _check("ellipse2d 1024x512 chord 64 full", _errors(orc, sim), 1e-5, 1e-5, bar_force=1e-5)
