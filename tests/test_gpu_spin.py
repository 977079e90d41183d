"""GPU check of the spin-rate study (Sec. 6.1, the optimised control
cylinders): dC_P/dxi from the window adjoint along the control circle's
velocity tangent against central differences of C_P itself, both at the same
(fixed) time steps, on a coarse version of the flow."""
import pytest

from paper_2407_16032_b300.spin_control import SpinControl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("viscous", [True, False])
@pytest.mark.parametrize("prec,hs,bar", [("f64", (1e-3, 1e-4), 1e-4), ("f32", (2e-2,), 2e-2)])
def test_cp_gradient_matches_central_differences(prec, hs, bar, viscous):
    # FP64: the solves converged to 1e-11, steps h = 1e-3 and 1e-4 (a limiter
    # branch switch within h spoils at most one of them); FP32: solves to 1e-6
    # and h = 2e-2, where C_P's rounding noise over 2h stays ~1e-4 of the slope
    tol = 1e-11 if prec == "f64" else 1e-6
    sc = SpinControl(D=16, Re=100.0, t_star=0.75, precision=prec, tol=tol, adj_tol=tol, ckpt_every=8,
                     viscous=viscous)
    xi = 4.0
    Cp, dCp, info = sc.cp(xi)
    assert info["steps"] > 20 and dCp is not None
    errs = []
    for h in hs:
        cp_p = sc.cp(xi + h, grad=False, dts=info["dts"])[0]
        cp_m = sc.cp(xi - h, grad=False, dts=info["dts"])[0]
        fd = (cp_p - cp_m) / (2 * h)
        errs.append(abs(dCp - fd) / abs(fd))
    assert min(errs) <= bar, (dCp, errs)
