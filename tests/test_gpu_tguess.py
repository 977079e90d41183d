"""The learned temporal guess (wl_tguess_*): a 1x1x1 convolution over each
projection stage's pressure history, fitted by least squares in the residual
norm to the solver's own projections. It may only change the iteration path:
the converged fields agree with plain multigrid's to the solve tolerance, and
on the data it was fitted to it lowers the initial residual."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_16032_b300 import build
    build.build()


def _sim(case, tol):
    import torch
    from paper_2407_16032_b300 import sim_from_case
    sim = sim_from_case(case, "f32", tol=tol, itmax=60)
    u, ue = synth.initial_velocity(case)
    sim.set_velocity(torch.tensor(u, dtype=torch.float32, device="cuda"),
                     torch.tensor(ue, dtype=torch.float32, device="cuda"))
    return sim


@pytest.mark.parametrize("case", [synth.config2_tgv(64),
                                  synth.Case("circle", 2, (192, 96, 1), (False, False, False), True, (1.0, 0, 0),
                                             0.05, synth.Body("sphere", (48.3, 47.6, 0.0), 12.0), init="noise",
                                             seed=2)],
                         ids=["tgv64", "circle2d"])
def test_temporal_guess_keeps_the_answer_and_lowers_the_initial_residual(case):
    sim = _sim(case, 1e-8)
    for _ in range(4):
        sim.mom_step(allow_unconverged=True)
    sim.tguess_mode(collect=True, use=False)
    r_plain_fit = []
    for _ in range(8):
        st, _ = sim.mom_step(allow_unconverged=True)
        r_plain_fit.append((st.proj[0].rel_initial, st.proj[1].rel_initial))
    w, ratio = sim.tguess_fit()
    assert np.all(np.isfinite(w)) and np.all(ratio <= 1.0 + 1e-9), (w, ratio)
    su, sue = sim.get_velocity()
    sp = sim.get_pressure()
    t, dt = sim.get_time()
    out = {}
    for use in (False, True):
        sim.set_velocity(su, sue)
        sim.set_pressure(sp)
        sim.set_time(t, dt)
        sim.tguess_mode(collect=False, use=use)
        r0 = []
        for n in range(6):
            st, rc = sim.mom_step(allow_unconverged=False)
            assert st.proj[0].rel_resid <= 1e-8 and st.proj[1].rel_resid <= 1e-8
            if n >= 2:   # the guess starts once two steps of history exist
                r0.append(st.proj[0].rel_initial + st.proj[1].rel_initial)
        u, _ = sim.get_velocity()
        out[use] = (u.double().cpu().numpy(), float(np.mean(r0)))
    # the same converged fields (only the solver's path differs)
    ref = np.abs(out[False][0]).max()
    assert np.abs(out[True][0] - out[False][0]).max() <= 1e-5 * ref
    # a lower initial residual than the plain warm start on this flow
    assert out[True][1] < out[False][1], (out[True][1], out[False][1])
    sim.close()


def test_plain_weights_reproduce_the_warm_start():
    # w = (0, 1) for both stages is the previous projection's pressure
    case = synth.config2_tgv(32)
    sim = _sim(case, 1e-7)
    for _ in range(3):
        sim.mom_step()
    su, sue = sim.get_velocity()
    sp = sim.get_pressure()
    t, dt = sim.get_time()
    res = {}
    for use in (False, True):
        sim.set_velocity(su, sue)
        sim.set_pressure(sp)
        sim.set_time(t, dt)
        sim.tguess_mode(collect=False, use=use)
        sim.tguess_weights([[0.0, 1.0], [0.0, 1.0]])
        r = []
        for _ in range(5):
            st, _ = sim.mom_step()
            r.append((st.proj[0].rel_initial, st.proj[1].rel_initial, st.proj[0].vcycles, st.proj[1].vcycles))
        res[use] = np.array(r)
    assert np.allclose(res[True][:, :2], res[False][:, :2], rtol=1e-3)
    # (a solve that ends right at the tolerance may take one cycle more or less)
    assert abs(res[True][:, 2:].sum() - res[False][:, 2:].sum()) <= 1
    sim.close()
