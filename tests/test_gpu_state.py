"""Checkpoint and resume (wl_state_size / wl_get_state / wl_set_state): a sim
loaded with another sim's state repeats its following steps bit for bit."""
import numpy as np
import pytest

import synth
from gpu_common import gpu_fields, gpu_sim

pytestmark = pytest.mark.gpu


def _start(sim, case):
    import torch
    u, ue = synth.initial_velocity(case)
    sim.set_velocity(torch.tensor(u, dtype=torch.float32, device="cuda"),
                     torch.tensor(ue, dtype=torch.float32, device="cuda"))


@pytest.mark.parametrize("which", ["moving_sphere", "tgv", "foil"])
def test_resume_repeats_the_steps_bit_for_bit(which):
    # a moving body (re-measured in a box every step), a body-free periodic
    # flow and a 2D moving foil: the state after 4 steps, 3 more steps on the
    # original and on two fresh sims loaded from a host and a device copy
    import torch
    case = {"moving_sphere": synth.config5_moving_sphere((96, 48, 48), D=9.0, centre=(24.0, 24.0, 24.0)),
            "tgv": synth.config2_tgv(32),
            "foil": synth.config4_ellipse((128, 64), chord=24.0, A=6.0, centre=(40.0, 32.0))}[which]
    a = gpu_sim(case, "f32")
    _start(a, case)
    for _ in range(4):
        a.mom_step()
    buf = a.get_state()
    for _ in range(3):
        a.mom_step()
    ua, uea, pa = gpu_fields(a)
    ta = a.get_time()
    for src in (buf, torch.tensor(buf, device="cuda")):
        b = gpu_sim(case, "f32")
        b.set_state(src)
        for _ in range(3):
            b.mom_step()
        ub, ueb, pb = gpu_fields(b)
        assert np.array_equal(ua, ub) and np.array_equal(pa, pb)
        if uea is not None:
            assert np.array_equal(uea, ueb)
        assert b.get_time() == ta
        b.close()


def test_a_state_of_another_grid_or_precision_is_rejected():
    from paper_2407_16032_b300.wl import WLError, WL_ERR_ARG
    case = synth.config2_tgv(32)
    a = gpu_sim(case, "f32")
    buf = a.get_state()
    for other, prec in ((synth.config2_tgv(64), "f32"), (case, "f64")):
        b = gpu_sim(other, prec)
        with pytest.raises(WLError) as e:
            b.set_state(np.resize(buf, max(buf.size, 1 << 26)) if other is not case else buf)
        assert e.value.code == WL_ERR_ARG
    with pytest.raises(WLError) as e:
        gpu_sim(case, "f32").set_state(buf[:100])
    assert e.value.code == WL_ERR_ARG
