"""GPU checks of the learned Poisson guess: the BF16 tensor-core network kernels
against the FP64 network oracle (forward, loss, weight gradients), and what a
network trained on the solver's own projections gains over the warm start."""
import numpy as np
import pytest

import synth
from oracle import net as onet
from gpu_common import gpu_sim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_16032_b300 import build
    build.build()


def _bf16(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _weights(seed, C=16):
    r = np.random.default_rng(seed)
    W = np.zeros((3, 27, 16, 16), np.float32)
    W[0, :, 0, :C] = r.normal(size=(27, C)) * np.sqrt(2 / 27)
    W[1, :, :C, :C] = r.normal(size=(27, C, C)) * np.sqrt(2 / (27 * C))
    W[2, :, :C, 0] = r.normal(size=(27, C)) * np.sqrt(2 / (27 * C))
    return W


# (96, 64, 32): 1536 tiles of 128 voxels, more than the tensor-core
# convolution's 1184 blocks, so some blocks run two tiles in a row
@pytest.mark.parametrize("shape,nd", [((7, 5, 6), 3), ((12, 9, 1), 2), ((16, 16, 16), 3), ((96, 64, 32), 3)])
def test_network_kernels_match_fp64_oracle(shape, nd):
    from paper_2407_16032_b300 import wl
    W = _weights(1)
    r = np.random.default_rng(2)
    grid = shape[::-1]  # [z, y, x]
    x = r.normal(size=grid).astype(np.float32)
    t = r.normal(size=grid).astype(np.float32)
    y, dw, loss = wl.net_eval(nd, shape, W, x, t)
    Wb = _bf16(W)
    Ws = (Wb[0][:, :1, :], Wb[1], Wb[2][:, :, :1])
    L, dWs, y_or = onet.backward(_bf16(x), Ws, t.astype(np.float64))
    # BF16 activations between layers (8-bit mantissa): a few parts in 1e3
    assert np.abs(y - y_or).max() <= 2e-2 * np.abs(y_or).max()
    assert loss == pytest.approx(L, rel=2e-2)
    got = (dw[0][:, :1, :], dw[1], dw[2][:, :, :1])
    for g_, o_ in zip(got, dWs):
        assert np.abs(g_ - o_).max() <= 4e-2 * np.abs(o_).max()
    # padded weights receive gradients but training keeps them at zero
    assert np.isfinite(dw).all()


def test_trained_guess_reduces_the_initial_residual():
    # Train on the solver's own projections of the Taylor-Green flow, then
    # compare projections of the continued run with and without the network.
    case = synth.config2_tgv(64)
    sim = gpu_sim(case, "f32", tol=1e-6)
    import torch
    u, ue = synth.initial_velocity(case)
    sim.set_velocity(torch.tensor(u, dtype=torch.float32).cuda())
    sim.guess_setup(level=2, capacity=64)
    sim.guess_mode(collect=True)
    for _ in range(16):
        sim.mom_step()
    lv, ns, _ = sim.guess_info()
    assert lv == 2 and ns == 32
    l0, l1 = sim.guess_train(iters=300, lr=2e-3, batch=4, seed=0)
    assert l1 < 0.5 * l0, (l0, l1)
    sim.guess_mode(collect=False, use=False)
    state_u, _ = sim.get_velocity()
    state_p = sim.get_pressure()
    t, dt = sim.get_time()
    base, learned = [], []
    for use, out in ((False, base), (True, learned)):
        sim.set_velocity(state_u)
        sim.set_pressure(state_p)
        sim.set_time(t, dt)
        sim.guess_mode(use=use)
        for _ in range(4):
            st, rc = sim.mom_step()
            out.append([(st.proj[k].rel_initial, st.proj[k].vcycles) for k in range(2)])
    r_base = np.mean([p[0] for s in base for p in s])
    r_learn = np.mean([p[0] for s in learned for p in s])
    v_base = np.mean([p[1] for s in base for p in s])
    v_learn = np.mean([p[1] for s in learned for p in s])
    print(f"initial residual {r_base:.3e} -> {r_learn:.3e}; V-cycles {v_base:.2f} -> {v_learn:.2f}")
    assert r_learn < r_base
