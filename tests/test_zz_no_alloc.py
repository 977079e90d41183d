"""The Poisson solve that allocates no device memory (wl_coarse_solve_static).

Callers that cannot call cudaMalloc when they need a solve (an application
whose device memory is all held by its own pool or budget, or a time-critical
loop that must not call cudaMalloc because it can synchronise the device) use
this entry point; its working memory is a fixed device array inside the
library. This test calls it through the C ABI and checks its
output against the FP64 oracle's solve and against the library's regular
solve (wl_poisson_solve) on the same problem, twice in a row (the shared array
keeps the previous call's contents).
It lives in its own file so that it runs after every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from gpu_common import gpu_sim, p_err, well_determined

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_16032_b300 import build
    build.build()


@pytest.mark.parametrize("prec,body", [
    ("f64", synth.Body("sphere", (14.3, 9.1, 0.0), 4.2)),
    # In FP32 the output x carries the constant level of the pressure too: with
    # a body, cells coupled only through tiny coefficients shift that level far
    # above the pressure's variation (FP32 then cannot hold the variation), so
    # the FP32 comparison uses walls and a periodic direction without a body.
    ("f32", synth.Body()),
])
def test_static_solve_matches_regular_solve_on_two_calls(prec, body):
    import torch
    from paper_2407_16032_b300 import wl
    # 35 x 18 cells: odd, so the regular solver has a single level and the same operator
    case = synth.Case("na", 2, (35, 18, 1), (False, True, False), False, (0, 0, 0), 0.0, body)
    sim = gpu_sim(case, prec, tol=5e-9 if prec == "f32" else 1e-12, itmax=60)
    c, _, _ = sim.get_body_fields()
    dt = torch.float32 if prec == "f32" else torch.float64
    cs = [c[a].contiguous() for a in range(2)]
    cnp = c.double().cpu().numpy()
    g = oracle.grid_from_case(case)
    c_or = oracle.coeffs(g, oracle.measure(g, oracle.make_body(body), 0.0)[0] if body.kind != "none" else None)
    for seed in (3, 4):  # two calls in a row on the shared array
        # divergence only where the cell is mostly fluid, as in a projection
        b = synth.random_scalar(seed, 2, case.n) * well_determined(c_or, 2)
        p_ref = np.zeros(b.shape)
        sim.poisson_solve(torch.tensor(b, dtype=dt).cuda(), p_ref)
        x = torch.full(b.shape, float("nan"), dtype=dt, device="cuda")
        rc, rel = wl.coarse_solve_static(2, case.n, case.periodic, cs, torch.tensor(b, dtype=dt).cuda(), x)
        assert rc == wl.WL_OK and rel <= 1e-12, (rc, rel)
        xs = x.double().cpu().numpy()
        tol = 2e-6 if prec == "f32" else 1e-10
        assert p_err(xs, p_ref, cnp, 2) < tol
        p_or, rc_or, _ = oracle.poisson_solve(g, c_or, b, tol=1e-12, itmax=100)
        assert rc_or == 0 and p_err(xs, p_or, c_or, 2) < tol


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_static_solve_on_the_1024_thread_path_matches_regular_solve(prec):
    # 100 x 60 = 6000 cells: at or above 4096 cells the entry point launches
    # its block with 1024 threads; walls on x, periodic y, no body, so both
    # precisions compare the full pressure
    import torch
    from paper_2407_16032_b300 import wl
    case = synth.Case("na", 2, (100, 60, 1), (False, True, False), False, (0, 0, 0), 0.0, synth.Body())
    sim = gpu_sim(case, prec, tol=5e-9 if prec == "f32" else 1e-12, itmax=60)
    c, _, _ = sim.get_body_fields()
    dt = torch.float32 if prec == "f32" else torch.float64
    cs = [c[a].contiguous() for a in range(2)]
    cnp = c.double().cpu().numpy()
    g = oracle.grid_from_case(case)
    c_or = oracle.coeffs(g, None)
    for seed in (5, 6):
        b = synth.random_scalar(seed, 2, case.n)
        p_ref = np.zeros(b.shape)
        sim.poisson_solve(torch.tensor(b, dtype=dt).cuda(), p_ref)
        x = torch.full(b.shape, float("nan"), dtype=dt, device="cuda")
        rc, rel = wl.coarse_solve_static(2, case.n, case.periodic, cs, torch.tensor(b, dtype=dt).cuda(), x,
                                         maxit=20000)
        assert rc == wl.WL_OK and rel <= 1e-12, (rc, rel)
        tol = 2e-6 if prec == "f32" else 1e-10
        xs = x.double().cpu().numpy()
        assert p_err(xs, p_ref, cnp, 2) < tol
        p_or, rc_or, _ = oracle.poisson_solve(g, c_or, b, tol=1e-12, itmax=100)
        assert rc_or == 0 and p_err(xs, p_or, c_or, 2) < tol


def test_static_solve_rejects_oversized_grids():
    import torch
    from paper_2407_16032_b300 import wl
    n = (256, 128)  # 32768 cells > WL_STATIC_MAX_CELLS
    c = [torch.ones(n[::-1], device="cuda") for _ in range(2)]
    r = torch.zeros(n[::-1], device="cuda")
    x = torch.zeros(n[::-1], device="cuda")
    rc, _ = wl.coarse_solve_static(2, n, (True, True), c, r, x)
    assert rc == wl.WL_ERR_ARG
