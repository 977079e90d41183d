"""CPU checks of the C ABI: the library builds, loads, and exports every
entry point include/wl.h declares (no compute call: there may be no GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "wl.h")).read()
    return sorted(set(re.findall(r"WL_API[^;]*?\b(wl_\w+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = _declared()
    for must in ("wl_sim_create", "wl_mom_step", "wl_project", "wl_forces", "wl_sim_destroy"):
        assert must in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2407_16032_b300 import build, wl
    build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", wl.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (wl_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    assert set(wl.EXPORTS) <= exported
    L = wl.lib()
    for n in _declared():
        assert hasattr(L, n)


def test_config_defaults_on_host():
    from paper_2407_16032_b300 import wl
    cfg = wl.Config()
    n = (C.c_int * 3)(64, 32, 16)
    wl.lib().wl_config_default(C.byref(cfg), 3, n)
    assert (cfg.ndim, list(cfg.n)) == (3, [64, 32, 16])
    assert cfg.tol == 1e-6 and cfg.itmax == 32 and cfg.smooth_iters == 4 and cfg.eps == 1.0
    assert wl.lib().wl_status_string(4).decode().startswith("Poisson")


def test_create_rejects_bad_configuration_without_touching_a_device():
    # validation happens before any CUDA call
    from paper_2407_16032_b300 import wl
    L = wl.lib()
    cfg = wl.Config()
    L.wl_config_default(C.byref(cfg), 3, (C.c_int * 3)(8, 8, 8))
    h = C.c_void_p()
    cfg.ndim = 4
    assert L.wl_sim_create(C.byref(cfg), None, C.byref(h)) == wl.WL_ERR_ARG
    cfg.ndim = 3
    cfg.eps = 0.0
    assert L.wl_sim_create(C.byref(cfg), None, C.byref(h)) == wl.WL_ERR_ARG
    cfg.eps = 1.0
    b = wl.Body()
    b.kind = 2  # ellipse in 3D
    b.semi[0], b.semi[1] = 4.0, 1.0
    assert L.wl_sim_create(C.byref(cfg), C.byref(b), C.byref(h)) == wl.WL_ERR_ARG
    assert not h.value


def test_product_package_does_not_reach_the_oracle():
    pkg = os.path.join(ROOT, "paper_2407_16032_b300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "liboracle" not in txt, f


def test_every_call_on_a_null_simulation_is_rejected_without_a_device():
    # each entry point that takes a simulation handle answers a NULL handle
    # (and NULL buffers) with WL_ERR_ARG before any CUDA call; destroy accepts
    # NULL as a no-op
    from paper_2407_16032_b300 import build, wl
    build.build()
    src = open(os.path.join(ROOT, "include", "wl.h")).read()
    L = C.CDLL(wl.LIB_PATH)
    seen = 0
    for name, params in re.findall(r"WL_API\s+int\s+(wl_\w+)\s*\(([^;]*?)\)\s*;", src, re.S):
        ps = [p.strip() for p in params.replace("\n", " ").split(",") if p.strip()]
        if not ps or not ps[0].startswith("wl_sim *"):
            continue
        types, args = [], []
        for p in ps:
            t = (C.c_void_p if "*" in p else C.c_double if p.startswith("double") else
                 C.c_size_t if p.startswith("size_t") else C.c_longlong if p.startswith("long long") else
                 C.c_uint if p.startswith("unsigned") else C.c_int)
            types.append(t)
            args.append(None if t is C.c_void_p else 0)
        f = getattr(L, name)
        f.argtypes, f.restype = types, C.c_int
        want = 0 if name == "wl_sim_destroy" else 1     # WL_OK / WL_ERR_ARG
        assert f(*args) == want, name
        seen += 1
    assert seen >= 30


def test_every_status_code_has_its_own_message():
    from paper_2407_16032_b300 import wl
    src = open(os.path.join(ROOT, "include", "wl.h")).read()
    codes = {int(v) for v in re.findall(r"\bWL_(?:OK|ERR_\w+)\s*=\s*(\d+)", src)}
    assert codes == set(range(len(codes)))
    L = wl.lib()
    msgs = [L.wl_status_string(c).decode() for c in sorted(codes)]
    assert all(msgs) and len(set(msgs)) == len(msgs)
    assert L.wl_status_string(max(codes) + 1).decode()          # unknown codes still get a message
    assert L.wl_last_error(None) is not None


def _bad_cases():
    def cfg(**kw):
        def f(c, b):
            for k, v in kw.items():
                if k in ("n0", "n1", "n2"):
                    c.n[int(k[1])] = v
                elif k == "periodic_x":
                    c.periodic[0] = v
                else:
                    setattr(c, k, v)
        return f

    def body(kind, **kw):
        def f(c, b):
            b.kind = kind
            b.radius = kw.get("radius", 3.0)
            b.semi[0], b.semi[1] = kw.get("semi", (4.0, 1.0))
            b.heave_axis = kw.get("heave_axis", 1)
            if "ndim" in kw:
                c.ndim = kw["ndim"]
                c.n[2] = 1 if kw["ndim"] == 2 else c.n[2]
        return f

    return {
        "n below 2": cfg(n0=1), "n above 2^20": cfg(n1=(1 << 20) + 1),
        "2^31 cells": cfg(n0=2048, n1=2048, n2=2048), "precision": cfg(precision=2),
        "negative nu": cfg(nu=-1.0), "NaN nu": cfg(nu=float("nan")),
        "exit on a periodic x": cfg(exit_hi_x=1, periodic_x=1), "tol 0": cfg(tol=0.0),
        "itmax < 0": cfg(itmax=-1), "no smoothing": cfg(smooth_iters=0), "65 smoothing": cfg(smooth_iters=65),
        "dt_init 0": cfg(dt_init=0.0), "cfl 0": cfg(cfl=0.0), "dt_max 0": cfg(dt_max=0.0),
        "unknown body": body(5), "cylinder in 2D": body(3, ndim=2), "cylinder radius 0": body(3, radius=0.0),
        "sphere radius 0": body(1, radius=0.0), "ellipse axis 0": body(2, ndim=2, semi=(4.0, 0.0)),
        "heave axis 3": body(1, heave_axis=3), "heave axis z in 2D": body(1, ndim=2, heave_axis=2),
    }


@pytest.mark.parametrize("case", sorted(_bad_cases()))
def test_create_rejects_each_invalid_setting_on_the_host(case):
    from paper_2407_16032_b300 import wl
    L = wl.lib()
    c = wl.Config()
    L.wl_config_default(C.byref(c), 3, (C.c_int * 3)(16, 12, 8))
    b = wl.Body()
    b.kind = 0
    _bad_cases()[case](c, b)
    h = C.c_void_p()
    assert L.wl_sim_create(C.byref(c), C.byref(b), C.byref(h)) == wl.WL_ERR_ARG
    assert not h.value


def test_the_default_configuration_passes_validation():
    # the control for the table above: without the bad setting, creation gets
    # past validation (on a machine without a GPU it then fails in CUDA)
    from paper_2407_16032_b300 import wl
    L = wl.lib()
    c = wl.Config()
    L.wl_config_default(C.byref(c), 3, (C.c_int * 3)(16, 12, 8))
    b = wl.Body()
    b.kind = 0
    h = C.c_void_p()
    rc = L.wl_sim_create(C.byref(c), C.byref(b), C.byref(h))
    if rc == wl.WL_OK:
        L.wl_sim_destroy(h)
    assert rc != wl.WL_ERR_ARG


def test_network_check_rejects_grids_beyond_32bit_voxel_channel_indexing():
    # the network kernels index voxel * 16 + channel in int: 2^31 / 16 voxels
    # and more are refused before any device work (no GPU needed)
    from paper_2407_16032_b300 import wl
    L = wl.lib()
    buf = (C.c_float * 16)()
    for n, want in [((512, 512, 512), wl.WL_ERR_ARG), ((1 << 27, 1, 1), wl.WL_ERR_ARG)]:
        nn = (C.c_int * 3)(*n)
        rc = L.wl_net_eval(3, nn, buf, buf, None, None, None, None)
        assert rc == want, (n, rc)


def test_static_solve_wrapper_rejects_mismatched_tensors_on_the_host():
    # each argument check of the binding fires before the library is called
    import torch
    from paper_2407_16032_b300 import wl
    n = (8, 6)
    ok = lambda dt=torch.float64, m=48: torch.zeros(m, dtype=dt)
    cases = [
        ("float32 or float64", lambda: wl.coarse_solve_static(2, n, (0, 0), [ok(), ok()], ok(torch.int32), ok())),
        ("coefficient arrays", lambda: wl.coarse_solve_static(2, n, (0, 0), [ok()], ok(), ok())),
        ("is torch.float32", lambda: wl.coarse_solve_static(2, n, (0, 0), [ok(), ok(torch.float32)], ok(), ok())),
        ("holds 40 values", lambda: wl.coarse_solve_static(2, n, (0, 0), [ok(), ok()], ok(), ok(m=40))),
        ("contiguous", lambda: wl.coarse_solve_static(2, n, (0, 0), [ok(), torch.zeros(96, dtype=torch.float64)[::2]],
                                                      ok(), ok())),
        ("CUDA tensor", lambda: wl.coarse_solve_static(2, n, (0, 0), [ok(), ok()], ok(), ok())),
    ]
    for msg, call in cases:
        with pytest.raises(ValueError, match=msg):
            call()
