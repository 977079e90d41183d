"""ctypes binding of libwl.so (include/wl.h): argument marshalling only.

Every step of the solver runs in the CUDA kernels of libwl.so. PyTorch provides
device memory (through the wl_allocator callback into its caching allocator)
and the CUDA stream. There is no CPU fallback: if the library or a CUDA device
is missing, construction raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwl.so")

WL_OK, WL_ERR_ARG, WL_ERR_CUDA, WL_ERR_ALLOC, WL_ERR_NOT_CONVERGED, WL_ERR_NONFINITE, WL_ERR_UNSTABLE, WL_ERR_STATE = range(8)
WL_F32, WL_F64 = 0, 1
BODY_KIND = {"none": 0, "sphere": 1, "ellipse": 2, "cylinder": 3, "user": 4}

EXPORTS = (
    "wl_config_default", "wl_sim_create", "wl_sim_destroy", "wl_set_velocity", "wl_get_velocity",
    "wl_get_pressure", "wl_set_pressure", "wl_set_time", "wl_get_time", "wl_mom_step", "wl_project",
    "wl_poisson_solve", "wl_conv_diff", "wl_forces", "wl_forces_viscous", "wl_body_update", "wl_get_body_fields",
    "wl_diagnostics", "wl_info", "wl_profile", "wl_profile_report", "wl_coarse_solve_static", "wl_guess_setup",
    "wl_guess_mode", "wl_guess_train", "wl_guess_weights", "wl_guess_info", "wl_net_eval", "wl_step_vjp",
    "wl_force_dp", "wl_window_forward", "wl_window_backward", "wl_set_body", "wl_tguess_mode", "wl_tguess_fit",
    "wl_tguess_weights", "wl_last_error", "wl_status_string", "wl_set_body_fields", "wl_set_body_velocity_tangent",
    "wl_window_forward_weighted", "wl_window_stats", "wl_state_size", "wl_get_state", "wl_set_state",
    "wl_set_coarse_dense_max",
)

_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("alloc", _ALLOC_FN), ("free", _FREE_FN)]


class Config(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("periodic", C.c_int * 3), ("exit_hi_x", C.c_int),
                ("U", C.c_double * 3), ("nu", C.c_double), ("eps", C.c_double), ("precision", C.c_int),
                ("cfl", C.c_double), ("dt_max", C.c_double), ("dt_init", C.c_double), ("dt_min", C.c_double),
                ("tol", C.c_double), ("itmax", C.c_int), ("smooth_iters", C.c_int), ("stream", C.c_void_p),
                ("allocator", Allocator)]


class Body(C.Structure):
    _fields_ = [("kind", C.c_int), ("centre", C.c_double * 3), ("radius", C.c_double), ("semi", C.c_double * 2),
                ("heave_amp", C.c_double), ("pitch_amp", C.c_double), ("omega", C.c_double),
                ("phase", C.c_double), ("heave_axis", C.c_int)]


class SolveStats(C.Structure):
    _fields_ = [("vcycles", C.c_int), ("rel_resid", C.c_double), ("bnorm", C.c_double), ("rel_initial", C.c_double)]


class StepStats(C.Structure):
    _fields_ = [("proj", SolveStats * 2), ("dt", C.c_double), ("t", C.c_double), ("dt_next", C.c_double)]


_lib = None


def lib() -> C.CDLL:
    """Load libwl.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libwl.so not built ({LIB_PATH}); run python -m paper_2407_16032_b300.build")
        L = C.CDLL(LIB_PATH)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
        sig = {
            "wl_config_default": ([C.POINTER(Config), ip, C.POINTER(C.c_int)], None),
            "wl_sim_create": ([C.POINTER(Config), C.POINTER(Body), C.POINTER(vp)], ip),
            "wl_sim_destroy": ([vp], ip),
            "wl_set_velocity": ([vp, vp, vp], ip),
            "wl_get_velocity": ([vp, vp, vp], ip),
            "wl_get_pressure": ([vp, vp], ip),
            "wl_set_pressure": ([vp, vp], ip),
            "wl_set_time": ([vp, C.c_double, C.c_double], ip),
            "wl_get_time": ([vp, dp, dp], ip),
            "wl_mom_step": ([vp, C.c_double, C.POINTER(StepStats)], ip),
            "wl_project": ([vp, C.c_double, C.c_double, C.POINTER(SolveStats)], ip),
            "wl_poisson_solve": ([vp, vp, vp, C.POINTER(SolveStats)], ip),
            "wl_conv_diff": ([vp, vp, vp, vp], ip),
            "wl_forces": ([vp, dp], ip),
            "wl_forces_viscous": ([vp, dp], ip),
            "wl_body_update": ([vp, C.c_double], ip),
            "wl_get_body_fields": ([vp, vp, vp, vp], ip),
            "wl_diagnostics": ([vp, dp, dp, dp], ip),
            "wl_info": ([vp, C.POINTER(C.c_int), C.POINTER(C.c_longlong)], ip),
            "wl_profile": ([vp, ip], ip),
            "wl_profile_report": ([vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)], ip),
            "wl_coarse_solve_static": ([ip, C.POINTER(C.c_int), C.POINTER(C.c_int), ip, C.POINTER(vp), vp, vp, ip,
                                        C.c_double, vp, dp], ip),
            "wl_guess_setup": ([vp, ip, ip], ip),
            "wl_guess_mode": ([vp, ip, ip], ip),
            "wl_guess_train": ([vp, ip, C.c_double, ip, C.c_uint, dp, dp], ip),
            "wl_guess_weights": ([vp, vp, vp], ip),
            "wl_guess_info": ([vp, C.POINTER(C.c_int), C.POINTER(C.c_int), dp], ip),
            "wl_net_eval": ([ip, C.POINTER(C.c_int), vp, vp, vp, vp, vp, dp], ip),
            "wl_step_vjp": ([vp, C.c_double, C.c_double, vp, vp, vp, vp, vp, vp, C.c_double, vp, vp,
                             C.POINTER(SolveStats)], ip),
            "wl_force_dp": ([vp, ip, C.c_double, vp], ip),
            "wl_window_forward": ([vp, ip, ip, vp, vp, dp, vp], ip),
            "wl_window_backward": ([vp, C.c_double, vp, vp, C.c_double, vp, vp, vp], ip),
            "wl_set_body": ([vp, C.POINTER(Body)], ip),
            "wl_set_coarse_dense_max": ([vp, ip], ip),
            "wl_set_body_fields": ([vp, vp, vp, vp, vp, vp], ip),
            "wl_set_body_velocity_tangent": ([vp, vp], ip),
            "wl_window_forward_weighted": ([vp, ip, ip, vp, vp, vp, ip, dp, vp], ip),
            "wl_window_stats": ([vp, vp, dp], ip),
            "wl_state_size": ([vp, C.POINTER(C.c_size_t)], ip),
            "wl_get_state": ([vp, vp, C.c_size_t], ip),
            "wl_set_state": ([vp, vp, C.c_size_t], ip),
            "wl_tguess_mode": ([vp, ip, ip], ip),
            "wl_tguess_fit": ([vp, vp, vp], ip),
            "wl_tguess_weights": ([vp, vp, vp], ip),
            "wl_last_error": ([vp], C.c_char_p),
            "wl_status_string": ([ip], C.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


class WLError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def _ptr(x) -> Optional[int]:
    """Address of a torch tensor (host or device) or a numpy array (host)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


def _body_struct(body) -> Body:
    """wl_body from a body description (kind, centre, radius, semi, heave_amp,
    pitch_amp, omega, phase, heave_axis)."""
    bd = Body()
    bd.kind = BODY_KIND[body.kind]
    for a in range(3):
        bd.centre[a] = float(body.centre[a])
    bd.radius = float(body.radius)
    bd.semi[0], bd.semi[1] = float(body.semi[0]), float(body.semi[1])
    bd.heave_amp, bd.pitch_amp = float(body.heave_amp), float(body.pitch_amp)
    bd.omega, bd.phase, bd.heave_axis = float(body.omega), float(body.phase), int(body.heave_axis)
    return bd


@dataclass
class SolveResult:
    vcycles: int
    rel_resid: float
    bnorm: float
    rel_initial: float = 0.0


class Sim:
    """A simulation object of libwl (wl_sim_create ... wl_sim_destroy)."""

    def __init__(self, ndim, n, periodic=(False, False, False), exit_hi_x=False, U=(0.0, 0.0, 0.0), nu=0.0,
                 eps=1.0, precision="f32", body=None, tol=1e-6, itmax=32, smooth_iters=4, cfl=1.0, dt_max=1.0,
                 dt_init=0.25, dt_min=1e-6, device=None, use_torch_allocator=True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libwl needs a CUDA device")
        self.torch = torch
        L = lib()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.ndim = ndim
        self.n = tuple(int(v) for v in (list(n) + [1, 1])[:3])
        if ndim == 2:
            self.n = (self.n[0], self.n[1], 1)
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        self.dtype = torch.float32 if precision in ("f32", WL_F32) else torch.float64
        self.exit = bool(exit_hi_x)
        cfg = Config()
        nn = (C.c_int * 3)(*self.n)
        L.wl_config_default(C.byref(cfg), ndim, nn)
        for a in range(3):
            cfg.periodic[a] = int(bool(periodic[a])) if a < len(periodic) else 0
            cfg.U[a] = float(U[a]) if a < len(U) else 0.0
        cfg.exit_hi_x = int(self.exit)
        cfg.nu, cfg.eps = float(nu), float(eps)
        cfg.precision = WL_F32 if self.dtype == torch.float32 else WL_F64
        cfg.tol, cfg.itmax, cfg.smooth_iters = float(tol), int(itmax), int(smooth_iters)
        cfg.cfl, cfg.dt_max, cfg.dt_init, cfg.dt_min = float(cfl), float(dt_max), float(dt_init), float(dt_min)
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream()
        cfg.stream = self.stream.cuda_stream
        self._blocks = {}
        if use_torch_allocator:
            def _alloc(ctx, nbytes):
                try:
                    t = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
                except RuntimeError:
                    return None
                self._blocks[t.data_ptr()] = t
                return t.data_ptr()

            def _free(ctx, p):
                self._blocks.pop(p, None)

            self._alloc_cb, self._free_cb = _ALLOC_FN(_alloc), _FREE_FN(_free)
            cfg.allocator.alloc, cfg.allocator.free = self._alloc_cb, self._free_cb
        bd = None
        if body is not None and getattr(body, "kind", "none") != "none":
            bd = _body_struct(body)
        self._h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = L.wl_sim_create(C.byref(cfg), C.byref(bd) if bd is not None else None, C.byref(self._h))
        if rc != WL_OK:
            raise WLError(rc, "wl_sim_create failed: " + L.wl_status_string(rc).decode())
        self.cfg = cfg
        self.body = body

    # -------------------------------------------------------------- plumbing
    def _check(self, rc, what, ok=(WL_OK,)):
        if rc not in ok:
            msg = lib().wl_last_error(self._h).decode()
            raise WLError(rc, f"{what}: {msg or lib().wl_status_string(rc).decode()}")
        return rc

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().wl_sim_destroy(self._h)
            self._h = C.c_void_p()
            self._blocks.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _shape(self):
        return (self.n[2], self.n[1], self.n[0]) if self.ndim == 3 else (self.n[1], self.n[0])

    def new_velocity(self, device=True):
        return self.torch.zeros((self.ndim,) + self._shape(), dtype=self.dtype,
                                device=self.device if device else "cpu")

    def new_plane(self, device=True):
        return self.torch.zeros(max(self.n[1] * self.n[2], 1), dtype=self.dtype,
                                device=self.device if device else "cpu")

    # ------------------------------------------------------------ C-ABI calls
    def set_velocity(self, u, ue=None):
        self._check(lib().wl_set_velocity(self._h, _ptr(u), _ptr(ue)), "wl_set_velocity")

    def get_velocity(self, u=None, ue=None):
        u = self.new_velocity() if u is None else u
        if ue is None and self.exit:
            ue = self.new_plane(device=u.is_cuda if hasattr(u, "is_cuda") else False)
        self._check(lib().wl_get_velocity(self._h, _ptr(u), _ptr(ue)), "wl_get_velocity")
        return u, ue

    def get_pressure(self, p=None):
        p = self.torch.zeros(self._shape(), dtype=self.torch.float64, device=self.device) if p is None else p
        self._check(lib().wl_get_pressure(self._h, _ptr(p)), "wl_get_pressure")
        return p

    def set_pressure(self, p):
        self._check(lib().wl_set_pressure(self._h, _ptr(p)), "wl_set_pressure")

    def set_time(self, t, dt_next):
        self._check(lib().wl_set_time(self._h, float(t), float(dt_next)), "wl_set_time")

    def get_time(self):
        t, dt = C.c_double(), C.c_double()
        self._check(lib().wl_get_time(self._h, C.byref(t), C.byref(dt)), "wl_get_time")
        return t.value, dt.value

    def mom_step(self, dt_fixed=0.0, allow_unconverged=False):
        st = StepStats()
        ok = (WL_OK, WL_ERR_NOT_CONVERGED) if allow_unconverged else (WL_OK,)
        rc = self._check(lib().wl_mom_step(self._h, float(dt_fixed), C.byref(st)), "wl_mom_step", ok)
        return st, rc

    def project(self, w, dt):
        st = SolveStats()
        self._check(lib().wl_project(self._h, float(w), float(dt), C.byref(st)), "wl_project")
        return SolveResult(st.vcycles, st.rel_resid, st.bnorm, st.rel_initial)

    def poisson_solve(self, b, p):
        st = SolveStats()
        rc = lib().wl_poisson_solve(self._h, _ptr(b), _ptr(p), C.byref(st))
        self._check(rc, "wl_poisson_solve", (WL_OK, WL_ERR_NOT_CONVERGED))
        return SolveResult(st.vcycles, st.rel_resid, st.bnorm, st.rel_initial), rc

    def conv_diff(self, u, ue=None, r=None):
        r = self.torch.empty_like(u) if r is None else r
        self._check(lib().wl_conv_diff(self._h, _ptr(u), _ptr(ue), _ptr(r)), "wl_conv_diff")
        return r

    def forces(self):
        F = (C.c_double * 3)()
        self._check(lib().wl_forces(self._h, F), "wl_forces")
        return np.array(F[:])

    def forces_viscous(self):
        """Viscous force nu sum_I K (grad u + grad u^T) . n on the body."""
        F = (C.c_double * 3)()
        self._check(lib().wl_forces_viscous(self._h, F), "wl_forces_viscous")
        return np.array(F[:])

    def body_update(self, t):
        self._check(lib().wl_body_update(self._h, float(t)), "wl_body_update")

    def get_body_fields(self):
        T = self.torch
        c = T.zeros((self.ndim,) + self._shape(), dtype=self.dtype, device=self.device)
        m = T.zeros((9,) + self._shape(), dtype=self.dtype, device=self.device)
        V = T.zeros((self.ndim,) + self._shape(), dtype=self.dtype, device=self.device)
        self._check(lib().wl_get_body_fields(self._h, _ptr(c), _ptr(m), _ptr(V)), "wl_get_body_fields")
        return c, m.reshape((3, 3) + self._shape())[: self.ndim], V

    def diagnostics(self):
        ke, en, md = C.c_double(), C.c_double(), C.c_double()
        self._check(lib().wl_diagnostics(self._h, C.byref(ke), C.byref(en), C.byref(md)), "wl_diagnostics")
        return ke.value, en.value, md.value

    def profile(self, on=True):
        self._check(lib().wl_profile(self._h, int(bool(on))), "wl_profile")

    def profile_report(self):
        """[(kernel, level, launches, total_ms, cells_per_launch)] from wl_profile_report."""
        need = C.c_size_t()
        self._check(lib().wl_profile_report(self._h, None, 0, C.byref(need)), "wl_profile_report")
        buf = C.create_string_buffer(need.value + 16)
        self._check(lib().wl_profile_report(self._h, buf, len(buf), None), "wl_profile_report")
        rows = []
        for line in buf.value.decode().splitlines():
            nm, lv, n, ms, cells = line.split()
            rows.append((nm, int(lv), int(n), float(ms), int(cells)))
        return rows

    # ------------------------------------------------------ learned guess
    def guess_setup(self, level=2, capacity=64):
        self._check(lib().wl_guess_setup(self._h, int(level), int(capacity)), "wl_guess_setup")

    def guess_mode(self, collect=False, use=False):
        self._check(lib().wl_guess_mode(self._h, int(bool(collect)), int(bool(use))), "wl_guess_mode")

    def guess_train(self, iters=200, lr=1e-3, batch=4, seed=0):
        l0, l1 = C.c_double(), C.c_double()
        self._check(lib().wl_guess_train(self._h, int(iters), float(lr), int(batch), int(seed), C.byref(l0),
                                         C.byref(l1)), "wl_guess_train")
        return l0.value, l1.value

    def guess_weights(self, set_to=None):
        out = np.zeros(3 * 27 * 16 * 16, dtype=np.float32)
        src = None if set_to is None else np.ascontiguousarray(set_to, dtype=np.float32)
        self._check(lib().wl_guess_weights(self._h, _ptr(src), _ptr(out)), "wl_guess_weights")
        return out.reshape(3, 27, 16, 16)

    def guess_info(self):
        lv, ns, gn = C.c_int(), C.c_int(), C.c_double()
        self._check(lib().wl_guess_info(self._h, C.byref(lv), C.byref(ns), C.byref(gn)), "wl_guess_info")
        return lv.value, ns.value, gn.value

    # ------------------------------------------------------------ adjoint
    def step_vjp(self, t, dt, u0, ue0, P0, lu, le=None, lP=None, tol=1e-8, ub=None, ueb=None):
        """wl_step_vjp: (ub, ueb) = J^T (lu, le, lP) of one step from (u0, ue0)
        at time t with step dt. Returns (ub, ueb, [predictor, corrector] solve
        results of the adjoint solves)."""
        ub = self.torch.empty_like(lu) if ub is None else ub
        if ueb is None and self.exit:
            ueb = self.new_plane(device=lu.is_cuda)
        st = (SolveStats * 2)()
        self._check(lib().wl_step_vjp(self._h, float(t), float(dt), _ptr(u0), _ptr(ue0), _ptr(P0), _ptr(lu),
                                      _ptr(le), _ptr(lP), float(tol), _ptr(ub), _ptr(ueb), st), "wl_step_vjp")
        return ub, ueb, [SolveResult(x.vcycles, x.rel_resid, x.bnorm, x.rel_initial) for x in st]

    def force_dp(self, axis, scale=1.0, out=None):
        """wl_force_dp: scale * dF_axis/dp per cell (float64)."""
        out = self.torch.zeros(self._shape(), dtype=self.torch.float64, device=self.device) if out is None else out
        self._check(lib().wl_force_dp(self._h, int(axis), float(scale), _ptr(out)), "wl_force_dp")
        return out

    def window_forward(self, nsteps, ckpt_every=20, dts=None, w=(0.0, 0.0, 0.0), step_w=None, viscous=False):
        """wl_window_forward (wl_window_forward_weighted with per-step weights
        step_w or the viscous force in the objective): returns (J, dts taken)."""
        J = C.c_double()
        out = np.zeros(int(nsteps))
        d = None if dts is None else np.ascontiguousarray(dts, dtype=np.float64)
        ww = np.ascontiguousarray((list(w) + [0.0, 0.0, 0.0])[:3], dtype=np.float64)
        if step_w is None and not viscous:
            self._check(lib().wl_window_forward(self._h, int(nsteps), int(ckpt_every), _ptr(d), _ptr(ww),
                                                C.byref(J), _ptr(out)), "wl_window_forward")
        else:
            sw = None if step_w is None else np.ascontiguousarray(step_w, dtype=np.float64)
            if sw is not None and sw.shape != (int(nsteps),):
                raise ValueError("step_w needs one weight per step")
            self._check(lib().wl_window_forward_weighted(self._h, int(nsteps), int(ckpt_every), _ptr(d), _ptr(ww),
                                                         _ptr(sw), int(bool(viscous)), C.byref(J), _ptr(out)),
                        "wl_window_forward_weighted")
        return J.value, out

    def window_backward(self, gJ=1.0, lu=None, le=None, tol=1e-7, params=True):
        """wl_window_backward: returns (du0, due0, dparams or None)."""
        du0 = self.new_velocity()
        due0 = self.new_plane() if self.exit else None
        dp = np.zeros(2) if params else None
        self._check(lib().wl_window_backward(self._h, float(gJ), _ptr(lu), _ptr(le), float(tol), _ptr(du0),
                                             _ptr(due0), _ptr(dp)), "wl_window_backward")
        return du0, due0, dp

    def _field(self, x, comps, what):
        """A (comps, *grid) array of the sim's dtype, contiguous, as given or
        converted (host arrays stay on the host: the library copies them)."""
        T = self.torch
        if isinstance(x, np.ndarray):
            x = T.from_numpy(np.ascontiguousarray(x))
        x = x.to(self.dtype).contiguous()
        if x.numel() != comps * self.ncell:
            raise ValueError(f"{what}: expected {comps} x {self.ncell} values, got {x.numel()}")
        return x

    def set_body_fields(self, d_face, n_face, V_face, d_cell, n_cell):
        """wl_set_body_fields: a "user" body from its samples (layouts of
        include/wl.h: d_face (ndim, *grid), n_face (ndim, ndim, *grid),
        V_face (ndim, *grid), d_cell (*grid), n_cell (ndim, *grid))."""
        nd = self.ndim
        f = [self._field(d_face, nd, "d_face"), self._field(n_face, nd * nd, "n_face"),
             self._field(V_face, nd, "V_face"), self._field(d_cell, 1, "d_cell"), self._field(n_cell, nd, "n_cell")]
        self._check(lib().wl_set_body_fields(self._h, *[_ptr(x) for x in f]), "wl_set_body_fields")

    def set_body_velocity_tangent(self, dV_face=None):
        """wl_set_body_velocity_tangent (None clears it)."""
        x = None if dV_face is None else self._field(dV_face, self.ndim, "dV_face")
        self._check(lib().wl_set_body_velocity_tangent(self._h, _ptr(x)), "wl_set_body_velocity_tangent")

    def get_state(self):
        """wl_get_state into a host byte array (numpy uint8)."""
        n = C.c_size_t()
        self._check(lib().wl_state_size(self._h, C.byref(n)), "wl_state_size")
        buf = np.zeros(n.value, dtype=np.uint8)
        self._check(lib().wl_get_state(self._h, _ptr(buf), n.value), "wl_get_state")
        return buf

    def set_state(self, buf):
        """wl_set_state from a byte array (numpy uint8 or a torch uint8 tensor)."""
        if isinstance(buf, np.ndarray):
            buf = np.ascontiguousarray(buf, dtype=np.uint8)
            size = buf.nbytes
        else:
            size = buf.numel() * buf.element_size()
        self._check(lib().wl_set_state(self._h, _ptr(buf), size), "wl_set_state")

    def window_stats(self):
        """wl_window_stats: adjoint solves of the last backward sweep as a dict."""
        c = np.zeros(4, dtype=np.int32)
        r = C.c_double()
        self._check(lib().wl_window_stats(self._h, _ptr(c), C.byref(r)), "wl_window_stats")
        return {"solves": int(c[0]), "unconverged": int(c[1]), "max_vcycles": int(c[2]), "worst_step": int(c[3]),
                "max_rel_resid": r.value}

    def set_body(self, body):
        """wl_set_body with a body description (kind unchanged)."""
        self._check(lib().wl_set_body(self._h, C.byref(_body_struct(body))), "wl_set_body")
        self.body = body

    def set_coarse_dense_max(self, max_cells):
        """wl_set_coarse_dense_max: coarsest levels of at most max_cells cells
        (0..1024; 256 at creation) are solved by the dense FP64 operator."""
        self._check(lib().wl_set_coarse_dense_max(self._h, int(max_cells)), "wl_set_coarse_dense_max")

    # ------------------------------------------------ learned temporal guess
    def tguess_mode(self, collect=False, use=False):
        self._check(lib().wl_tguess_mode(self._h, int(bool(collect)), int(bool(use))), "wl_tguess_mode")

    def tguess_fit(self):
        """Returns (weights (2, 2): [stage][w1, w2], residual ratio per stage)."""
        w, r = np.zeros(4), np.zeros(2)
        self._check(lib().wl_tguess_fit(self._h, _ptr(w), _ptr(r)), "wl_tguess_fit")
        return w.reshape(2, 2), r

    def tguess_weights(self, set_to=None):
        out = np.zeros(4)
        src = None if set_to is None else np.ascontiguousarray(set_to, dtype=np.float64).ravel()
        self._check(lib().wl_tguess_weights(self._h, _ptr(src), _ptr(out)), "wl_tguess_weights")
        return out.reshape(2, 2)

    def info(self):
        lv, nl = C.c_int(), C.c_longlong()
        self._check(lib().wl_info(self._h, C.byref(lv), C.byref(nl)), "wl_info")
        return lv.value, nl.value


def sim_from_case(case, precision="f32", **kw) -> Sim:
    """Build a Sim from a workload description with the attributes of a case
    (ndim, n, periodic, exit_hi_x, U, nu, eps, body, cfl, dt_max, dt0)."""
    return Sim(case.ndim, case.n, case.periodic, case.exit_hi_x, case.U, case.nu, case.eps, precision,
               case.body, cfl=case.cfl, dt_max=case.dt_max, dt_init=case.dt0, **kw)


def coarse_solve_static(ndim, n, periodic, c, r, x, maxit=2000, rtol=1e-12, stream=None, want_resid=True):
    """wl_coarse_solve_static: the small Poisson solve that allocates no device
    memory, for callers that must not allocate when they solve (an application
    whose device memory is all held by its own pool, or a loop that must not
    stall on an allocation). c: sequence of ndim CUDA tensors, r, x: CUDA
    tensors; all contiguous, of one dtype (float32 or float64) and at least
    prod(n) elements each. want_resid=False passes no residual pointer: the
    call then only enqueues work (no copy to the host, no synchronisation) and
    returns None for the residual. Returns (status, final relative residual)."""
    import torch
    if r.dtype not in (torch.float32, torch.float64):
        raise ValueError("coarse_solve_static: r must be float32 or float64")
    if len(c) != ndim:
        raise ValueError(f"coarse_solve_static: need {ndim} coefficient arrays, got {len(c)}")
    cells = int(np.prod([int(v) for v in list(n)[:ndim]]))
    named = [("r", r), ("x", x)] + [(f"c[{a}]", t) for a, t in enumerate(c)]
    for name, t in named:
        if t.dtype != r.dtype:
            raise ValueError(f"coarse_solve_static: {name} is {t.dtype}, r is {r.dtype}")
        if t.numel() < cells:
            raise ValueError(f"coarse_solve_static: {name} holds {t.numel()} values, the grid has {cells} cells")
        if not t.is_contiguous():
            raise ValueError(f"coarse_solve_static: {name} must be contiguous")
    for name, t in named:
        if not t.is_cuda:
            raise ValueError(f"coarse_solve_static: {name} must be a CUDA tensor")
    prec = WL_F32 if r.dtype == torch.float32 else WL_F64
    nn = (C.c_int * 3)(*(list(n) + [1, 1, 1])[:3])
    pp = (C.c_int * 3)(*[int(bool(v)) for v in (list(periodic) + [0, 0, 0])[:3]])
    cp = (C.c_void_p * 3)(*([t.data_ptr() for t in c] + [None] * (3 - len(c))))
    rel = C.c_double()
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    rc = lib().wl_coarse_solve_static(ndim, nn, pp, prec, cp, r.data_ptr(), x.data_ptr(), int(maxit),
                                      float(rtol), st, C.byref(rel) if want_resid else None)
    return rc, (rel.value if want_resid else None)


def net_eval(ndim, n, w, x, t=None):
    """wl_net_eval: one forward/backward pass of the guess network (host arrays).
    w: (3, 27, 16, 16) float32; x, t: grid-shaped float32. Returns (y, dw, loss)."""
    nn = (C.c_int * 3)(*(list(n) + [1, 1, 1])[:3])
    w = np.ascontiguousarray(w, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    tt = None if t is None else np.ascontiguousarray(t, dtype=np.float32)
    y = np.zeros(x.shape, dtype=np.float32)
    dw = np.zeros(w.shape, dtype=np.float32)
    loss = C.c_double()
    rc = lib().wl_net_eval(ndim, nn, _ptr(w), _ptr(x), _ptr(tt), _ptr(y), _ptr(dw), C.byref(loss))
    if rc != WL_OK:
        raise WLError(rc, "wl_net_eval failed")
    return y, dw, loss.value
