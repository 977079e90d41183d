"""FP64 CPU oracle of the BDIM time step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg
may import this package. The product path (``paper_2407_16032_b300``) never
imports, loads or calls it; the two share no code except the seeded input
generators in ``synth``.

The arithmetic lives in ``wl_oracle.c`` (plain C loops, FP64); this module
compiles it with gcc and marshals numpy arrays through ctypes. Every routine
cites the part of the paper it follows in the C source.

Parity status: every function here is pinned by ``tests/test_oracle.py``
(closed forms, invariants, brute force); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wl_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain gcc, no fast-math, no FMA contraction; OpenMP
    over cells with results independent of the thread count)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fopenmp",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("periodic", C.c_int * 3),
                ("exit_hi_x", C.c_int), ("U", C.c_double * 3), ("nu", C.c_double),
                ("eps", C.c_double)]


class BodyS(C.Structure):
    _fields_ = [("kind", C.c_int), ("centre", C.c_double * 3), ("radius", C.c_double),
                ("semi", C.c_double * 2), ("heave_amp", C.c_double), ("pitch_amp", C.c_double),
                ("omega", C.c_double), ("phase", C.c_double), ("heave_axis", C.c_int)]


class Solver(C.Structure):
    _fields_ = [("tol", C.c_double), ("itmax", C.c_int), ("smooth_iters", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("vcycles", C.c_int), ("rel_resid", C.c_double), ("bnorm", C.c_double)]


_lib = None
_P = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        for name, args, res in [
            ("orc_set_threads", [C.c_int], None),
            ("orc_get_threads", [], C.c_int),
            ("orc_quick", [C.c_double] * 3, C.c_double),
            ("orc_mu0", [C.c_double, C.c_double], C.c_double),
            ("orc_mu1", [C.c_double, C.c_double], C.c_double),
            ("orc_kernel", [C.c_double, C.c_double], C.c_double),
            ("orc_conv_diff", [C.POINTER(Grid), _P, _P, _P], None),
            ("orc_body_eval", [C.POINTER(BodyS), C.c_int, _P, C.c_double, _P, _P, _P], None),
            ("orc_measure", [C.POINTER(Grid), C.POINTER(BodyS), C.c_double, _P, _P, _P], None),
            ("orc_coeffs", [C.POINTER(Grid), _P, _P], None),
            ("orc_measure_sampled", [C.POINTER(Grid), _P, _P, _P, _P, _P, _P], None),
            ("orc_forces_sampled", [C.POINTER(Grid), _P, _P, _P, _P], None),
            ("orc_forces_viscous_sampled", [C.POINTER(Grid), _P, _P, _P, _P, _P], None),
            ("orc_force_dp_sampled", [C.POINTER(Grid), _P, _P, C.c_int, _P], None),
            ("orc_forces_viscous_sampled_vjp", [C.POINTER(Grid), _P, _P, _P, _P, _P], None),
            ("orc_bdim", [C.POINTER(Grid), _P, _P, C.c_double, _P, _P, _P, _P, _P], None),
            ("orc_exit_bc", [C.POINTER(Grid), _P, _P, _P, C.c_double, C.c_int, _P, _P, _P], None),
            ("orc_divergence", [C.POINTER(Grid), _P, _P, _P], None),
            ("orc_poisson_apply", [C.POINTER(Grid), _P, _P, _P], None),
            ("orc_poisson_diag", [C.POINTER(Grid), _P, _P], None),
            ("orc_mg_levels", [C.POINTER(Grid)], C.c_int),
            ("orc_poisson_solve", [C.POINTER(Grid), _P, _P, _P, C.POINTER(Solver), C.POINTER(Stats)], C.c_int),
            ("orc_grad_update", [C.POINTER(Grid), _P, _P, C.c_double, _P], None),
            ("orc_project", [C.POINTER(Grid), _P, _P, _P, _P, C.c_double, C.c_double, C.POINTER(Solver), C.POINTER(Stats)], C.c_int),
            ("orc_cfl", [C.POINTER(Grid), _P, _P, C.c_double, C.c_double], C.c_double),
            ("orc_forces", [C.POINTER(Grid), C.POINTER(BodyS), C.c_double, _P, _P], None),
            ("orc_forces_viscous", [C.POINTER(Grid), C.POINTER(BodyS), C.c_double, _P, _P, _P], None),
            ("orc_step", [C.POINTER(Grid), C.POINTER(BodyS), C.c_double, C.c_double, _P, _P, _P, C.POINTER(Solver), C.POINTER(Stats)], C.c_int),
            ("orc_diagnostics", [C.POINTER(Grid), _P, _P, _P, _P], None),
            ("orc_conv_diff_vjp", [C.POINTER(Grid), _P, _P, _P, _P, _P], None),
            ("orc_force_dp", [C.POINTER(Grid), C.POINTER(BodyS), C.c_double, C.c_int, _P], None),
            ("orc_step_fields", [C.POINTER(Grid), _P, _P, _P, C.c_double, _P, _P, _P, C.POINTER(Solver),
                                 C.POINTER(Stats)], C.c_int),
            ("orc_step_vjp_fields", [C.POINTER(Grid), _P, _P, _P, C.c_double, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                     _P, _P], None),
            ("orc_step_vjp", [C.POINTER(Grid), C.POINTER(BodyS), C.c_double, C.c_double, _P, _P, _P, _P, _P, _P, _P, _P],
             None),
        ]:
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
    return _lib


def set_threads(n: int) -> None:
    """Threads of the oracle's per-cell loops (results do not depend on it)."""
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], (a.dtype, a.flags)
    return a.ctypes.data_as(_P)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_grid(ndim, n, periodic=(False, False, False), exit_hi_x=False, U=(0.0, 0.0, 0.0), nu=0.0, eps=1.0):
    g = Grid()
    g.ndim = ndim
    nn = list(n) + [1] * (3 - len(n))
    if ndim == 2:
        nn[2] = 1
    for a in range(3):
        g.n[a] = int(nn[a])
        g.periodic[a] = int(bool(periodic[a])) if a < len(periodic) else 0
        g.U[a] = float(U[a]) if a < len(U) else 0.0
    g.exit_hi_x = int(bool(exit_hi_x))
    g.nu = float(nu)
    g.eps = float(eps)
    return g


def grid_from_case(case):
    return make_grid(case.ndim, case.n, case.periodic, case.exit_hi_x, case.U, case.nu, case.eps)


def make_body(body):
    b = BodyS()
    b.kind = body.kind_id
    for a in range(3):
        b.centre[a] = float(body.centre[a])
    b.radius = float(body.radius)
    b.semi[0], b.semi[1] = float(body.semi[0]), float(body.semi[1])
    b.heave_amp, b.pitch_amp = float(body.heave_amp), float(body.pitch_amp)
    b.omega, b.phase = float(body.omega), float(body.phase)
    b.heave_axis = int(body.heave_axis)
    return b


def make_solver(tol=1e-10, itmax=64, smooth_iters=4):
    s = Solver()
    s.tol, s.itmax, s.smooth_iters = float(tol), int(itmax), int(smooth_iters)
    return s


def _shape(g):
    return (g.n[2], g.n[1], g.n[0]) if g.ndim == 3 else (g.n[1], g.n[0])


def plane_size(g):
    return g.n[1] * g.n[2]


# ---------------------------------------------------------------- wrappers
def quick(u, c, d):
    return lib().orc_quick(float(u), float(c), float(d))


def mu0(d, eps=1.0):
    return lib().orc_mu0(float(d), float(eps))


def mu1(d, eps=1.0):
    return lib().orc_mu1(float(d), float(eps))


def kernel(d, eps=1.0):
    return lib().orc_kernel(float(d), float(eps))


def conv_diff(g, u, ue):
    u, ue = _d(u), _d(ue)
    r = np.zeros_like(u)
    lib().orc_conv_diff(C.byref(g), _p(u), _p(ue), _p(r))
    return r


def body_eval(body_s, ndim, x, t):
    xx = _d(np.array(list(x) + [0.0] * (3 - len(x))))
    d = np.zeros(1)
    n = np.zeros(3)
    V = np.zeros(3)
    lib().orc_body_eval(C.byref(body_s), ndim, _p(xx), float(t), _p(d), _p(n), _p(V))
    return d[0], n, V


def measure(g, body_s, t):
    sh = _shape(g)
    mu0a = np.zeros((g.ndim,) + sh)
    mu1n = np.zeros((g.ndim, 3) + sh)
    V = np.zeros((g.ndim,) + sh)
    lib().orc_measure(C.byref(g), C.byref(body_s), float(t), _p(mu0a), _p(mu1n), _p(V))
    return mu0a, mu1n, V


def measure_sampled(g, d, n, V):
    """Face moments of a body given by samples: d (ndim, *grid) signed distance
    at the faces, n (ndim, ndim, *grid) unit normal (n[a, b]: component b at
    face a), V (ndim, *grid) body velocity. Returns (mu0, mu1n, V) in the
    layout of measure()."""
    sh = _shape(g)
    mu0a = np.zeros((g.ndim,) + sh)
    mu1n = np.zeros((g.ndim, 3) + sh)
    Vo = np.zeros((g.ndim,) + sh)
    lib().orc_measure_sampled(C.byref(g), _p(_d(d)), _p(_d(n)), _p(_d(V)), _p(mu0a), _p(mu1n), _p(Vo))
    return mu0a, mu1n, Vo


def forces_sampled(g, dc, ncen, p):
    """Pressure force of a sampled body from the distance dc (grid) and normal
    ncen (ndim, *grid) at the cell centres."""
    F = np.zeros(3)
    lib().orc_forces_sampled(C.byref(g), _p(_d(dc)), _p(_d(ncen)), _p(_d(p)), _p(F))
    return F


def forces_viscous_sampled(g, dc, ncen, u, ue):
    """Viscous force of a sampled body from centre samples dc, ncen."""
    F = np.zeros(3)
    ue = _d(ue) if ue is not None else np.zeros(max(plane_size(g), 1))
    lib().orc_forces_viscous_sampled(C.byref(g), _p(_d(dc)), _p(_d(ncen)), _p(_d(u)), _p(ue), _p(F))
    return F


def forces_viscous_sampled_vjp(g, dc, ncen, w):
    """d(w . F_v)/d(u, ue) of the sampled body's viscous force: (ub, ueb)."""
    ub = np.zeros((g.ndim,) + _shape(g))
    ueb = np.zeros(max(plane_size(g), 1))
    ww = np.zeros(3)
    ww[: len(w)] = w
    lib().orc_forces_viscous_sampled_vjp(C.byref(g), _p(_d(dc)), _p(_d(ncen)), _p(ww), _p(ub), _p(ueb))
    return ub, ueb


def force_dp_sampled(g, dc, ncen, axis):
    """dF_axis/dp per cell of a sampled body."""
    out = np.zeros(_shape(g))
    lib().orc_force_dp_sampled(C.byref(g), _p(_d(dc)), _p(_d(ncen)), int(axis), _p(out))
    return out


def coeffs(g, mu0a=None):
    c = np.zeros((g.ndim,) + _shape(g))
    lib().orc_coeffs(C.byref(g), _p(_d(mu0a)) if mu0a is not None else None, _p(c))
    return c


def bdim(g, u0, r, dt, mu0a=None, mu1n=None, V=None, ustar=None):
    out = np.zeros_like(_d(u0))
    keep = [_d(u0), _d(r)] + [(_d(x) if x is not None else None) for x in (mu0a, mu1n, V, ustar)]
    lib().orc_bdim(C.byref(g), _p(keep[0]), _p(keep[1]), float(dt), _p(keep[2]), _p(keep[3]),
                   _p(keep[4]), _p(keep[5]), _p(out))
    return out


def exit_bc(g, ue0, uG, ueG, dt, corrector, ustar_e, u_new, ue):
    ue = _d(ue).copy()
    args = [_d(ue0), _d(uG), _d(ueG), _d(ustar_e) if ustar_e is not None else None, _d(u_new)]
    lib().orc_exit_bc(C.byref(g), _p(args[0]), _p(args[1]), _p(args[2]), float(dt), int(corrector),
                      _p(args[3]), _p(args[4]), _p(ue))
    return ue


def divergence(g, u, ue):
    b = np.zeros(_shape(g))
    lib().orc_divergence(C.byref(g), _p(_d(u)), _p(_d(ue)), _p(b))
    return b


def poisson_apply(g, c, p):
    out = np.zeros(_shape(g))
    lib().orc_poisson_apply(C.byref(g), _p(_d(c)), _p(_d(p)), _p(out))
    return out


def poisson_diag(g, c):
    out = np.zeros(_shape(g))
    lib().orc_poisson_diag(C.byref(g), _p(_d(c)), _p(out))
    return out


def mg_levels(g):
    return lib().orc_mg_levels(C.byref(g))


def poisson_solve(g, c, b, p0=None, tol=1e-10, itmax=64, smooth_iters=4):
    p = np.zeros(_shape(g)) if p0 is None else _d(p0).copy()
    S = make_solver(tol, itmax, smooth_iters)
    st = Stats()
    rc = lib().orc_poisson_solve(C.byref(g), _p(_d(c)), _p(_d(b)), _p(p), C.byref(S), C.byref(st))
    return p, rc, st


def grad_update(g, c, p, wdt, u):
    u = _d(u).copy()
    lib().orc_grad_update(C.byref(g), _p(_d(c)), _p(_d(p)), float(wdt), _p(u))
    return u


def project(g, c, u, ue, P, w, dt, tol=1e-10, itmax=64, smooth_iters=4):
    u = _d(u).copy()
    P = _d(P).copy()
    S = make_solver(tol, itmax, smooth_iters)
    st = Stats()
    rc = lib().orc_project(C.byref(g), _p(_d(c)), _p(u), _p(_d(ue)), _p(P), float(w), float(dt), C.byref(S), C.byref(st))
    return u, P, rc, st


def cfl(g, u, ue, cfl=1.0, dt_max=1.0):
    return lib().orc_cfl(C.byref(g), _p(_d(u)), _p(_d(ue)), float(cfl), float(dt_max))


def forces(g, body_s, t, p):
    F = np.zeros(3)
    lib().orc_forces(C.byref(g), C.byref(body_s), float(t), _p(_d(p)), _p(F))
    return F


def forces_viscous(g, body_s, t, u, ue):
    """Viscous force nu sum_I K (grad u + grad u^T) . n at the cell centres."""
    F = np.zeros(3)
    lib().orc_forces_viscous(C.byref(g), C.byref(body_s), float(t), _p(_d(u)), _p(_d(ue)), _p(F))
    return F


def diagnostics(g, u, ue):
    ke = np.zeros(1)
    en = np.zeros(1)
    lib().orc_diagnostics(C.byref(g), _p(_d(u)), _p(_d(ue)), _p(ke), _p(en))
    return ke[0], en[0]


def force_dp(g, body_s, t, axis):
    """dF_axis/dp per cell (the force is linear in the pressure)."""
    out = np.zeros(_shape(g))
    lib().orc_force_dp(C.byref(g), C.byref(body_s), float(t), int(axis), _p(out))
    return out


def conv_diff_vjp(g, u, ue, lam):
    """(J_R(u, ue))^T lam -> (ubar, uebar)."""
    ub = np.zeros_like(_d(u))
    ueb = np.zeros(max(plane_size(g), 1))
    lib().orc_conv_diff_vjp(C.byref(g), _p(_d(u)), _p(_d(ue)), _p(_d(lam)), _p(ub), _p(ueb))
    return ub, ueb


def step_vjp(g, body_s, t, dt, u0, ue0, P0, lu, le, lP=None):
    """Vector-Jacobian product of one step (orc_step) w.r.t. (u0, ue0), given
    the cotangents (lu, le, lP) of its outputs (u, ue, P); lP may be None."""
    ub = np.zeros_like(_d(u0))
    ueb = np.zeros(max(plane_size(g), 1))
    le = _d(le) if le is not None else np.zeros(max(plane_size(g), 1))
    lPd = _d(lP) if lP is not None else None
    lib().orc_step_vjp(C.byref(g), C.byref(body_s), float(t), float(dt), _p(_d(u0)), _p(_d(ue0)), _p(_d(P0)),
                       _p(_d(lu)), _p(le), _p(lPd) if lPd is not None else None, _p(ub), _p(ueb))
    return ub, ueb


def step_fields_fn(g, fields, dt, u0, ue0, P0, tol=1e-13):
    """One orc_step_fields on copies with explicit face fields (mu0, mu1n, V)
    (None: no body): returns (u, ue, P)."""
    u, ue, P = _d(u0).copy(), _d(ue0).copy(), _d(P0).copy()
    S = make_solver(tol, 200, 4)
    st = (Stats * 2)()
    fk = [None, None, None] if fields is None else [_d(x) for x in fields]
    lib().orc_step_fields(C.byref(g), *[(_p(x) if x is not None else None) for x in fk], float(dt), _p(u), _p(ue),
                          _p(P), C.byref(S), st)
    return u, ue, P


def step_vjp_fields(g, fields, dt, u0, ue0, P0, lu, le, lP=None):
    """Vector-Jacobian product of orc_step_fields: returns (ub, ueb, mu0b,
    mu1nb, Vb), the last three the cotangents of the face fields."""
    mu0, mu1n, V = (_d(x) for x in fields)
    ub = np.zeros_like(_d(u0))
    ueb = np.zeros(max(plane_size(g), 1))
    le = _d(le) if le is not None else np.zeros(max(plane_size(g), 1))
    lPd = _d(lP) if lP is not None else None
    mu0b, mu1nb, Vb = np.zeros_like(mu0), np.zeros_like(mu1n), np.zeros_like(V)
    lib().orc_step_vjp_fields(C.byref(g), _p(mu0), _p(mu1n), _p(V), float(dt), _p(_d(u0)), _p(_d(ue0)),
                              _p(_d(P0)), _p(_d(lu)), _p(le), _p(lPd) if lPd is not None else None, _p(ub), _p(ueb),
                              _p(mu0b), _p(mu1nb), _p(Vb))
    return ub, ueb, mu0b, mu1nb, Vb


def step_fn(g, body_s, t, dt, u0, ue0, P0, tol=1e-13):
    """One orc_step on copies: returns (u, ue, P)."""
    u, ue, P = _d(u0).copy(), _d(ue0).copy(), _d(P0).copy()
    S = make_solver(tol, 200, 4)
    st = (Stats * 2)()
    lib().orc_step(C.byref(g), C.byref(body_s), float(t), float(dt), _p(u), _p(ue), _p(P), C.byref(S), st)
    return u, ue, P


@dataclass
class State:
    u: np.ndarray
    ue: np.ndarray
    P: np.ndarray
    t: float
    dt: float


class Sim:
    """Host-side stepping loop around ``orc_step`` (the same Heun step as C6)."""

    def __init__(self, case, tol=1e-10, itmax=64, smooth_iters=4, u=None, ue=None):
        from synth import initial_velocity
        self.case = case
        self.g = grid_from_case(case)
        self.b = make_body(case.body)
        self.S = make_solver(tol, itmax, smooth_iters)
        if u is None:
            u, ue = initial_velocity(case)
        self.u = _d(u).copy()
        self.ue = _d(ue).copy() if case.exit_hi_x else np.zeros(max(plane_size(self.g), 1))
        self.P = np.zeros(_shape(self.g))
        self.t = 0.0
        self.dt = case.dt0
        # boundary values of the initial field: inflow / wall faces carry U
        for a in range(case.ndim):
            if not case.periodic[a]:
                idx = [slice(None)] * case.ndim
                idx[case.ndim - 1 - a] = 0
                self.u[(a,) + tuple(idx)] = case.U[a]
        self.stats = []

    def step(self, dt=None):
        dt = self.dt if dt is None else float(dt)
        st = (Stats * 2)()
        bad = lib().orc_step(C.byref(self.g), C.byref(self.b), self.t, dt, _p(self.u), _p(self.ue),
                             _p(self.P), C.byref(self.S), st)
        self.stats.append((st[0].vcycles, st[0].rel_resid, st[1].vcycles, st[1].rel_resid))
        self.t += dt
        self.dt = cfl(self.g, self.u, self.ue, self.case.cfl, self.case.dt_max)
        return bad, dt
