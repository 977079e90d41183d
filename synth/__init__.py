"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the solver itself: it only produces initial
velocity fields, noise and workload descriptions (grid sizes, viscosity, body
placement and motion). Both the FP64 CPU oracle and the CUDA path receive what
it returns as plain arrays / plain numbers.

Workloads follow the paper's benchmark and validation cases (Sec. 4, the
Taylor-Green vortex, fixed sphere and moving-body cases) at the sizes used for
this solver's five measurement configurations.

Noise generator: SplitMix64 (Steele, Lea & Flood 2014), counter-based.  The
value for component ``a`` at linear cell index ``i`` is
``splitmix64(seed ^ (a * 2**32 + i))`` mapped to [0,1) with its top 53 bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

_M64 = (1 << 64) - 1


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied elementwise to uint64 counters."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, comp: int, count: int) -> np.ndarray:
    """Counter-based uniform [0,1) doubles for one component."""
    ctr = (np.uint64(comp) << np.uint64(32)) + np.arange(count, dtype=np.uint64)
    z = splitmix64(np.uint64(seed & _M64) ^ ctr)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


@dataclass
class Body:
    """Analytic immersed body (Sec. 3: AutoBody = signed distance + motion map).

    kind: "none", "sphere" (a circle when ndim == 2), "ellipse" (2D only),
    "cylinder" (3D, axis along z through the centre's x and y) or "user" (a
    body given by grid samples, see ``sample_body``; the other members unused).
    Motion: centre moves along ``heave_axis`` as
    ``centre + heave_amp * sin(omega * t + phase)``; the ellipse pitches about
    its centre by ``pitch_amp * sin(omega * t + phase + pi/2)``.
    """
    kind: str = "none"
    centre: tuple = (0.0, 0.0, 0.0)
    radius: float = 0.0
    semi: tuple = (0.0, 0.0)          # ellipse semi-axes (chord/2, thickness/2)
    heave_amp: float = 0.0
    pitch_amp: float = 0.0
    omega: float = 0.0
    phase: float = 0.0
    heave_axis: int = 1

    @property
    def kind_id(self) -> int:
        return {"none": 0, "sphere": 1, "ellipse": 2, "cylinder": 3, "user": 4}[self.kind]


@dataclass
class Case:
    """One workload: grid, boundary conditions, viscosity, body, initial field."""
    name: str
    ndim: int
    n: tuple
    periodic: tuple
    exit_hi_x: bool
    U: tuple
    nu: float
    body: Body = field(default_factory=Body)
    eps: float = 1.0
    init: str = "noise"               # "noise" | "tgv2d" | "tgv3d" | "uniform+noise"
    seed: int = 0
    noise_amp: float = 1e-3
    dt0: float = 0.25
    dt_max: float = 1.0
    cfl: float = 1.0
    steps: int = 10

    @property
    def ncell(self) -> int:
        return int(np.prod(self.n[: self.ndim]))

    def with_(self, **kw) -> "Case":
        return replace(self, **kw)


def face_coords(ndim: int, n: tuple, a: int):
    """Coordinates of the lower a-face centres of every cell (cell centre I+1/2)."""
    axes = [np.arange(n[d], dtype=np.float64) + 0.5 for d in range(ndim)]
    axes[a] = axes[a] - 0.5
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]  # x fastest in memory
    return grids  # list [x, y(, z)] each shaped n[::-1]


def initial_velocity(case: Case):
    """Initial staggered velocity u[a] (shape ndim x n[::-1]) and exit plane.

    * "noise": zero field plus i.i.d. uniform noise of +-noise_amp on every
      stored face of every component (then the inflow/wall faces are set by the
      solver's boundary condition).
    * "uniform+noise": U plus the same noise.
    * "tgv3d": u = sin(kx)cos(ky)cos(kz), v = -cos(kx)sin(ky)cos(kz), w = 0,
      k = 2*pi/N (x, y, z taken at each component's own face centre).
    * "tgv2d": u = -sin(kx)cos(ky), v = cos(kx)sin(ky) (Sec. 4 sign convention).
    """
    nd = case.ndim
    shape = tuple(case.n[:nd][::-1])
    u = np.zeros((nd,) + shape, dtype=np.float64)
    if case.init in ("noise", "uniform+noise"):
        cnt = int(np.prod(shape))
        for a in range(nd):
            r = uniform01(case.seed, a, cnt).reshape(shape)
            u[a] = case.noise_amp * (2.0 * r - 1.0)
            if case.init == "uniform+noise":
                u[a] += case.U[a]
    elif case.init == "tgv3d":
        k = 2.0 * math.pi / case.n[0]
        x, y, z = face_coords(3, case.n, 0)
        u[0] = np.sin(k * x) * np.cos(k * y) * np.cos(k * z)
        x, y, z = face_coords(3, case.n, 1)
        u[1] = -np.cos(k * x) * np.sin(k * y) * np.cos(k * z)
    elif case.init == "tgv3d_octant":
        # the same field on one octant of its period: k = pi / n
        k = math.pi / case.n[0]
        x, y, z = face_coords(3, case.n, 0)
        u[0] = np.sin(k * x) * np.cos(k * y) * np.cos(k * z)
        x, y, z = face_coords(3, case.n, 1)
        u[1] = -np.cos(k * x) * np.sin(k * y) * np.cos(k * z)
    elif case.init == "tgv2d":
        k = 2.0 * math.pi / case.n[0]
        x, y = face_coords(2, case.n, 0)
        u[0] = -np.sin(k * x) * np.cos(k * y)
        x, y = face_coords(2, case.n, 1)
        u[1] = np.cos(k * x) * np.sin(k * y)
    else:
        raise ValueError(case.init)
    plane = (case.n[1] * (case.n[2] if nd == 3 else 1))
    ue = np.full(plane, case.U[0], dtype=np.float64) if case.exit_hi_x else np.zeros(max(plane, 1))
    return u, ue


def random_field(seed: int, ndim: int, n: tuple, amp: float = 1.0, offset=(0.0, 0.0, 0.0)):
    """Seeded uniform field in [-amp, amp] (+offset[a]) on every stored face."""
    shape = tuple(n[:ndim][::-1])
    cnt = int(np.prod(shape))
    u = np.empty((ndim,) + shape, dtype=np.float64)
    for a in range(ndim):
        u[a] = amp * (2.0 * uniform01(seed, a, cnt).reshape(shape) - 1.0) + offset[a]
    return u


def random_scalar(seed: int, ndim: int, n: tuple, amp: float = 1.0, comp: int = 7):
    shape = tuple(n[:ndim][::-1])
    cnt = int(np.prod(shape))
    return amp * (2.0 * uniform01(seed, comp, cnt).reshape(shape) - 1.0)


# ---------------------------------------------------------------------------
# The five measurement workloads (readings of their free parameters are stated
# in the design notes: nu from Re on the stated length, body placement, motion).
# ---------------------------------------------------------------------------

def config1_circle(n=(128, 64)) -> Case:
    """2D flow past a fixed circle D=16 at (32,32), Re=250, FP64 (Sec. 4 shape class)."""
    return Case("circle2d", 2, (n[0], n[1], 1), (False, False, False), True,
                (1.0, 0.0, 0.0), 16.0 / 250.0,
                Body("sphere", (32.0, 32.0, 0.0), 8.0), init="noise", steps=200)


def config2_tgv(N=256) -> Case:
    """3D Taylor-Green vortex, triply periodic N^3, Re=1600 on 1/k (Sec. 4 case 1)."""
    k = 2.0 * math.pi / N
    return Case(f"tgv{N}", 3, (N, N, N), (True, True, True), False,
                (0.0, 0.0, 0.0), 1.0 / (k * 1600.0), init="tgv3d", steps=500)


def tgv_octant(N=256) -> Case:
    """The Taylor-Green vortex of period N on its symmetric octant (Sec. 4
    runs the TGV on a reduced domain with symmetry planes): (N/2)^3 cells,
    slip walls on every face (normal velocity 0, tangential zero gradient:
    the field's mirror planes), the same Reynolds number as config2_tgv(N)."""
    k = 2.0 * math.pi / N
    h = N // 2
    return Case(f"tgv_octant{N}", 3, (h, h, h), (False, False, False), False,
                (0.0, 0.0, 0.0), 1.0 / (k * 1600.0), init="tgv3d_octant", steps=500)


def config3_sphere(n=(256, 128, 128), D=32.0, centre=(64.0, 64.0, 64.0), seed=4) -> Case:
    """3D fixed sphere D=32 at (64,64,64), Re=3700, slip walls, convective exit (Sec. 4 case 2)."""
    return Case("sphere3d", 3, tuple(n), (False, False, False), True,
                (1.0, 0.0, 0.0), D / 3700.0,
                Body("sphere", centre, D / 2.0), init="noise", seed=seed, steps=2000)


def config4_ellipse(n=(1024, 512), chord=64.0, A=16.0, theta=math.radians(15.0), centre=(256.0, 256.0)) -> Case:
    """2D heaving + pitching ellipse, chord 64, t/c = 0.12, Re=1000, St=0.3 on the chord."""
    omega = 2.0 * math.pi * 0.3 / chord
    return Case("ellipse2d", 2, (n[0], n[1], 1), (False, False, False), True,
                (1.0, 0.0, 0.0), chord / 1000.0,
                Body("ellipse", (centre[0], centre[1], 0.0), 0.0, (chord / 2.0, 0.06 * chord),
                     heave_amp=A, pitch_amp=theta, omega=omega, heave_axis=1),
                init="noise", steps=400)


def config5_moving_sphere(n=(512, 256, 256), D=48.0, centre=(128.0, 128.0, 128.0)) -> Case:
    """3D sphere D=48 oscillating transversely, amplitude 0.25D, St=0.2, Re=5000."""
    omega = 2.0 * math.pi * 0.2 / D
    return Case("msphere3d", 3, tuple(n), (False, False, False), True,
                (1.0, 0.0, 0.0), D / 5000.0,
                Body("sphere", centre, D / 2.0, heave_amp=0.25 * D, omega=omega, heave_axis=1),
                init="noise", steps=1000)


def cylinder_benchmark(L=64, moving=True) -> Case:
    """The paper's moving-cylinder benchmark shape (Sec. 4): D = L, domain
    9L x 6L x 2L, spanwise periodic, Re = 1000 on D. Readings: centre at
    (2L, 3L), transverse heave of 0.25 D at St = 0.2 (as the moving sphere)."""
    D = float(L)
    omega = 2.0 * math.pi * 0.2 / D if moving else 0.0
    return Case(f"cylinder{L}", 3, (9 * L, 6 * L, 2 * L), (False, False, True), True,
                (1.0, 0.0, 0.0), D / 1000.0,
                Body("cylinder", (2.0 * D, 3.0 * D, 0.0), D / 2.0, heave_amp=0.25 * D if moving else 0.0,
                     omega=omega, heave_axis=1),
                init="noise", steps=100)


def scaled(case: Case, factor: float) -> Case:
    """The same workload on a grid scaled by ``factor`` (sizes, body and nu scale)."""
    nd = case.ndim
    n = tuple(int(round(case.n[d] * factor)) if d < nd else 1 for d in range(3))
    b = case.body
    body = replace(b, centre=tuple(c * factor for c in b.centre), radius=b.radius * factor,
                   semi=tuple(s * factor for s in b.semi), heave_amp=b.heave_amp * factor,
                   omega=b.omega / factor)
    return replace(case, n=n, nu=case.nu * factor, body=body)


# ------------------------------------------------------------- sampled bodies
# A body of any shape is a signed distance function plus a velocity field (the
# paper's distance function and coordinate map, Sec. 3); a user evaluates them
# at the grid's faces and cell centres and hands the samples to
# wl_set_body_fields. The shapes below play that user: each evaluates its
# distance d (> 0 in the fluid), unit normal grad d and body velocity at given
# points; union and difference combine them the way the paper's body
# arithmetic does (Sec. 6: `big + small`, a sphere minus a plane).

class SDF:
    def eval(self, x):
        """x: list of ndim coordinate arrays -> (d, [n_b], [V_b])."""
        raise NotImplementedError

    def __add__(self, other):
        return Union(self, other)

    def __sub__(self, other):
        return Difference(self, other)


@dataclass
class Circle(SDF):
    """Sphere (a circle when ndim == 2) of radius ``radius`` about ``centre``,
    translating with ``velocity`` and, in 2D, spinning at rate ``spin``: the
    map rot(spin t)(x - c) gives the body velocity spin (y - c_y, -(x - c_x))
    (clockwise for spin > 0)."""
    centre: tuple
    radius: float
    velocity: tuple = (0.0, 0.0, 0.0)
    spin: float = 0.0

    def eval(self, x):
        nd = len(x)
        r = [x[a] - self.centre[a] for a in range(nd)]
        rr = np.sqrt(sum(ra * ra for ra in r))
        safe = np.where(rr > 0.0, rr, 1.0)
        n = [np.where(rr > 0.0, ra / safe, 1.0 if a == 0 else 0.0) for a, ra in enumerate(r)]
        V = [np.full_like(rr, float(self.velocity[a])) for a in range(nd)]
        if self.spin != 0.0:
            V[0] = V[0] + self.spin * r[1]
            V[1] = V[1] - self.spin * r[0]
        return rr - self.radius, n, V


@dataclass
class HalfSpace(SDF):
    """The solid half-space behind a plane: d = (x - point) . normal, so the
    fluid lies on the side the unit ``normal`` points to."""
    point: tuple
    normal: tuple

    def eval(self, x):
        nd = len(x)
        nv = np.asarray(self.normal[:nd], dtype=np.float64)
        nv = nv / np.linalg.norm(nv)
        d = sum((x[a] - self.point[a]) * nv[a] for a in range(nd))
        return d, [np.full_like(d, nv[a]) for a in range(nd)], [np.zeros_like(d) for _ in range(nd)]


@dataclass
class Union(SDF):
    """Solid where either body is: d = min(d_a, d_b); normal and velocity of
    the body with the smaller distance (the first on ties)."""
    a: SDF
    b: SDF

    def eval(self, x):
        da, na, Va = self.a.eval(x)
        db, nb, Vb = self.b.eval(x)
        pick = db < da
        return (np.where(pick, db, da), [np.where(pick, q, p) for p, q in zip(na, nb)],
                [np.where(pick, q, p) for p, q in zip(Va, Vb)])


@dataclass
class Difference(SDF):
    """Solid where body a is and body b is not: d = max(d_a, -d_b); normal and
    velocity of the side that sets d (b's normal reversed)."""
    a: SDF
    b: SDF

    def eval(self, x):
        da, na, Va = self.a.eval(x)
        db, nb, Vb = self.b.eval(x)
        pick = -db > da
        return (np.where(pick, -db, da), [np.where(pick, -q, p) for p, q in zip(na, nb)],
                [np.where(pick, q, p) for p, q in zip(Va, Vb)])


def cell_coords(ndim: int, n: tuple):
    """Coordinates of every cell centre (I + 1/2), x fastest in memory."""
    axes = [np.arange(n[d], dtype=np.float64) + 0.5 for d in range(ndim)]
    return np.meshgrid(*axes[::-1], indexing="ij")[::-1]


def sample_body(shape: SDF, ndim: int, n: tuple, dtype=np.float64):
    """Samples of a body for wl_set_body_fields, in ``dtype``:
    d_face (ndim, *grid), n_face (ndim, ndim, *grid), V_face (ndim, *grid) at
    the lower a-face of every cell (component a of the velocity on face a),
    d_cell (*grid) and n_cell (ndim, *grid) at the cell centres."""
    d_face, n_face, V_face = [], [], []
    for a in range(ndim):
        d, nv, V = shape.eval(face_coords(ndim, n, a))
        d_face.append(d)
        n_face.append(np.stack(nv))
        V_face.append(V[a])
    dc, nc, _ = shape.eval(cell_coords(ndim, n))
    cast = lambda v: np.ascontiguousarray(np.asarray(v), dtype=dtype)
    return cast(np.stack(d_face)), cast(np.stack(n_face)), cast(np.stack(V_face)), cast(dc), cast(np.stack(nc))


def spinning_cylinders(D=96, Re=500.0, d_D=0.15, g_D=0.05, xi=1.0, U=1.0):
    """The controlled-cylinder flow of Sec. 6.1: a fixed circle of diameter D at
    (2D, 0) on the symmetry plane y = 0 (a slip wall) of a 6D x 2D domain (the
    upper half of the full flow; uniform inflow U, convective exit), and a small circle of radius r = d_D D / 2 centred at
    distance D/2 + r + g_D D from it, 60 degrees above the downstream axis,
    spinning with surface speed xi U (rate xi U / r). Returns (case, shape,
    spin tangent shape): the last is the small circle's velocity per unit xi
    on the union's geometry, i.e. d(shape velocity)/d xi."""
    R = D / 2.0
    r = d_D * R
    C = (2.0 * D, 0.0)
    c = (C[0] + (R + r + g_D * D) * 0.5, C[1] + (R + r + g_D * D) * math.sqrt(3.0) / 2.0)
    big = Circle(C, R)
    case = Case(f"spin{D}", 2, (6 * D, 2 * D, 1), (False, False, False), True, (U, 0.0, 0.0), U * D / Re,
                Body("user"), init="uniform+noise", steps=0)
    shape = big + Circle(c, r, spin=xi * U / r)
    tangent = Circle(C, R) + Circle(c, r, spin=U / r)
    # the tangent's distance and normal equal the shape's; its velocity is the
    # small circle's at unit xi (the big circle is at rest)
    return case, shape, tangent
