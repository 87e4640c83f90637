"""Seeded synthetic workloads for the cut-cell elliptic solver.

This module holds problem *data* only: domain descriptions (curve kinds and
parameters), grid sizes, PDE coefficients, manufactured solutions given in
closed form, and seeded random draws.  It contains none of the method's
arithmetic (no cut cells, cubature, stencils, fits or solvers), so both the
CUDA path and the CPU oracle may import it without sharing any of the method.

Problem statement (Sec. 1, eq. ccEllipticEq): a u_xx + b u_xy + c u_yy = f in
Omega with b^2 - 4ac < 0; boundary operators (Sec. 3.3): Dirichlet (N = I) and
Neumann (N = d/dn, n the outward unit normal of Omega).

Curve conventions (shared by every consumer):
  CIRCLE  p = (cx, cy, r)                 gamma(t) = c + r (cos t, sin t)
  ELLIPSE p = (cx, cy, a, b, phi)         gamma(t) = c + Rot(phi) (a cos t, b sin t)
  STAR    p = (cx, cy, r0, amp, k)        gamma(t) = c + (r0 + amp cos(k t)) (cos t, sin t)
with t in [0, 2 pi), counter-clockwise.  orient = +1 means Omega lies inside the
curve, -1 means the curve bounds a hole.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

CIRCLE, ELLIPSE, STAR, POLYGON, SPLINE = 1, 2, 3, 4, 5
NONE, DIRICHLET, NEUMANN, ROBIN = 0, 1, 2, 3


@dataclass
class Curve:
    kind: int
    params: Sequence[float]
    orient: int = -1
    bc: int = DIRICHLET
    robin: Sequence[float] = (1.0, 0.0)   # ROBIN: (gamma1, gamma2) of gamma1 u + gamma2 du/dn


@dataclass
class Problem:
    """Box R = [x0, x0 + nx h] x [y0, y0 + ny h] and the curves cut out of it."""
    a: float
    b: float
    c: float
    x0: float
    y0: float
    h: float
    nx: int
    ny: int
    box_bc: int
    curves: List[Curve] = field(default_factory=list)
    name: str = ""


@dataclass
class Manufactured:
    """Closed-form u and its derivatives (vectorised over numpy arrays)."""
    u: Callable
    ux: Callable
    uy: Callable
    uxx: Callable
    uxy: Callable
    uyy: Callable
    name: str = ""

    def f(self, a: float, b: float, c: float) -> Callable:
        return lambda x, y: a * self.uxx(x, y) + b * self.uxy(x, y) + c * self.uyy(x, y)


# ---------------------------------------------------------------- manufactured solutions

def mms_disk() -> Manufactured:
    """u = sin(2 pi x) cos(3 pi y) exp(x y)."""
    P2, P3 = 2 * math.pi, 3 * math.pi

    def u(x, y):
        return np.sin(P2 * x) * np.cos(P3 * y) * np.exp(x * y)

    def ux(x, y):
        e = np.exp(x * y)
        return (P2 * np.cos(P2 * x) + y * np.sin(P2 * x)) * np.cos(P3 * y) * e

    def uy(x, y):
        e = np.exp(x * y)
        return np.sin(P2 * x) * (-P3 * np.sin(P3 * y) + x * np.cos(P3 * y)) * e

    def uxx(x, y):
        e = np.exp(x * y)
        s, co = np.sin(P2 * x), np.cos(P2 * x)
        return (-P2 * P2 * s + 2 * y * P2 * co + y * y * s) * np.cos(P3 * y) * e

    def uyy(x, y):
        e = np.exp(x * y)
        s, co = np.sin(P3 * y), np.cos(P3 * y)
        return np.sin(P2 * x) * (-P3 * P3 * co - 2 * x * P3 * s + x * x * co) * e

    def uxy(x, y):
        e = np.exp(x * y)
        sx, cx = np.sin(P2 * x), np.cos(P2 * x)
        sy, cy = np.sin(P3 * y), np.cos(P3 * y)
        A = P2 * cx + y * sx          # d/dx of (sin(2pi x) e^{xy}) / e^{xy}
        B = -P3 * sy + x * cy         # d/dy of (cos(3pi y) e^{xy}) / e^{xy}
        # u = sx*cy*e ; u_x = A cy e ; u_xy = d/dy[A cy e] = sx cy e + A (-P3 sy) e + A cy x e
        return (sx * cy + A * B) * e

    return Manufactured(u, ux, uy, uxx, uxy, uyy, "sin(2pi x)cos(3pi y)exp(xy)")


def mms_star() -> Manufactured:
    """u = exp(x) sin(pi y) + x^4."""
    P = math.pi
    return Manufactured(
        u=lambda x, y: np.exp(x) * np.sin(P * y) + x ** 4,
        ux=lambda x, y: np.exp(x) * np.sin(P * y) + 4 * x ** 3,
        uy=lambda x, y: P * np.exp(x) * np.cos(P * y),
        uxx=lambda x, y: np.exp(x) * np.sin(P * y) + 12 * x ** 2,
        uxy=lambda x, y: P * np.exp(x) * np.cos(P * y),
        uyy=lambda x, y: -P * P * np.exp(x) * np.sin(P * y),
        name="exp(x)sin(pi y)+x^4")


def mms_ellipses() -> Manufactured:
    """u = cos(pi x) cos(pi y) + x y^3."""
    P = math.pi
    return Manufactured(
        u=lambda x, y: np.cos(P * x) * np.cos(P * y) + x * y ** 3,
        ux=lambda x, y: -P * np.sin(P * x) * np.cos(P * y) + y ** 3,
        uy=lambda x, y: -P * np.cos(P * x) * np.sin(P * y) + 3 * x * y ** 2,
        uxx=lambda x, y: -P * P * np.cos(P * x) * np.cos(P * y),
        uxy=lambda x, y: P * P * np.sin(P * x) * np.sin(P * y) + 3 * y ** 2,
        uyy=lambda x, y: -P * P * np.cos(P * x) * np.cos(P * y) + 6 * x * y,
        name="cos(pi x)cos(pi y)+x y^3")


def mms_polynomial(coef: Sequence[float]) -> Manufactured:
    """u = sum_{p+q<=4} coef[k] x^p y^q (graded order (0,0),(1,0),(0,1),(2,0),...)."""
    exps = [(d - q, q) for d in range(5) for q in range(d + 1)]
    coef = list(coef) + [0.0] * (15 - len(coef))

    def mk(dx, dy):
        def g(x, y):
            out = np.zeros(np.broadcast(x, y).shape)
            for cf, (p, q) in zip(coef, exps):
                if cf == 0.0 or p < dx or q < dy:
                    continue
                fp = math.perm(p, dx)
                fq = math.perm(q, dy)
                out = out + cf * fp * fq * np.power(x, p - dx) * np.power(y, q - dy)
            return out
        return g

    return Manufactured(mk(0, 0), mk(1, 0), mk(0, 1), mk(2, 0), mk(1, 1), mk(0, 2), "poly4")


# ---------------------------------------------------------------- domains

def disk_minus(n: int, r: float = 0.2) -> Problem:
    """Unit square minus a disk of radius r centred at (0.5, 0.5); Dirichlet everywhere."""
    return Problem(1.0, 0.0, 1.0, 0.0, 0.0, 1.0 / n, n, n, DIRICHLET,
                   [Curve(CIRCLE, (0.5, 0.5, r), -1, DIRICHLET)], name=f"disk_minus_{n}")


def disk_robin(n: int, gamma=(1.0, 0.5), r: float = 0.2, abc=(1.0, 0.0, 1.0)) -> Problem:
    """Unit square minus a disk of radius r centred at (0.5, 0.5): Dirichlet on the box, the
    Robin condition gamma1 u + gamma2 du/dn = g on the circle (n the outward normal of the
    domain, pointing into the disk)."""
    a, b, c = abc
    return Problem(a, b, c, 0.0, 0.0, 1.0 / n, n, n, DIRICHLET,
                   [Curve(CIRCLE, (0.5, 0.5, r), -1, ROBIN, tuple(gamma))], name=f"disk_robin_{n}")


def spline_blob(n: int, npts: int = 12, seed: int = 0, abc=(1.0, 0.5, 2.0), bc: int = DIRICHLET) -> Problem:
    """Interior of a closed cubic spline (a Y_c boundary, Sec. 2) through npts points
    (0.5, 0.5) + r_k (cos th_k, sin th_k), th_k = 2 pi (k + u_k) / npts with u_k ~ U[-0.2, 0.2]
    and r_k ~ U[0.25, 0.35] drawn with numpy's PCG64(seed), inside [0,1]^2; bc on the curve."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.uniform(-0.2, 0.2, npts)
    r = rng.uniform(0.25, 0.35, npts)
    th = 2 * math.pi * (np.arange(npts) + u) / npts
    pts = np.column_stack([0.5 + r * np.cos(th), 0.5 + r * np.sin(th)]).ravel()
    a, b, c = abc
    return Problem(a, b, c, 0.0, 0.0, 1.0 / n, n, n, NONE, [Curve(SPLINE, tuple(float(v) for v in pts), +1, bc)],
                   name=f"spline_blob_{n}")


def star(n: int, abc=(1.0, 0.5, 2.0), r0=0.3, amp=0.08, k=5, centre=(0.5, 0.5)) -> Problem:
    """Interior of the star r(t) = r0 + amp cos(k t) inside [0,1]^2; Dirichlet on the curve."""
    a, b, c = abc
    return Problem(a, b, c, 0.0, 0.0, 1.0 / n, n, n, NONE,
                   [Curve(STAR, (centre[0], centre[1], r0, amp, float(k)), +1, DIRICHLET)],
                   name=f"star_{n}")


GEOMETRY_GRIDS = (128, 256, 512, 1024)


def geometry_of_seed(seed: int) -> Tuple[Problem, "Manufactured"]:
    """One geometry of the many-geometry workload, with its manufactured solution.  numpy's
    PCG64(seed) draws, in this order: the grid n uniformly from {128, 256, 512, 1024}; the kind
    (star or three-ellipse domain, even odds); then for a star r = r0 + amp cos(k t) centred at
    (0.5, 0.5) the values r0 ~ U[0.25, 0.32], amp ~ U[0.05, 0.1], k uniform in {3, ..., 7}
    with the coefficients and manufactured u of the star workload ((a, b, c) = (1, 0.5, 2),
    Dirichlet on the curve); for the other kind the unit square minus three ellipses placed
    with PCG64(seed) (three_ellipses), with the coefficients, boundary conditions and
    manufactured u of the three-ellipse workload ((1, 0, 1), Neumann on the ellipses,
    Dirichlet on the box)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(GEOMETRY_GRIDS[rng.integers(0, len(GEOMETRY_GRIDS))])
    if rng.integers(0, 2) == 0:
        r0, amp = float(rng.uniform(0.25, 0.32)), float(rng.uniform(0.05, 0.1))
        k = int(rng.integers(3, 8))
        p = star(n, (1.0, 0.5, 2.0), r0, amp, k)
        p.name = f"geom{seed}_star{k}_{n}"
        return p, mms_star()
    p = three_ellipses(n, seed=seed, min_gap=1.0 / 8)
    p.name = f"geom{seed}_ellipses_{n}"
    return p, mms_ellipses()


def many_geometries(count: int = 64, seed0: int = 0) -> List[Tuple[Problem, "Manufactured"]]:
    """The independent geometries (with manufactured solutions) of seeds seed0 .. seed0 +
    count - 1 (geometry_of_seed)."""
    return [geometry_of_seed(seed0 + k) for k in range(count)]


def three_ellipses(n: int, seed: int = 0, abc=(1.0, 0.0, 1.0), curve_bc: int = NEUMANN,
                   gap_cells: float = 4.0, min_gap: float = 1.0 / 16) -> Problem:
    """Unit square minus three disjoint ellipses (semi-axes 0.10x0.06, 0.08x0.08, 0.12x0.05).

    Centres (uniform in the unit square) and rotations (uniform in [0, pi)) are drawn with
    numpy's PCG64(seed) by rejection, so that every pair of ellipses and every ellipse and
    the box keep a gap of at least max(gap_cells*h, 1/16), checked on 720 samples per
    curve.  The floor min_gap (1/16) keeps the geometry the same for every n >= 64 and leaves
    the curves separated on the coarse multigrid levels too."""
    h = 1.0 / n
    rng = np.random.Generator(np.random.PCG64(seed))
    axes = [(0.10, 0.06), (0.08, 0.08), (0.12, 0.05)]
    gap = max(gap_cells * h, min_gap)
    ts = np.linspace(0.0, 2 * math.pi, 721)
    placed, params = [], []
    for (ea, eb) in axes:
        for _ in range(100000):
            cx, cy = rng.uniform(0.0, 1.0, size=2)
            phi = rng.uniform(0.0, math.pi)
            px = cx + ea * np.cos(ts) * math.cos(phi) - eb * np.sin(ts) * math.sin(phi)
            py = cy + ea * np.cos(ts) * math.sin(phi) + eb * np.sin(ts) * math.cos(phi)
            if px.min() < gap or py.min() < gap or px.max() > 1 - gap or py.max() > 1 - gap:
                continue
            ok = True
            for (qx, qy, qc) in placed:
                d = np.sqrt((px[:, None] - qx[None, :]) ** 2 + (py[:, None] - qy[None, :]) ** 2)
                if d.min() < gap:
                    ok = False
                    break
            if ok:
                placed.append((px, py, (cx, cy)))
                params.append((float(cx), float(cy), ea, eb, float(phi)))
                break
        else:  # pragma: no cover
            raise RuntimeError("could not place ellipses")
    a, b, c = abc
    curves = [Curve(ELLIPSE, p, -1, curve_bc) for p in params]
    return Problem(a, b, c, 0.0, 0.0, h, n, n, DIRICHLET, curves, name=f"three_ellipses_{n}")


def smoothed_normal_rhs(n: int, nrhs: int, mask: np.ndarray, seed: int = 0) -> np.ndarray:
    """nrhs fields of i.i.d. N(0,1) cell values smoothed by three sweeps of
    v <- v/2 + (sum of the 4 neighbours)/8 restricted to the cells where mask is true.
    Returns an array [nrhs, n, n] (zero outside mask)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal((nrhs, n, n)) * mask[None]
    m = mask.astype(np.float64)[None]
    for _ in range(3):
        s = np.zeros_like(v)
        s[:, 1:, :] += v[:, :-1, :]
        s[:, :-1, :] += v[:, 1:, :]
        s[:, :, 1:] += v[:, :, :-1]
        s[:, :, :-1] += v[:, :, 1:]
        v = (0.5 * v + 0.125 * s) * m
    return v


CONFIGS = {
    "disk64": lambda: (disk_minus(64), mms_disk()),
    "star256": lambda: (star(256), mms_star()),
    "star1024": lambda: (star(1024), mms_star()),
    "star4096": lambda: (star(4096), mms_star()),
    "ellipses2048": lambda: (three_ellipses(2048), mms_ellipses()),
    "disk512": lambda: (disk_minus(512), mms_disk()),
    "star2048_adj": lambda: (star(2048, (1.0, 0.3, 1.0)), mms_star()),
}


def paper_problem1(n: int) -> Problem:
    """The paper's Problem 1 (Sec. 5.1): Poisson on the unit box centred at the origin outside
    the flower r >= 0.25 + 0.05 cos(6 theta); Dirichlet on the box, Neumann on the flower."""
    return Problem(1.0, 0.0, 1.0, -0.5, -0.5, 1.0 / n, n, n, DIRICHLET,
                   [Curve(STAR, (0.0, 0.0, 0.25, 0.05, 6.0), -1, NEUMANN)], name=f"paper_problem1_{n}")


def mms_problem1() -> Manufactured:
    """u = r^4 cos(3 theta) = r (x^3 - 3 x y^2), r = |(x, y)| (Problem 1; smooth away from 0)."""
    def parts(x, y):
        s = np.sqrt(x * x + y * y)
        return s, x ** 3 - 3 * x * y * y

    def u(x, y):
        s, q = parts(x, y)
        return s * q

    def ux(x, y):
        s, q = parts(x, y)
        return x / s * q + s * (3 * x * x - 3 * y * y)

    def uy(x, y):
        s, q = parts(x, y)
        return y / s * q - 6 * s * x * y

    def uxx(x, y):
        s, q = parts(x, y)
        return y * y / s ** 3 * q + 2 * x / s * (3 * x * x - 3 * y * y) + 6 * x * s

    def uyy(x, y):
        s, q = parts(x, y)
        return x * x / s ** 3 * q - 12 * x * y * y / s - 6 * x * s

    def uxy(x, y):
        s, q = parts(x, y)
        return -x * y / s ** 3 * q - 6 * x * x * y / s + y / s * (3 * x * x - 3 * y * y) - 6 * y * s

    return Manufactured(u, ux, uy, uxx, uxy, uyy, "r^4 cos 3theta")


def paper_problem3(n: int) -> Problem:
    """The paper's Problem 3, case (i) (Sec. 5.1): a u_xx + c u_yy = f with (a, b, c) = (1, 0, 2)
    on the unit box [0,1]^2, Dirichlet on its sides (no curve: every boundary piece is a
    box wall)."""
    return Problem(1.0, 0.0, 2.0, 0.0, 0.0, 1.0 / n, n, n, DIRICHLET, [], name=f"paper_problem3_{n}")


def mms_problem3() -> Manufactured:
    """u = sin(4 x) cos(3 y) (Problem 3, case (i))."""
    return Manufactured(lambda x, y: np.sin(4 * x) * np.cos(3 * y),
                        lambda x, y: 4 * np.cos(4 * x) * np.cos(3 * y),
                        lambda x, y: -3 * np.sin(4 * x) * np.sin(3 * y),
                        lambda x, y: -16 * np.sin(4 * x) * np.cos(3 * y),
                        lambda x, y: -12 * np.cos(4 * x) * np.sin(3 * y),
                        lambda x, y: -9 * np.sin(4 * x) * np.cos(3 * y),
                        "sin 4x cos 3y")


ROT3 = math.pi / 6          # Problem 3, case (ii): the box rotated counter-clockwise by pi/6
ROT3_CENTRE = (0.5, 0.5)


def paper_problem3_rotated(n: int) -> Problem:
    """The paper's Problem 3, case (ii) (Sec. 5.1): the unit box rotated counter-clockwise by
    pi/6 (here about its centre (1/2, 1/2)), with (a, b, c) = (5/4, -sqrt(3)/2, 7/4), the
    coefficients of case (i) seen in the rotated frame; Dirichlet on the four sides.  The box
    is a polygon curve; the grid has cell size 1/n on the square [-1/4, 5/4]^2 (3n/2 cells a
    side), which holds the rotated box with a margin of 0.067."""
    c, s = math.cos(ROT3), math.sin(ROT3)
    cx, cy = ROT3_CENTRE
    verts = []
    for (X, Y) in ((-0.5, -0.5), (0.5, -0.5), (0.5, 0.5), (-0.5, 0.5)):
        verts += [cx + c * X - s * Y, cy + s * X + c * Y]
    m = 3 * n // 2
    return Problem(1.25, -math.sqrt(3.0) / 2.0, 1.75, -0.25, -0.25, 1.0 / n, m, m, NONE,
                   [Curve(POLYGON, tuple(verts), +1, DIRICHLET)], name=f"paper_problem3_rotated_{n}")


def mms_problem3_rotated() -> Manufactured:
    """Case (ii)'s exact solution: v(x') = sin(4 x1') cos(3 x2') of case (i) at the pre-image
    x' = Q^T (x - c) + c of x under the rotation Q by pi/6 about c = (1/2, 1/2); its gradient
    and Hessian are Q grad v and Q (Hess v) Q^T."""
    c, s = math.cos(ROT3), math.sin(ROT3)
    cx, cy = ROT3_CENTRE

    def pre(x, y):
        dx, dy = x - cx, y - cy
        return cx + c * dx + s * dy, cy - s * dx + c * dy

    def v(x, y):
        X, Y = pre(x, y)
        return np.sin(4 * X) * np.cos(3 * Y), 4 * np.cos(4 * X) * np.cos(3 * Y), -3 * np.sin(4 * X) * np.sin(3 * Y), \
            -16 * np.sin(4 * X) * np.cos(3 * Y), -12 * np.cos(4 * X) * np.sin(3 * Y), -9 * np.sin(4 * X) * np.cos(3 * Y)

    def ux(x, y):
        _, v1, v2, *_ = v(x, y)
        return c * v1 - s * v2

    def uy(x, y):
        _, v1, v2, *_ = v(x, y)
        return s * v1 + c * v2

    def uxx(x, y):
        _, _, _, h11, h12, h22 = v(x, y)
        return c * c * h11 - 2 * c * s * h12 + s * s * h22

    def uxy(x, y):
        _, _, _, h11, h12, h22 = v(x, y)
        return c * s * (h11 - h22) + (c * c - s * s) * h12

    def uyy(x, y):
        _, _, _, h11, h12, h22 = v(x, y)
        return s * s * h11 + 2 * c * s * h12 + c * c * h22

    return Manufactured(lambda x, y: v(x, y)[0], ux, uy, uxx, uxy, uyy, "sin 4x' cos 3y', x' rotated by pi/6")


def mms_sinsin() -> Manufactured:
    """u = sin(pi x) sin(pi y) (the exact solution of the paper's Problem 2)."""
    P = math.pi
    return Manufactured(
        u=lambda x, y: np.sin(P * x) * np.sin(P * y),
        ux=lambda x, y: P * np.cos(P * x) * np.sin(P * y),
        uy=lambda x, y: P * np.sin(P * x) * np.cos(P * y),
        uxx=lambda x, y: -P * P * np.sin(P * x) * np.sin(P * y),
        uxy=lambda x, y: P * P * np.cos(P * x) * np.cos(P * y),
        uyy=lambda x, y: -P * P * np.sin(P * x) * np.sin(P * y),
        name="sin(pi x)sin(pi y)")


def paper_problem2(n: int, curve_bc: int = DIRICHLET) -> Problem:
    """The paper's Problem 2 (Sec. 5.1): Poisson on [0,1]^2 minus the ellipse with centre
    (1/2, 1/2) and semi-axes (1/8, 1/4); Dirichlet on the box."""
    return Problem(1.0, 0.0, 1.0, 0.0, 0.0, 1.0 / n, n, n, DIRICHLET,
                   [Curve(ELLIPSE, (0.5, 0.5, 0.125, 0.25, 0.0), -1, curve_bc)],
                   name=f"paper_problem2_{n}")
