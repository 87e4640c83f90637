"""Oracle geometry: cut cells, their moments, and Alg. 1 merging.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows Sec. 3.1 (cells C_i = (ih, (i+1)h), cut cells C_i cap Omega, boundary
pieces S_i = C_i cap dOmega; empty / pure / interface cells; Alg. 1 cut-cell
generation and merging with threshold theta) and Sec. 2.4 (Green's formula
turning area integrals into boundary integrals, eq. volumeIntegral and
eq. iteratedIntegral, with xi_0 the centre of the cell).

Conventions (shared specification with the CUDA path, implemented separately):
  * cell (i, j): x-index i (fastest), y-index j; arrays are [ny, nx].
  * local frame of cell (i, j): X = (x - xc)/h, Y = (y - yc)/h with (xc, yc) the
    Cartesian cell centre; moments are dimensionless:
        mom[(p, q)] = int_{region} X^p Y^q dX dY       (p + q <= 4)
  * boundary moments over the boundary piece S (arc length s in units of h,
    n the outward unit normal of Omega):
        bm0[(p,q)] = int_S X^p Y^q ds,  bmx = int_S X^p Y^q n_x ds,  bmy likewise.
  * Box walls: where the box is part of dOmega (box_bc != NONE) the wall edges of
    a cell's closure are its boundary piece (reading: open cells never meet the
    box, but the boundary condition must enter through the wall cells).
  * Alg. 1 merge target: the non-empty 4-neighbour with the longest common cut
    face; ties: larger current volume, then the order (+x, -x, +y, -y).  Absorbed
    cells count as empty (volume 0), as in Alg. 1 line 4.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Tuple

import numpy as np
from scipy.optimize import brentq

CIRCLE, ELLIPSE, STAR, POLYGON, SPLINE = 1, 2, 3, 4, 5
NONE, DIRICHLET, NEUMANN, ROBIN = 0, 1, 2, 3
EMPTY, PURE, CUT = 0, 1, 2

# graded monomial order used everywhere: (0,0),(1,0),(0,1),(2,0),(1,1),(0,2),...
EXPS = [(d - q, q) for d in range(5) for q in range(d + 1)]
EIDX = {e: k for k, e in enumerate(EXPS)}

GL_ARC = 12      # Gauss-Legendre points on a curved piece
GL_INNER = 8     # points of the inner (xi) integral of eq. iteratedIntegral


class GeometryError(Exception):
    pass


# ------------------------------------------------------------------ curves

class OCurve:
    """Closed parametric curve gamma(t), t in [0, 2 pi), counter-clockwise.

    POLYGON: params = (x0, y0, x1, y1, ...), n >= 3 vertices in counter-clockwise order; edge
    k is traversed for t in [2 pi k / n, 2 pi (k + 1) / n) at constant speed, so the curve
    has a kink at every t = 2 pi k / n (breaks()).
    SPLINE: params = (x0, y0, ...), n >= 3 points in counter-clockwise order; the periodic
    cubic spline interpolating them in each coordinate, with knots at the cumulative chord
    lengths scaled to [0, 2 pi) (the curves of the Yin sets Y_c, Sec. 2).  The curve is C^2;
    its knots are returned by breaks() so that a Gauss rule never spans two cubics."""

    def __init__(self, kind, params, orient, bc, robin=(1.0, 0.0)):
        self.kind, self.p, self.orient, self.bc = int(kind), tuple(float(v) for v in params), int(orient), int(bc)
        self.robin = (float(robin[0]), float(robin[1]))   # gamma1, gamma2 (Sec. 3.3, the Robin N)
        if self.kind == POLYGON:
            self.V = np.array(self.p, dtype=np.float64).reshape(-1, 2)
            if len(self.V) < 3:
                raise GeometryError("a polygon needs three vertices")
            x, y = self.V[:, 0], self.V[:, 1]
            if np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y) <= 0.0:
                raise GeometryError("polygon vertices must run counter-clockwise")
        if self.kind == SPLINE:
            self.V = np.array(self.p, dtype=np.float64).reshape(-1, 2)
            n = len(self.V)
            if n < 3:
                raise GeometryError("a spline needs three points")
            x, y = self.V[:, 0], self.V[:, 1]
            if np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y) <= 0.0:
                raise GeometryError("spline points must run counter-clockwise")
            chord = np.hypot(np.roll(x, -1) - x, np.roll(y, -1) - y)
            if np.any(chord <= 0.0):
                raise GeometryError("repeated spline point")
            tau = np.concatenate([[0.0], np.cumsum(chord)])
            self.knots = 2 * math.pi * tau / tau[-1]          # t_0 = 0 .. t_n = 2 pi
            self.knots[-1] = 2 * math.pi
            hk = np.diff(self.knots)
            # second derivatives M of the periodic spline: for every knot k (indices mod n)
            # h_{k-1} M_{k-1} + 2 (h_{k-1} + h_k) M_k + h_k M_{k+1}
            #   = 6 ((v_{k+1} - v_k) / h_k - (v_k - v_{k-1}) / h_{k-1})
            A = np.zeros((n, n))
            for k in range(n):
                A[k, (k - 1) % n] += hk[k - 1]
                A[k, k] += 2 * (hk[k - 1] + hk[k])
                A[k, (k + 1) % n] += hk[k]
            self.M = []
            for v in (x, y):
                d = (np.roll(v, -1) - v) / hk
                self.M.append(np.linalg.solve(A, 6 * (d - np.roll(d, 1))))

    def breaks(self):
        """Parameters in [0, 2 pi) where gamma is not smooth."""
        if self.kind == POLYGON:
            n = len(self.V)
            return [2 * math.pi * k / n for k in range(n)]
        if self.kind == SPLINE:
            return list(self.knots[:-1])
        return []

    def _spline(self, t, deriv):
        """The spline's coordinates (deriv 0) or their t-derivatives (deriv 1) at t."""
        n = len(self.V)
        tt = np.mod(np.asarray(t, dtype=np.float64), 2 * math.pi)
        k = np.clip(np.searchsorted(self.knots, tt, side="right") - 1, 0, n - 1)
        k1 = (k + 1) % n
        hk = self.knots[k + 1] - self.knots[k]
        a = (self.knots[k + 1] - tt) / hk
        b = (tt - self.knots[k]) / hk
        out = []
        for c, M in enumerate(self.M):
            v = self.V[:, c]
            if deriv == 0:
                out.append(a * v[k] + b * v[k1] + ((a ** 3 - a) * M[k] + (b ** 3 - b) * M[k1]) * hk * hk / 6)
            else:
                out.append((v[k1] - v[k]) / hk + ((1 - 3 * a * a) * M[k] + (3 * b * b - 1) * M[k1]) * hk / 6)
        return out[0], out[1]

    def _edge(self, t):
        n = len(self.V)
        u = np.asarray(t, dtype=np.float64) * (n / (2 * math.pi))
        k = np.floor(u)
        s = u - k
        k = k.astype(np.int64) % n
        return k, (k + 1) % n, s, n

    def xy(self, t):
        t = np.asarray(t, dtype=np.float64)
        p = self.p
        if self.kind == CIRCLE:
            return p[0] + p[2] * np.cos(t), p[1] + p[2] * np.sin(t)
        if self.kind == ELLIPSE:
            cx, cy, a, b, phi = p
            X, Y = a * np.cos(t), b * np.sin(t)
            return cx + X * math.cos(phi) - Y * math.sin(phi), cy + X * math.sin(phi) + Y * math.cos(phi)
        if self.kind == STAR:
            cx, cy, r0, amp, k = p
            r = r0 + amp * np.cos(k * t)
            return cx + r * np.cos(t), cy + r * np.sin(t)
        if self.kind == POLYGON:
            a, b, s, _ = self._edge(t)
            A, B = self.V[a], self.V[b]
            return A[..., 0] + (B[..., 0] - A[..., 0]) * s, A[..., 1] + (B[..., 1] - A[..., 1]) * s
        if self.kind == SPLINE:
            return self._spline(t, 0)
        raise GeometryError("unknown curve kind")

    def dxy(self, t):
        t = np.asarray(t, dtype=np.float64)
        p = self.p
        if self.kind == CIRCLE:
            return -p[2] * np.sin(t), p[2] * np.cos(t)
        if self.kind == ELLIPSE:
            cx, cy, a, b, phi = p
            dX, dY = -a * np.sin(t), b * np.cos(t)
            return dX * math.cos(phi) - dY * math.sin(phi), dX * math.sin(phi) + dY * math.cos(phi)
        if self.kind == STAR:
            cx, cy, r0, amp, k = p
            r = r0 + amp * np.cos(k * t)
            dr = -amp * k * np.sin(k * t)
            return dr * np.cos(t) - r * np.sin(t), dr * np.sin(t) + r * np.cos(t)
        if self.kind == POLYGON:
            a, b, _, n = self._edge(t)
            A, B = self.V[a], self.V[b]
            sc = n / (2 * math.pi)
            return (B[..., 0] - A[..., 0]) * sc, (B[..., 1] - A[..., 1]) * sc
        if self.kind == SPLINE:
            return self._spline(t, 1)
        raise GeometryError("unknown curve kind")

    def inside(self, x, y):
        """Strictly inside the region the curve encloses."""
        p = self.p
        if self.kind == CIRCLE:
            return (x - p[0]) ** 2 + (y - p[1]) ** 2 < p[2] ** 2
        if self.kind == ELLIPSE:
            cx, cy, a, b, phi = p
            dx, dy = x - cx, y - cy
            X = dx * math.cos(phi) + dy * math.sin(phi)
            Y = -dx * math.sin(phi) + dy * math.cos(phi)
            return (X / a) ** 2 + (Y / b) ** 2 < 1.0
        if self.kind == STAR:
            cx, cy, r0, amp, k = p
            dx, dy = x - cx, y - cy
            th = np.arctan2(dy, dx)
            return np.hypot(dx, dy) < r0 + amp * np.cos(k * th)
        if self.kind == POLYGON:
            # even-odd rule: a ray towards +x crosses the boundary an odd number of times
            x = np.asarray(x, dtype=np.float64)
            y = np.asarray(y, dtype=np.float64)
            ins = np.zeros(np.broadcast(x, y).shape, dtype=bool)
            n = len(self.V)
            for k in range(n):
                (xa, ya), (xb, yb) = self.V[k], self.V[(k + 1) % n]
                if ya == yb:
                    continue
                hit = (ya > y) != (yb > y)
                xs = xa + (y - ya) * (xb - xa) / (yb - ya)
                ins ^= hit & (x < xs)
            return ins
        if self.kind == SPLINE:
            # even-odd rule against the spline sampled 64 times per cubic: used only for
            # centres of cells the curve does not enter (h/2 or more from the curve), far
            # beyond the polyline's deviation from the spline
            t = np.concatenate([np.linspace(self.knots[k], self.knots[k + 1], 64, endpoint=False)
                                for k in range(len(self.V))])
            px, py = self._spline(t, 0)
            return OCurve(POLYGON, np.column_stack([px, py]).ravel(), 1, self.bc).inside(x, y)
        raise GeometryError("unknown curve kind")


def subintervals(c: OCurve, t0: float, t1: float):
    """[t0, t1] (either direction) cut at the curve's kinks, in the order of traversal, so
    that a Gauss rule on each part integrates a smooth integrand."""
    br = c.breaks()
    if not br:
        return [(t0, t1)]
    lo, hi = min(t0, t1), max(t0, t1)
    cuts = []
    for b in br:
        m = math.ceil((lo - b) / (2 * math.pi))
        v = b + 2 * math.pi * m
        while v < hi:
            if v > lo:
                cuts.append(v)
            v += 2 * math.pi
    cuts.sort(reverse=t1 < t0)
    pts = [t0] + cuts + [t1]
    return [(pts[k], pts[k + 1]) for k in range(len(pts) - 1)]


def in_omega(prob, curves, x, y):
    ok = np.ones(np.broadcast(x, y).shape, dtype=bool)
    for c in curves:
        ins = c.inside(x, y)
        ok &= ins if c.orient > 0 else ~ins
    return ok


# ------------------------------------------------------------------ moment helpers

def pure_moments() -> np.ndarray:
    """int_{[-1/2,1/2]^2} X^p Y^q (closed form)."""
    def m1(p):
        return 0.0 if p % 2 else 2.0 * 0.5 ** (p + 1) / (p + 1)
    return np.array([m1(p) * m1(q) for (p, q) in EXPS])


PURE_MOM = pure_moments()


def shift_matrix(dx: float, dy: float) -> np.ndarray:
    """T with (T m)[(p,q)] = sum_{a<=p, b<=q} C(p,a) C(q,b) dx^(p-a) dy^(q-b) m[(a,b)]:
    the moments about a frame with X' = X + dx, Y' = Y + dy (binomial theorem)."""
    T = np.zeros((15, 15))
    for k, (p, q) in enumerate(EXPS):
        for a in range(p + 1):
            for b in range(q + 1):
                T[k, EIDX[(a, b)]] = math.comb(p, a) * math.comb(q, b) * dx ** (p - a) * dy ** (q - b)
    return T


_SHIFT_CACHE: dict = {}


def shift_moments(m: np.ndarray, dx: float, dy: float) -> np.ndarray:
    """Moments about a frame whose origin is moved by (-dx, -dy): X' = X + dx, Y' = Y + dy."""
    key = (dx, dy)
    T = _SHIFT_CACHE.get(key)
    if T is None:
        T = shift_matrix(dx, dy)
        if len(_SHIFT_CACHE) < 100000:
            _SHIFT_CACHE[key] = T
    return T @ m


_GLX, _GLW = np.polynomial.legendre.leggauss(GL_ARC)


# ------------------------------------------------------------------ data model

@dataclass
class Piece:
    """A piece of a cut cell's boundary, in global coordinates.

    kind 'arc': curve index, parameter from t0 to t1 (direction of traversal with
    Omega on the left).  kind 'seg': straight segment P0 -> P1 on a cell edge."""
    kind: str
    curve: int = -1
    t0: float = 0.0
    t1: float = 0.0
    P0: Tuple[float, float] = (0.0, 0.0)
    P1: Tuple[float, float] = (0.0, 0.0)
    wall: bool = False


@dataclass
class Region:
    """One connected piece of a cell: its boundary loop (global coordinates)."""
    pieces: List[Piece]
    home: Tuple[int, int]     # Cartesian cell the loop lives in


@dataclass
class CutGrid:
    x0: float
    y0: float
    h: float
    nx: int
    ny: int
    status: np.ndarray                   # [ny, nx] EMPTY / PURE / CUT (post-merge)
    owner: np.ndarray                    # [ny, nx] linear index of the survivor, -1 if empty
    vol: np.ndarray                      # [ny, nx] volume / h^2 (post-merge, 0 for empty)
    interface: np.ndarray                # [ny, nx] bool: pre-merge interface cells
    regions: Dict[int, List[Region]]     # non-pure cells: constituent loops
    mom: Dict[int, np.ndarray]           # non-pure cells: 15 moments in own frame
    bpieces: Dict[int, List[Piece]]      # cells with a boundary piece
    bm0: Dict[int, np.ndarray] = field(default_factory=dict)
    bmx: Dict[int, np.ndarray] = field(default_factory=dict)
    bmy: Dict[int, np.ndarray] = field(default_factory=dict)
    bc: Dict[int, int] = field(default_factory=dict)
    robin: Dict[int, tuple] = field(default_factory=dict)   # ROBIN cells: (gamma1, gamma2)
    arcs_of: Dict[int, list] = field(default_factory=dict)   # pre-merge arcs per interface cell

    def centre(self, i, j):
        return self.x0 + (i + 0.5) * self.h, self.y0 + (j + 0.5) * self.h

    def moments(self, lin: int) -> np.ndarray:
        if lin in self.mom:
            return self.mom[lin]
        return PURE_MOM

    def nonempty(self) -> np.ndarray:
        return self.status != EMPTY


# ------------------------------------------------------------------ Green integrals of a piece

def piece_moments(pc: Piece, curves, xc, yc, h) -> np.ndarray:
    """sum over the piece of int X^{p+1}/(p+1) Y^q dY (eq. volumeIntegral with xi0 = xc)."""
    out = np.zeros(15)
    if pc.kind == 'seg':
        X0, Y0 = (pc.P0[0] - xc) / h, (pc.P0[1] - yc) / h
        X1, Y1 = (pc.P1[0] - xc) / h, (pc.P1[1] - yc) / h
        if Y0 == Y1:
            return out
        # straight segment: parametrise linearly, integrate exactly with GL (degree <= 6)
        z, w = np.polynomial.legendre.leggauss(6)
        s = 0.5 * (z + 1.0)
        X = X0 + (X1 - X0) * s
        Y = Y0 + (Y1 - Y0) * s
        dY = (Y1 - Y0) * 0.5 * w
        for k, (p, q) in enumerate(EXPS):
            out[k] = np.sum(X ** (p + 1) / (p + 1) * Y ** q * dY)
        return out
    c = curves[pc.curve]
    for (a, b) in subintervals(c, pc.t0, pc.t1):
        tm, tr = 0.5 * (a + b), 0.5 * (b - a)
        t = tm + tr * _GLX
        x, y = c.xy(t)
        _, dy = c.dxy(t)
        X, Y = (x - xc) / h, (y - yc) / h
        dY = dy / h * tr * _GLW
        for k, (p, q) in enumerate(EXPS):
            out[k] += np.sum(X ** (p + 1) / (p + 1) * Y ** q * dY)
    return out


def piece_boundary_moments(pc: Piece, curves, xc, yc, h):
    """int X^p Y^q ds, int X^p Y^q n_x ds, int X^p Y^q n_y ds over one boundary piece.

    The piece is traversed with Omega on its left, so the outward normal is the
    right-hand normal (dY/ds, -dX/ds)."""
    if pc.kind == 'seg':
        z, w = np.polynomial.legendre.leggauss(6)
        s = 0.5 * (z + 1.0)
        X0, Y0 = (pc.P0[0] - xc) / h, (pc.P0[1] - yc) / h
        X1, Y1 = (pc.P1[0] - xc) / h, (pc.P1[1] - yc) / h
        X = X0 + (X1 - X0) * s
        Y = Y0 + (Y1 - Y0) * s
        L = math.hypot(X1 - X0, Y1 - Y0)
        ds = L * 0.5 * w
        nx_, ny_ = (Y1 - Y0) / L, -(X1 - X0) / L
        nx_ = np.full_like(X, nx_)
        ny_ = np.full_like(X, ny_)
    else:
        c = curves[pc.curve]
        parts = []
        for (a, b) in subintervals(c, pc.t0, pc.t1):
            tm, tr = 0.5 * (a + b), 0.5 * (b - a)
            t = tm + tr * _GLX
            x, y = c.xy(t)
            dx, dy = c.dxy(t)
            sp = np.hypot(dx, dy)
            sgn = 1.0 if tr > 0 else -1.0
            parts.append(((x - xc) / h, (y - yc) / h, sp / h * abs(tr) * _GLW, sgn * dy / sp, -sgn * dx / sp))
        X, Y, ds, nx_, ny_ = (np.concatenate([pt[m] for pt in parts]) for m in range(5))
    b0, bx, by = np.zeros(15), np.zeros(15), np.zeros(15)
    for k, (p, q) in enumerate(EXPS):
        mono = X ** p * Y ** q * ds
        b0[k] = np.sum(mono)
        bx[k] = np.sum(mono * nx_)
        by[k] = np.sum(mono * ny_)
    return b0, bx, by


# ------------------------------------------------------------------ cut-cell generation

def _crossings(c: OCurve, idx: int, x0, y0, h, nx, ny):
    """All transversal crossings of curve c with the grid lines, sorted by t in [0, 2 pi).

    The curve is sampled periodically (the last sample is the first one again), a
    crossing of the line x = x0 + k h is bracketed where floor((x - x0)/h) changes
    between neighbouring samples, and refined by Brent's method."""
    ts = np.linspace(0.0, 2 * math.pi, 4097)
    px, py = c.xy(ts)
    tot = np.sum(np.hypot(np.diff(px), np.diff(py)))
    ns = int(max(4096, math.ceil(64.0 * tot / h)))
    t = np.linspace(0.0, 2 * math.pi, ns + 1)
    x, y = c.xy(t)
    x[ns], y[ns] = x[0], y[0]
    out = []
    for axis, v, org in ((0, x, x0), (1, y, y0)):
        fl = np.floor((v - org) / h).astype(np.int64)
        ch = np.nonzero(fl[1:] != fl[:-1])[0]
        for s in ch:
            lo, hi = min(fl[s], fl[s + 1]), max(fl[s], fl[s + 1])
            for k in range(lo + 1, hi + 1):
                L = org + k * h
                fa = v[s] - L
                fb = v[s + 1] - L
                if fa == 0.0:
                    tr = t[s]
                elif fb == 0.0:
                    tr = t[s + 1]
                elif fa * fb > 0.0:
                    # the cell index changed only by the rounding of (v - org) / h: the curve
                    # stays on one side of the line
                    continue
                else:
                    if axis == 0:
                        f = lambda tt: float(c.xy(tt)[0]) - L
                    else:
                        f = lambda tt: float(c.xy(tt)[1]) - L
                    if f(t[s + 1]) * fa > 0.0:      # only at the seam t = 2 pi
                        tr = t[s + 1]
                    else:
                        tr = brentq(f, t[s], t[s + 1], xtol=1e-16, rtol=8.9e-16, maxiter=200)
                out.append((float(tr) % (2 * math.pi), axis, k))
    out.sort()
    # a curve that only touches a grid line gives two crossings of that line at the
    # same parameter: they cancel (the touching point is not a crossing)
    changed = True
    while changed and len(out) > 1:
        changed = False
        for a in range(len(out)):
            b = (a + 1) % len(out)
            ta, axa, ka = out[a]
            tb, axb, kb = out[b]
            dt = (tb - ta) % (2 * math.pi)
            if axa == axb and ka == kb and dt < 1e-12:
                out = [c for n_, c in enumerate(out) if n_ not in (a, b)]
                changed = True
                break
    return out


def _sigma(X, Y, edge):
    """Counter-clockwise perimeter coordinate of a point on the unit cell's boundary."""
    if edge == 0:   # bottom
        return X + 0.5
    if edge == 1:   # right
        return 1.0 + Y + 0.5
    if edge == 2:   # top
        return 2.0 + 0.5 - X
    return 3.0 + 0.5 - Y   # left


_CORNERS = [(-0.5, -0.5), (0.5, -0.5), (0.5, 0.5), (-0.5, 0.5)]   # at sigma = 0, 1, 2, 3


def _sigma_point(s):
    s = s % 4.0
    e = int(math.floor(s))
    f = s - e
    if e == 0:
        return (-0.5 + f, -0.5)
    if e == 1:
        return (0.5, -0.5 + f)
    if e == 2:
        return (0.5 - f, 0.5)
    return (-0.5, 0.5 - f)


def cut_cells(prob, theta: float = 0.3) -> CutGrid:
    """Cut cells of prob's grid, with Alg. 1 merging (threshold theta)."""
    x0, y0, h, nx, ny = prob.x0, prob.y0, prob.h, prob.nx, prob.ny
    curves = [OCurve(c.kind, c.params, c.orient, c.bc, getattr(c, "robin", (1.0, 0.0))) for c in prob.curves]
    walls = prob.box_bc != NONE

    # ---- arcs: curve pieces between consecutive grid-line crossings (one cell each)
    arcs_of: Dict[int, list] = {}
    for ci, c in enumerate(curves):
        cr = _crossings(c, ci, x0, y0, h, nx, ny)
        if len(cr) < 2:
            raise GeometryError("curve does not cross the grid")
        m = len(cr)
        for a in range(m):
            ta, axa, ka = cr[a]
            tb, axb, kb = cr[(a + 1) % m]
            if a == m - 1:
                tb += 2 * math.pi
            if tb - ta < 1e-12:
                continue      # zero-length piece where the curve passes through a grid vertex
            xm, ym = c.xy(0.5 * (ta + tb))
            i = int(math.floor((float(xm) - x0) / h))
            j = int(math.floor((float(ym) - y0) / h))
            if not (0 <= i < nx and 0 <= j < ny):
                raise GeometryError("curve leaves the box")
            xc, yc = x0 + (i + 0.5) * h, y0 + (j + 0.5) * h

            def endpoint(tt, ax, k):
                px, py = c.xy(tt)
                X, Y = (float(px) - xc) / h, (float(py) - yc) / h
                if ax == 0:
                    if k == i:
                        return -0.5, min(max(Y, -0.5), 0.5), 3
                    if k == i + 1:
                        return 0.5, min(max(Y, -0.5), 0.5), 1
                else:
                    if k == j:
                        return min(max(X, -0.5), 0.5), -0.5, 0
                    if k == j + 1:
                        return min(max(X, -0.5), 0.5), 0.5, 2
                raise GeometryError("inconsistent crossing")

            Xa, Ya, ea = endpoint(ta, axa, ka)
            Xb, Yb, eb = endpoint(tb, axb, kb)
            if c.orient > 0:
                arc = (ci, ta, tb, _sigma(Xa, Ya, ea), _sigma(Xb, Yb, eb), (Xa, Ya), (Xb, Yb))
            else:
                arc = (ci, tb, ta, _sigma(Xb, Yb, eb), _sigma(Xa, Ya, ea), (Xb, Yb), (Xa, Ya))
            arcs_of.setdefault(j * nx + i, []).append(arc)

    # ---- classification of cells without arcs by their centres
    ic = x0 + (np.arange(nx) + 0.5) * h
    jc = y0 + (np.arange(ny) + 0.5) * h
    XX, YY = np.meshgrid(ic, jc)
    inside = in_omega(prob, curves, XX, YY)
    status = np.where(inside, PURE, EMPTY).astype(np.int8)
    interface = np.zeros((ny, nx), dtype=bool)
    for lin in arcs_of:
        interface[lin // nx, lin % nx] = True
        status[lin // nx, lin % nx] = CUT

    # ---- loops of every interface cell
    regions: Dict[int, List[Region]] = {}
    for lin, arcs in arcs_of.items():
        j, i = divmod(lin, nx)
        xc, yc = x0 + (i + 0.5) * h, y0 + (j + 0.5) * h
        todo = list(range(len(arcs)))
        loops = []
        while todo:
            first = todo[0]
            cur = first
            pieces = []
            guard = 0
            while True:
                guard += 1
                if guard > 4 * len(arcs) + 4:
                    raise GeometryError("loop construction failed")
                todo.remove(cur)
                ci, ts, te, s_in, s_out, P_in, P_out = arcs[cur]
                pieces.append(Piece('arc', curve=ci, t0=ts, t1=te))
                # next entry counter-clockwise from the exit point
                best, bd = None, None
                for k, ak in enumerate(arcs):
                    d = (ak[3] - s_out) % 4.0
                    if bd is None or d < bd:
                        best, bd = k, d
                # straight walk from s_out to s_out + bd through the corners
                sa, sb = s_out, s_out + bd
                pts = [_sigma_point(sa)]
                cidx = math.floor(sa) + 1
                while cidx < sb:
                    pts.append(_CORNERS[cidx % 4])
                    cidx += 1
                pts.append(_sigma_point(sb))
                # exact endpoints for the arc ends
                pts[0] = P_out
                pts[-1] = arcs[best][5]
                for (Pa, Pb) in zip(pts[:-1], pts[1:]):
                    if Pa == Pb:
                        continue
                    G0 = (xc + Pa[0] * h, yc + Pa[1] * h)
                    G1 = (xc + Pb[0] * h, yc + Pb[1] * h)
                    on_wall = walls and (
                        (Pa[0] == Pb[0] == -0.5 and i == 0) or (Pa[0] == Pb[0] == 0.5 and i == nx - 1) or
                        (Pa[1] == Pb[1] == -0.5 and j == 0) or (Pa[1] == Pb[1] == 0.5 and j == ny - 1))
                    pieces.append(Piece('seg', P0=G0, P1=G1, wall=on_wall))
                cur = best
                if cur == first:
                    break
                if cur not in todo:
                    raise GeometryError("loop construction failed")
            loops.append(Region(pieces, (i, j)))
        regions[lin] = loops

    def loop_moments(reg: Region):
        i, j = reg.home
        xc, yc = x0 + (i + 0.5) * h, y0 + (j + 0.5) * h
        m = np.zeros(15)
        for pc in reg.pieces:
            m += piece_moments(pc, curves, xc, yc, h)
        return m

    def face_len(reg: Region, d: int) -> float:
        """Length (units of h) of the loop's straight pieces on edge d (0:+x,1:-x,2:+y,3:-y)."""
        i, j = reg.home
        xc, yc = x0 + (i + 0.5) * h, y0 + (j + 0.5) * h
        L = 0.0
        for pc in reg.pieces:
            if pc.kind != 'seg':
                continue
            X0, Y0 = (pc.P0[0] - xc) / h, (pc.P0[1] - yc) / h
            X1, Y1 = (pc.P1[0] - xc) / h, (pc.P1[1] - yc) / h
            if d == 0 and abs(X0 - 0.5) < 1e-12 and abs(X1 - 0.5) < 1e-12:
                L += abs(Y1 - Y0)
            elif d == 1 and abs(X0 + 0.5) < 1e-12 and abs(X1 + 0.5) < 1e-12:
                L += abs(Y1 - Y0)
            elif d == 2 and abs(Y0 - 0.5) < 1e-12 and abs(Y1 - 0.5) < 1e-12:
                L += abs(X1 - X0)
            elif d == 3 and abs(Y0 + 0.5) < 1e-12 and abs(Y1 + 0.5) < 1e-12:
                L += abs(X1 - X0)
        return L

    DIRS = [(1, 0), (-1, 0), (0, 1), (0, -1)]

    # per-cell state: list of regions, volume, moments in own frame
    mom: Dict[int, np.ndarray] = {}
    vol = np.where(status == PURE, 1.0, 0.0)
    loop_mom = {}
    for lin, loops in regions.items():
        ms = [loop_moments(r) for r in loops]
        loop_mom[lin] = ms
        vol[lin // nx, lin % nx] = sum(m[0] for m in ms)
    owner = np.where(status != EMPTY, np.arange(nx * ny).reshape(ny, nx), -1).astype(np.int64)
    members: Dict[int, List[Tuple[Region, np.ndarray]]] = {}
    for lin, loops in regions.items():
        members[lin] = list(zip(loops, loop_mom[lin]))
    absorbed_pure: Dict[int, bool] = {}

    def cell_members(lin):
        if lin in members:
            return members[lin]
        j, i = divmod(lin, nx)
        xc, yc = x0 + (i + 0.5) * h, y0 + (j + 0.5) * h
        # a pure cell as one region: its four edges counter-clockwise
        P = [(xc - h / 2, yc - h / 2), (xc + h / 2, yc - h / 2), (xc + h / 2, yc + h / 2), (xc - h / 2, yc + h / 2)]
        segs = []
        for k in range(4):
            Pa, Pb = P[k], P[(k + 1) % 4]
            on_wall = walls and ((k == 0 and j == 0) or (k == 1 and i == nx - 1) or
                                 (k == 2 and j == ny - 1) or (k == 3 and i == 0))
            segs.append(Piece('seg', P0=Pa, P1=Pb, wall=on_wall))
        members[lin] = [(Region(segs, (i, j)), PURE_MOM.copy())]
        return members[lin]

    def absorb(dst, src_members):
        jd, idd = divmod(dst, nx)
        lst = cell_members(dst)
        for (reg, m) in src_members:
            lst.append((reg, m))
        status[jd, idd] = CUT
        vol[jd, idd] = 0.0
        for (reg, m) in lst:
            # volume is the shift-invariant (0,0) moment
            vol[jd, idd] += m[0]

    # ---- Alg. 1 line 2: multi-component cells keep their largest component
    for lin in sorted(regions):
        loops = members[lin]
        if len(loops) < 2:
            continue
        j, i = divmod(lin, nx)
        order = sorted(range(len(loops)), key=lambda k: (-loops[k][1][0], k))
        keep = order[0]
        kept = [loops[keep]]
        for k in order[1:]:
            reg, m = loops[k]
            best, bkey = None, None
            for d, (di, dj) in enumerate(DIRS):
                if face_len(reg, d) <= 0.0:
                    continue
                ii, jj = i + di, j + dj
                if not (0 <= ii < nx and 0 <= jj < ny) or vol[jj, ii] <= 0.0:
                    continue
                key = (vol[jj, ii], -d)
                if bkey is None or key > bkey:
                    best, bkey = jj * nx + ii, key
            if best is None:
                raise GeometryError("isolated cut-cell component")
            absorb(best, [(reg, m)])
        members[lin] = kept
        vol[j, i] = kept[0][1][0]

    # ---- Alg. 1 lines 3-7: merge small interface cells
    parent: Dict[int, int] = {}
    cand = [lin for lin in regions if vol[lin // nx, lin % nx] <= theta]
    cand.sort(key=lambda lin: (vol[lin // nx, lin % nx], lin))
    for lin in cand:
        j, i = divmod(lin, nx)
        if owner[j, i] != lin or vol[j, i] > theta or vol[j, i] <= 0.0:
            continue
        own = members[lin]
        best, bkey = None, None
        for d, (di, dj) in enumerate(DIRS):
            ii, jj = i + di, j + dj
            if not (0 <= ii < nx and 0 <= jj < ny) or vol[jj, ii] <= 0.0:
                continue
            fl = sum(face_len(reg, d) for (reg, m) in own if reg.home == (i, j))
            key = (fl, vol[jj, ii], -d)
            if bkey is None or key > bkey:
                best, bkey = jj * nx + ii, key
        if best is None or bkey[0] <= 0.0:
            raise GeometryError("small cut cell without a face to merge through")
        absorb(best, own)
        members[lin] = []
        vol[j, i] = 0.0
        status[j, i] = EMPTY
        parent[lin] = best

    # absorbed cells point at their final survivor
    for lin in parent:
        s = parent[lin]
        while s in parent:
            s = parent[s]
        owner[lin // nx, lin % nx] = s

    # ---- final moments (own frame), boundary pieces and boundary moments
    CG = CutGrid(x0, y0, h, nx, ny, status, owner, vol, interface, {}, mom, {})
    CG.arcs_of = arcs_of
    for lin, lst in members.items():
        if not lst:
            continue
        j, i = divmod(lin, nx)
        if status[j, i] == PURE:
            continue      # a pure cell that merely got materialised
        m = np.zeros(15)
        for (reg, mm) in lst:
            hi, hj = reg.home
            m += shift_moments(mm, hi - i, hj - j)
        mom[lin] = m
        CG.regions[lin] = [reg for (reg, _) in lst]
    # boundary pieces: arcs of all constituent regions, wall segments
    for lin in list(CG.regions.keys()) + [int(v) for v in np.nonzero((status == PURE).ravel())[0]]:
        j, i = divmod(lin, nx)
        if status[j, i] == PURE:
            if not walls or not (i == 0 or j == 0 or i == nx - 1 or j == ny - 1):
                continue
            regs = [reg for (reg, _) in cell_members(lin)]
        else:
            regs = CG.regions[lin]
        bp = [pc for reg in regs for pc in reg.pieces if pc.kind == 'arc' or pc.wall]
        if not bp:
            continue
        kinds = set()
        for pc in bp:
            if pc.kind == 'seg':
                kinds.add((prob.box_bc, 1.0, 0.0))
            else:
                cv = curves[pc.curve]
                kinds.add((cv.bc,) + (cv.robin if cv.bc == ROBIN else (1.0, 0.0)))
        if len(kinds) != 1:
            raise GeometryError("a cell mixes boundary-condition types")
        CG.bpieces[lin] = bp
        kind = kinds.pop()
        CG.bc[lin] = kind[0]
        if kind[0] == ROBIN:
            CG.robin[lin] = kind[1:]
        xc, yc = CG.centre(i, j)
        b0, bx, by = np.zeros(15), np.zeros(15), np.zeros(15)
        for pc in bp:
            a0, ax, ay = piece_boundary_moments(pc, curves, xc, yc, h)
            b0 += a0
            bx += ax
            by += ay
        CG.bm0[lin], CG.bmx[lin], CG.bmy[lin] = b0, bx, by
    CG.curves = curves
    return CG
