"""Pins of the oracle's geometry (cut cells, Green-formula moments, Alg. 1 merging)
against closed forms and library quadrature (Sec. 2.4, Sec. 3.1)."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import workloads as W
from oracle import geometry as G


def global_moment(cg, p, q, xg=0.0, yg=0.0):
    """int_Omega (x - xg)^p (y - yg)^q dA assembled from the per-cell moments."""
    h = cg.h
    tot = 0.0
    pure = np.argwhere(cg.status == G.PURE)
    k = G.EIDX[(p, q)]
    for (j, i) in pure:
        if j * cg.nx + i in cg.mom:
            continue
        xc, yc = cg.centre(i, j)
        m = G.shift_moments(G.PURE_MOM, (xc - xg) / h, (yc - yg) / h)
        tot += m[k]
    for lin, m0 in cg.mom.items():
        j, i = divmod(lin, cg.nx)
        xc, yc = cg.centre(i, j)
        tot += G.shift_moments(m0, (xc - xg) / h, (yc - yg) / h)[k]
    return tot * h ** (2 + p + q)


@pytest.mark.parametrize("n", [16, 64])
def test_disk_hole_area_and_second_moment(n):
    r = 0.2
    cg = G.cut_cells(W.disk_minus(n, r))
    assert abs(cg.vol.sum() * cg.h ** 2 - (1 - math.pi * r * r)) < 1e-13
    # int (x - 1/2)^2 over box minus disk = 1/12 - pi r^4 / 4
    assert abs(global_moment(cg, 2, 0, 0.5, 0.5) - (1 / 12 - math.pi * r ** 4 / 4)) < 1e-13
    assert abs(global_moment(cg, 1, 1, 0.5, 0.5)) < 1e-14
    assert abs(global_moment(cg, 1, 0, 0.0, 0.0) - 0.5 * (1 - math.pi * r * r)) < 1e-13


def test_star_area_and_polar_moment():
    r0, amp, k = 0.3, 0.08, 5
    cg = G.cut_cells(W.star(64, r0=r0, amp=amp, k=k))
    area = math.pi * (r0 ** 2 + amp ** 2 / 2)
    assert abs(cg.vol.sum() * cg.h ** 2 - area) < 1e-13
    # int r^2 dA = (1/4) int r(t)^4 dt = (pi/2)(r0^4 + 3 r0^2 amp^2 + 3 amp^4 / 8)
    J = global_moment(cg, 2, 0, 0.5, 0.5) + global_moment(cg, 0, 2, 0.5, 0.5)
    assert abs(J - 0.5 * math.pi * (r0 ** 4 + 3 * r0 ** 2 * amp ** 2 + 3 * amp ** 4 / 8)) < 1e-13


def test_rotated_ellipse_moments():
    prob = W.three_ellipses(64)
    cg = G.cut_cells(prob)
    area = 1 - sum(math.pi * c.params[2] * c.params[3] for c in prob.curves)
    assert abs(cg.vol.sum() * cg.h ** 2 - area) < 1e-13
    # second moment about the box centre: box part minus each ellipse's (parallel axes)
    want = 1 / 12
    for c in prob.curves:
        cx, cy, a, b, phi = c.params
        A = math.pi * a * b
        Ixx = A * (a * a * math.cos(phi) ** 2 + b * b * math.sin(phi) ** 2) / 4
        want -= Ixx + A * (cx - 0.5) ** 2
    assert abs(global_moment(cg, 2, 0, 0.5, 0.5) - want) < 1e-13


def test_boundary_length_and_divergence_identities():
    """Sum of boundary-piece lengths = perimeter (scipy quad of |gamma'|); the outward
    normals satisfy int n ds = 0 and int x n_x ds = |Omega| (divergence theorem)."""
    r0, amp, k = 0.3, 0.08, 5
    cg = G.cut_cells(W.star(128, r0=r0, amp=amp, k=k))
    h = cg.h
    per = quad(lambda t: math.hypot(-amp * k * math.sin(k * t), r0 + amp * math.cos(k * t)),
               0, 2 * math.pi, limit=200, epsabs=1e-14)[0]
    L = sum(b[0] for b in cg.bm0.values()) * h
    assert abs(L - per) < 1e-12
    nx_ = sum(b[0] for b in cg.bmx.values()) * h
    ny_ = sum(b[0] for b in cg.bmy.values()) * h
    assert abs(nx_) < 1e-13 and abs(ny_) < 1e-13
    # int x n_x ds over the star boundary = area (x about any origin)
    xn = 0.0
    for lin, bx in cg.bmx.items():
        j, i = divmod(lin, cg.nx)
        xc, _ = cg.centre(i, j)
        xn += (bx[G.EIDX[(1, 0)]] * h + (xc - 0.5) * bx[0]) * h
    assert abs(xn - math.pi * (r0 ** 2 + amp ** 2 / 2)) < 1e-13


def test_box_walls_are_boundary_pieces():
    cg = G.cut_cells(W.disk_minus(32))
    h = cg.h
    walls = [lin for lin in cg.bpieces if cg.status.ravel()[lin] == G.PURE]
    assert len(walls) == 4 * 32 - 4
    L = sum(cg.bm0[lin][0] for lin in walls) * h
    assert abs(L - 4.0) < 1e-14
    # left wall cell: outward normal (-1, 0)
    lin = 10 * 32 + 0
    assert abs(cg.bmx[lin][0] + 1.0) < 1e-14 and abs(cg.bmy[lin][0]) < 1e-14


def test_shift_matches_direct_integration():
    """Binomial shift of square moments equals the closed-form moments of a shifted square."""
    dx, dy = 1.5, -2.0
    got = G.shift_moments(G.PURE_MOM, dx, dy)
    for k, (p, q) in enumerate(G.EXPS):
        ix = ((dx + 0.5) ** (p + 1) - (dx - 0.5) ** (p + 1)) / (p + 1)
        iy = ((dy + 0.5) ** (q + 1) - (dy - 0.5) ** (q + 1)) / (q + 1)
        assert abs(got[k] - ix * iy) < 1e-12 * max(1.0, abs(ix * iy))


@pytest.mark.parametrize("theta", [0.3, 0.5])
def test_merging_postcondition(theta):
    """Alg. 1 postcondition: volumes add up and every surviving interface cell exceeds theta h^2."""
    prob = W.star(64)
    cg0 = G.cut_cells(prob, theta=0.0)
    cg = G.cut_cells(prob, theta=theta)
    assert abs(cg.vol.sum() - cg0.vol.sum()) < 1e-11
    surv = cg.interface & (cg.status != G.EMPTY)
    assert np.all(cg.vol[surv] > theta)
    absorbed = cg.interface & (cg.status == G.EMPTY) & (cg0.vol > 0)
    assert absorbed.sum() > 0
    for (j, i) in np.argwhere(absorbed):
        o = cg.owner[j, i]
        oj, oi = divmod(int(o), cg.nx)
        assert cg.status[oj, oi] != G.EMPTY


def test_vertex_and_tangent_degeneracies():
    """The paper's Problem 2 ellipse passes through grid vertices and touches grid lines."""
    for n in (32, 64):
        cg = G.cut_cells(W.paper_problem2(n))
        assert abs(cg.vol.sum() * cg.h ** 2 - (1 - math.pi / 32)) < 1e-13


def _polygon_moment(V, p, q):
    """int over the polygon of x^p y^q by Green's formula edge by edge, int x^{p+1}/(p+1) y^q dy,
    with a Gauss rule exact for the edge polynomial (independent of the cut cells)."""
    z, w = np.polynomial.legendre.leggauss(8)
    s = 0.5 * (z + 1.0)
    tot = 0.0
    n = len(V)
    for k in range(n):
        (xa, ya), (xb, yb) = V[k], V[(k + 1) % n]
        x = xa + (xb - xa) * s
        y = ya + (yb - ya) * s
        tot += np.sum(x ** (p + 1) / (p + 1) * y ** q * (yb - ya) * 0.5 * w)
    return tot


@pytest.mark.parametrize("n", [16, 64])
def test_rotated_box_polygon_moments(n):
    """The box rotated by pi/6 (Problem 3, case (ii)): area 1, centroid (1/2, 1/2), and the
    central moments of a unit square rotated by theta: int x^2 = 1/12, int x y = 0, int x^4 =
    (c^4 + s^4)/80 + 6 c^2 s^2/144.  Every corner lies inside a cut cell, so this fails unless
    the integrals along a piece are split at the corners."""
    cg = G.cut_cells(W.paper_problem3_rotated(n))
    c, s = math.cos(math.pi / 6), math.sin(math.pi / 6)
    assert abs(cg.vol.sum() * cg.h ** 2 - 1.0) < 1e-13
    assert abs(global_moment(cg, 1, 0) - 0.5) < 1e-13 and abs(global_moment(cg, 0, 1) - 0.5) < 1e-13
    assert abs(global_moment(cg, 2, 0, 0.5, 0.5) - 1 / 12) < 1e-14
    assert abs(global_moment(cg, 1, 1, 0.5, 0.5)) < 1e-14
    want4 = (c ** 4 + s ** 4) / 80 + 6 * c * c * s * s / 144
    assert abs(global_moment(cg, 4, 0, 0.5, 0.5) - want4) < 1e-14


@pytest.mark.parametrize("n", [16, 64])
def test_nonconvex_polygon_moments(n):
    """A pentagon with a reflex corner (even-odd inside test, a non-convex cut cell): every
    moment up to degree 4 equals the polygon's own Green integral."""
    V = [(0.2, 0.2), (0.8, 0.2), (0.8, 0.8), (0.53, 0.45), (0.2, 0.8)]
    prob = W.Problem(1.0, 0.0, 1.0, 0.0, 0.0, 1.0 / n, n, n, W.NONE,
                     [W.Curve(W.POLYGON, tuple(v for xy in V for v in xy), +1, W.DIRICHLET)])
    cg = G.cut_cells(prob)
    for (p, q) in G.EXPS:
        assert abs(global_moment(cg, p, q) - _polygon_moment(V, p, q)) < 1e-13, (p, q)
    ins = G.OCurve(W.POLYGON, prob.curves[0].params, 1, W.DIRICHLET).inside
    assert ins(0.5, 0.3) and not ins(0.53, 0.6) and ins(0.25, 0.7) and not ins(0.3, 0.7) and not ins(0.9, 0.5)


def test_polygon_subintervals():
    c = G.OCurve(W.POLYGON, (0, 0, 1, 0, 1, 1, 0, 1), 1, W.DIRICHLET)
    q = math.pi / 2
    assert G.subintervals(c, 0.1, 0.2) == [(0.1, 0.2)]
    assert G.subintervals(c, 1.0, 2.0) == [(1.0, q), (q, 2.0)]
    assert G.subintervals(c, 2.0, 1.0) == [(2.0, q), (q, 1.0)]                  # reversed traversal
    parts = G.subintervals(c, 6.0, 6.6)                                          # across t = 2 pi
    assert len(parts) == 2 and abs(parts[0][1] - 2 * math.pi) < 1e-15
    x, y = c.xy(np.array([0.0, q / 2, q, 3 * q + q / 2]))
    assert np.allclose(x, [0, 0.5, 1, 0]) and np.allclose(y, [0, 0, 0, 0.5])
    with pytest.raises(G.GeometryError):
        G.OCurve(W.POLYGON, (0, 0, 0, 1, 1, 1, 1, 0), 1, W.DIRICHLET)          # clockwise


def _scipy_spline(c):
    from scipy.interpolate import CubicSpline
    P = np.vstack([c.V, c.V[:1]])
    return (CubicSpline(c.knots, P[:, 0], bc_type="periodic"), CubicSpline(c.knots, P[:, 1], bc_type="periodic"))


def test_spline_is_the_periodic_cubic_spline():
    """The oracle's Y_c curve equals scipy's periodic cubic spline on the same knots (values and
    derivatives), interpolates its points and has chord-length knots."""
    prob = W.spline_blob(64)
    c = G.OCurve(W.SPLINE, prob.curves[0].params, 1, W.DIRICHLET)
    sx, sy = _scipy_spline(c)
    t = np.linspace(0.0, 2 * math.pi, 2001)
    x, y = c.xy(t)
    dx, dy = c.dxy(t)
    assert np.abs(x - sx(t)).max() < 1e-14 and np.abs(y - sy(t)).max() < 1e-14
    assert np.abs(dx - sx(t, 1)).max() < 1e-13 and np.abs(dy - sy(t, 1)).max() < 1e-13
    xk, yk = c.xy(c.knots[:-1])
    assert np.abs(xk - c.V[:, 0]).max() < 1e-15 and np.abs(yk - c.V[:, 1]).max() < 1e-15
    ch = np.hypot(*(np.roll(c.V, -1, axis=0) - c.V).T)
    assert np.allclose(np.diff(c.knots), 2 * math.pi * ch / ch.sum(), rtol=1e-14)


@pytest.mark.parametrize("n", [16, 64])
def test_spline_domain_moments(n):
    """Every moment up to degree 4 of a spline domain, assembled from the cut cells, equals
    Green's integral of x^{p+1}/(p+1) y^q dy along scipy's spline, one adaptive quadrature per
    cubic.  A Gauss rule spanning a knot (where the third derivative jumps) misses this at the
    1e-13 level."""
    prob = W.spline_blob(n)
    cg = G.cut_cells(prob)
    c = G.OCurve(W.SPLINE, prob.curves[0].params, 1, W.DIRICHLET)
    sx, sy = _scipy_spline(c)
    for (p, q) in G.EXPS:
        want = sum(quad(lambda t: sx(t) ** (p + 1) / (p + 1) * sy(t) ** q * sy(t, 1), c.knots[k], c.knots[k + 1],
                        epsabs=1e-15, epsrel=1e-13, limit=200)[0] for k in range(len(c.V)))
        assert abs(global_moment(cg, p, q) - want) < 1e-13, (p, q)
