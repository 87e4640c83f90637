"""Oracle cubature: cell averages <f>_i and boundary averages <<g>>_i of given functions.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3.2 defines the averages over cut cells and boundary pieces; Sec. 2.4
evaluates area integrals over a cut cell by Green's formula (eq. volumeIntegral)
as the iterated integral of eq. iteratedIntegral:
    int_C f = sum over boundary pieces of int y'(t) int_{xi0}^{x(t)} f(xi, y(t)) dxi dt,
both one-dimensional integrals by Gauss-Legendre quadrature, xi0 the x-centre
of the (survivor) cell.  Pure cells use the 5 x 5 tensor Gauss rule.
"""
from __future__ import annotations

import math
from typing import Callable

import numpy as np

from .geometry import CutGrid, PURE, CUT, EMPTY, DIRICHLET, NEUMANN, GL_ARC, GL_INNER, subintervals

_G5X, _G5W = np.polynomial.legendre.leggauss(5)
_GAX, _GAW = np.polynomial.legendre.leggauss(GL_ARC)
_GIX, _GIW = np.polynomial.legendre.leggauss(GL_INNER)


def _piece_nodes(cg: CutGrid, pc):
    """Outer Gauss nodes along a piece: points, dy/dt * weight, speed * weight, normal."""
    if pc.kind == 'seg':
        s = 0.5 * (_GAX + 1.0)
        x = pc.P0[0] + (pc.P1[0] - pc.P0[0]) * s
        y = pc.P0[1] + (pc.P1[1] - pc.P0[1]) * s
        dyw = (pc.P1[1] - pc.P0[1]) * 0.5 * _GAW
        L = math.hypot(pc.P1[0] - pc.P0[0], pc.P1[1] - pc.P0[1])
        dsw = L * 0.5 * _GAW
        n = ((pc.P1[1] - pc.P0[1]) / L, -(pc.P1[0] - pc.P0[0]) / L)
        return x, y, dyw, dsw, (np.full_like(x, n[0]), np.full_like(x, n[1]))
    c = cg.curves[pc.curve]
    parts = []
    for (a, b) in subintervals(c, pc.t0, pc.t1):      # one Gauss rule per smooth part
        tm, tr = 0.5 * (a + b), 0.5 * (b - a)
        t = tm + tr * _GAX
        x, y = c.xy(t)
        dx, dy = c.dxy(t)
        sp_ = np.hypot(dx, dy)
        sgn = 1.0 if tr > 0 else -1.0
        parts.append((x, y, dy * tr * _GAW, sp_ * abs(tr) * _GAW, sgn * dy / sp_, -sgn * dx / sp_))
    x, y, dyw, dsw, n0, n1 = (np.concatenate([pt[m] for pt in parts]) for m in range(6))
    return x, y, dyw, dsw, (n0, n1)


def region_integral(cg: CutGrid, regions, f: Callable, xi0: float) -> float:
    tot = 0.0
    for reg in regions:
        for pc in reg.pieces:
            x, y, dyw, _, _ = _piece_nodes(cg, pc)
            if not np.any(dyw != 0.0):
                continue
            half = 0.5 * (x - xi0)
            xi = xi0 + half[:, None] * (_GIX[None, :] + 1.0)
            F = np.sum(f(xi, np.broadcast_to(y[:, None], xi.shape)) * _GIW[None, :], axis=1) * half
            tot += float(np.sum(F * dyw))
    return tot


def cell_averages(cg: CutGrid, f: Callable) -> np.ndarray:
    """<f>_i for every non-empty cell (0 elsewhere), array [ny, nx]."""
    h = cg.h
    out = np.zeros((cg.ny, cg.nx))
    pj, pi = np.nonzero(cg.status == PURE)
    xc = cg.x0 + (pi + 0.5) * h
    yc = cg.y0 + (pj + 0.5) * h
    acc = np.zeros(xc.shape)
    for a in range(5):
        for b in range(5):
            acc += _G5W[a] * _G5W[b] * f(xc + 0.5 * h * _G5X[a], yc + 0.5 * h * _G5X[b])
    out[pj, pi] = acc / 4.0
    for lin, regs in cg.regions.items():
        j, i = divmod(lin, cg.nx)
        if cg.status[j, i] != CUT:
            continue
        xc_, _ = cg.centre(i, j)
        out[j, i] = region_integral(cg, regs, f, xc_) / (cg.vol[j, i] * h * h)
    return out


def boundary_averages(cg: CutGrid, segs, u: Callable, ux: Callable, uy: Callable) -> np.ndarray:
    """<<N u>>_i over every boundary segment: u (Dirichlet), grad u . n (Neumann) or
    gamma1 u + gamma2 grad u . n (Robin)."""
    out = np.zeros(len(segs))
    for k, lin in enumerate(segs):
        lin = int(lin)
        tot, length = 0.0, 0.0
        for pc in cg.bpieces[lin]:
            x, y, _, dsw, (nx_, ny_) = _piece_nodes(cg, pc)
            if cg.bc[lin] == DIRICHLET:
                val = u(x, y)
            elif cg.bc[lin] == NEUMANN:
                val = ux(x, y) * nx_ + uy(x, y) * ny_
            else:                      # Robin: gamma1 u + gamma2 du/dn
                g1, g2 = cg.robin[lin]
                val = g1 * u(x, y) + g2 * (ux(x, y) * nx_ + uy(x, y) * ny_)
            tot += float(np.sum(val * dsw))
            length += float(np.sum(dsw))
        out[k] = tot / length
    return out
