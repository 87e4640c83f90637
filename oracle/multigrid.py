"""Oracle multigrid: the paper's V-cycle with its smoother and grid transfers.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows Sec. 4: the level hierarchy Omega^(m) with h^(m) = 2^m h, each level
re-embedded and re-discretized; Alg. 2 (VCycle); the smoother SMO-1 (omega-
weighted pointwise Jacobi on the regular unknowns u1) followed by SMO-2 (block
update L22 u2' = r2 - L21 u1'); volume-weighted restriction and patchwise-
constant prolongation on regular cells with zero residual / correction on the
other cells; an LU bottom solve; and Alg. 3, the ordering of the irregular cells
along the boundary, with the cyclic bandwidth of the reordered L22
(eq. L_22_decomposition).

Readings of the paper:
  * SMO-1 is printed as u1' = D^-1[(1-w)D + wO]u1 + w D^-1 O (r1 - L12 u2), which
    applies O to a residual; it is read as the standard weighted Jacobi step
    u1' = D^-1[(1-w)D + wO]u1 + w D^-1 (r1 - L12 u2)
        = u1 + w D^-1 (r1 - (L u)_1),  O = D - L11,
    which is the form the error formula eq. errorOfE1 requires.
  * "Volume weighted restriction ... for regular cells, while leaving the
    correction and the residual for partial cells to zero": after SMO-2 the
    residual of every irregular cell is zero, so the restriction is applied to the
    whole residual field and every non-empty coarse cell receives the
    volume-weighted mean of its children (restricting only into coarse cells that
    are regular on the coarse level starves the coarse grids, which are almost all
    irregular, and the V-cycle then stalls).  The prolongation adds the parent's
    correction to the fine regular cells only; the irregular cells are recomputed
    by the next SMO-2.
  * The coarsest level is the first level with at most 16 cells per side.
  * The relative residual is ||r - L u||_inf / ||r||_inf over non-empty cells.
  * SMO-2 solves with L22 directly (a sparse LU, a library primitive): the paper
    uses a banded LU in the Alg. 3 order, which gives the same solution.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import geometry as G
from . import discretization as D


@dataclass
class Level:
    prob: object
    cg: G.CutGrid
    dz: D.Discretization
    h: float
    nx: int
    ny: int
    ne: np.ndarray          # flat bool, non-empty
    reg: np.ndarray         # flat bool, regular
    irr: np.ndarray         # flat bool, irregular
    diag: float             # D, the diagonal of L11 (physical)
    irr_idx: np.ndarray
    reg_idx: np.ndarray
    L22: Optional[object] = None      # splu of L22
    L21: Optional[sp.csr_matrix] = None
    owner: Optional[np.ndarray] = None


@dataclass
class Hierarchy:
    levels: List[Level]
    bottom_lu: object = None
    bottom_idx: np.ndarray = None


def coarsen(prob, m: int):
    """Problem of level m: same box and curves, h * 2^m."""
    import copy
    p = copy.copy(prob)
    f = 2 ** m
    if prob.nx % f or prob.ny % f:
        raise ValueError("grid not divisible")
    p.nx, p.ny, p.h = prob.nx // f, prob.ny // f, prob.h * f
    return p


def n_levels(prob, coarsest: int = 16) -> int:
    m = 0
    while prob.nx // (2 ** m) > coarsest and (prob.nx // 2 ** (m + 1)) * 2 ** (m + 1) == prob.nx \
            and (prob.ny // 2 ** (m + 1)) * 2 ** (m + 1) == prob.ny:
        m += 1
    return m + 1


def build_hierarchy(prob, theta: float = 0.3, coarsest: int = 16, fine=None) -> Hierarchy:
    nl = n_levels(prob, coarsest)
    levels = []
    for m in range(nl):
        p = coarsen(prob, m)
        if m == 0 and fine is not None:
            cg, dz = fine
        else:
            cg = G.cut_cells(p, theta)
            dz = D.discretize(cg, p.a, p.b, p.c)
        ne = (cg.status != G.EMPTY).ravel()
        reg = dz.regular.ravel()
        irr = dz.irregular.ravel()
        st = D.regular_stencil(p.a, p.b, p.c)
        lv = Level(p, cg, dz, p.h, p.nx, p.ny, ne, reg, irr, st[(0, 0)] / p.h ** 2,
                   np.nonzero(irr)[0], np.nonzero(reg)[0])
        lv.owner = cg.owner.ravel()
        if m < nl - 1:
            L = dz.L
            lv.L22 = spla.splu(L[lv.irr_idx][:, lv.irr_idx].tocsc())
            lv.L21 = L[lv.irr_idx][:, lv.reg_idx].tocsr()
        levels.append(lv)
    H = Hierarchy(levels)
    last = levels[-1]
    idx = np.nonzero(last.ne)[0]
    H.bottom_idx = idx
    H.bottom_lu = sla.lu_factor(last.dz.L[idx][:, idx].toarray())
    return H


# ------------------------------------------------------------------ components

def residual(lv: Level, u: np.ndarray, r: np.ndarray) -> np.ndarray:
    out = np.zeros_like(r)
    out[lv.ne] = (r - lv.dz.L @ u)[lv.ne]
    return out


def smo1(lv: Level, u: np.ndarray, r: np.ndarray, omega: float) -> None:
    """u1 <- u1 + omega D^-1 (r1 - (L u)_1) on the regular cells (SMO-1)."""
    Lu = lv.dz.L @ u
    u[lv.reg] += omega / lv.diag * (r[lv.reg] - Lu[lv.reg])


def smo2(lv: Level, u: np.ndarray, r: np.ndarray) -> None:
    """u2 <- L22^{-1} (r2 - L21 u1) (SMO-2, eq. updateByBlock)."""
    rhs = r[lv.irr_idx] - lv.L21 @ u[lv.reg_idx]
    u[lv.irr_idx] = lv.L22.solve(rhs)


def smooth(lv: Level, u, r, omega, nu):
    for _ in range(nu):
        smo1(lv, u, r, omega)
        smo2(lv, u, r)


def restrict(fine: Level, coarse: Level, res: np.ndarray) -> np.ndarray:
    """Volume-weighted restriction of the residual (Sec. 4.1):
    r^(m+1)_I = sum_children |C_c| r_c / sum_children |C_c| on every non-empty coarse
    cell (for four pure children this is 2^-D times their sum)."""
    R = res.reshape(fine.ny, fine.nx)
    V = fine.cg.vol
    num = V * R
    num = num[0::2, 0::2] + num[1::2, 0::2] + num[0::2, 1::2] + num[1::2, 1::2]
    den = V[0::2, 0::2] + V[1::2, 0::2] + V[0::2, 1::2] + V[1::2, 1::2]
    rc = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
    return np.where(coarse.ne.reshape(coarse.ny, coarse.nx), rc, 0.0).ravel()


def prolong(fine: Level, coarse: Level, uc: np.ndarray) -> np.ndarray:
    """Patchwise-constant interpolation (Sec. 4.1): u^(m)_i = u^(m+1)_{floor(i/2)} on fine
    regular cells (their parent is never empty or merged away), 0 on the other cells."""
    Uc = uc.reshape(coarse.ny, coarse.nx)
    up = np.repeat(np.repeat(Uc, 2, axis=0), 2, axis=1).ravel()
    return np.where(fine.reg, up, 0.0)


def bottom(H: Hierarchy, r: np.ndarray) -> np.ndarray:
    u = np.zeros_like(r)
    u[H.bottom_idx] = sla.lu_solve(H.bottom_lu, r[H.bottom_idx])
    return u


def vcycle(H: Hierarchy, m: int, u: np.ndarray, r: np.ndarray, omega=0.5, nu1=3, nu2=3) -> np.ndarray:
    """Alg. 2."""
    if m == len(H.levels) - 1:
        return bottom(H, r)
    lv, lc = H.levels[m], H.levels[m + 1]
    smooth(lv, u, r, omega, nu1)
    rc = restrict(lv, lc, residual(lv, u, r))
    uc = vcycle(H, m + 1, np.zeros(lc.nx * lc.ny), rc, omega, nu1, nu2)
    u += prolong(lv, lc, uc)
    smooth(lv, u, r, omega, nu2)
    return u


def fmg(H: Hierarchy, r: np.ndarray, omega=0.5, nu1=3, nu2=3) -> np.ndarray:
    """One FMG cycle (Sec. 4, the FMG figure) for L^(0) u = r from a zero guess: the right-hand
    side is restricted down to the bottom level and solved there; then on every finer level
    the coarse solution, prolonged, is the initial guess of one V-cycle (Alg. 2)."""
    M = len(H.levels) - 1
    rs = [r]
    for m in range(M):
        rs.append(restrict(H.levels[m], H.levels[m + 1], rs[m]))
    u = bottom(H, rs[M])
    for m in range(M - 1, -1, -1):
        u = vcycle(H, m, prolong(H.levels[m], H.levels[m + 1], u), rs[m], omega, nu1, nu2)
    return u


def fmg_solve(H: Hierarchy, r: np.ndarray, rtol=1e-10, max_iter=100, omega=0.5, nu1=3, nu2=3,
              history: Optional[list] = None) -> np.ndarray:
    """FMG cycles iterated on the residual equation (the paper's "FMG cycle iterations"):
    u <- u + FMG(r - L u), from u = 0, until the relative residual is <= rtol."""
    lv = H.levels[0]
    u = np.zeros_like(r)
    for it in range(max_iter + 1):
        rr = rel_residual(lv, u, r)
        if history is not None:
            history.append(rr)
        if rr <= rtol or it == max_iter:
            return u
        u = u + fmg(H, residual(lv, u, r), omega, nu1, nu2)
    return u


def rel_residual(lv: Level, u, r) -> float:
    return float(np.abs(residual(lv, u, r)).max() / np.abs(r[lv.ne]).max())


def solve(H: Hierarchy, r: np.ndarray, u0=None, rtol=1e-10, max_iter=100, omega=0.5, nu1=3, nu2=3,
          history: Optional[list] = None) -> np.ndarray:
    """Repeated V-cycles on the finest level until the relative residual is <= rtol."""
    lv = H.levels[0]
    u = np.zeros_like(r) if u0 is None else u0.copy()
    for it in range(max_iter):
        rr = rel_residual(lv, u, r)
        if history is not None:
            history.append(rr)
        if rr <= rtol:
            return u
        u = vcycle(H, 0, u, r, omega, nu1, nu2)
    rr = rel_residual(lv, u, r)
    if history is not None:
        history.append(rr)
    return u


def direct_solve(dz: D.Discretization, r: np.ndarray) -> np.ndarray:
    """u = L^{-1} r over the non-empty cells (sparse direct)."""
    ne = (dz.cg.status != G.EMPTY).ravel()
    idx = np.nonzero(ne)[0]
    u = np.zeros(dz.L.shape[0])
    u[idx] = spla.spsolve(dz.L[idx][:, idx].tocsc(), r[idx])
    return u


# ------------------------------------------------------------------ Alg. 3

def _nearest_param(c: G.OCurve, x, y, ns=20000) -> float:
    t = np.linspace(0.0, 2 * math.pi, ns, endpoint=False)
    px, py = c.xy(t)
    k = int(np.argmin((px - x) ** 2 + (py - y) ** 2))
    return float(t[k])


def alg3_order(lv: Level) -> np.ndarray:
    """P(i) for the irregular cells (flat indices in numbering order), Alg. 3.

    The boundary components are taken one after the other (box first, then the
    curves in input order); within a component the interface cells are sorted by
    the parameter s(i) of the boundary point nearest to the cell centre.  Cells
    that Alg. 3 leaves unnumbered (farther than 2 from every interface cell) are
    numbered right after the interface cell nearest to them."""
    cg = lv.cg
    nx, ny = cg.nx, cg.ny
    keys = []
    for lin in range(nx * ny):
        j, i = divmod(lin, nx)
        xc, yc = cg.centre(i, j)
        if cg.interface[j, i]:
            ci = cg.arcs_of[lin][0][0]
            keys.append(((1 + ci, _nearest_param(cg.curves[ci], xc, yc)), lin))
        elif lin in cg.bpieces and cg.status[j, i] == G.PURE:
            # box wall cell: perimeter coordinate of the nearest wall point
            X0, Y0 = cg.x0, cg.y0
            W, Hh = nx * cg.h, ny * cg.h
            d = [yc - Y0, X0 + W - xc, Y0 + Hh - yc, xc - X0]
            e = int(np.argmin(d))
            s = [xc - X0, W + (yc - Y0), W + Hh + (X0 + W - xc), 2 * W + Hh + (Y0 + Hh - yc)][e]
            keys.append(((0, s), lin))
    keys.sort()
    P = -np.ones(nx * ny, dtype=np.int64)
    order = []
    irr = lv.irr
    # irregular cells farther than 2 from every interface cell (possible only on
    # coarse levels and next to merged cells) ride with their nearest interface cell
    near = {}
    bj = np.array([lin // nx for _, lin in keys])
    bi = np.array([lin % nx for _, lin in keys])
    for q in np.nonzero(irr)[0]:
        j, i = divmod(int(q), nx)
        d = np.maximum(np.abs(bi - i), np.abs(bj - j))
        if d.min() > 2:
            near.setdefault(int(np.argmin(d)), []).append(int(q))
    for k, (_, lin) in enumerate(keys):
        j, i = divmod(lin, nx)
        for dj in range(-2, 3):
            for di in range(-2, 3):
                ii, jj = i + di, j + dj
                if 0 <= ii < nx and 0 <= jj < ny:
                    q = jj * nx + ii
                    if irr[q] and P[q] < 0:
                        P[q] = len(order)
                        order.append(q)
        for q in near.get(k, []):
            if P[q] < 0:
                P[q] = len(order)
                order.append(q)
    return np.array(order, dtype=np.int64)


def cyclic_bandwidth(lv: Level, order: np.ndarray) -> int:
    """max over the nonzeros of the reordered L22 of min(|r - c|, N - |r - c|)."""
    L22 = lv.dz.L[order][:, order].tocoo()
    n = len(order)
    d = np.abs(L22.row - L22.col)
    return int(np.minimum(d, n - d).max())
