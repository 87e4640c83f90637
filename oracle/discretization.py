"""Oracle discretization: regular stencils, PLG stencils, fitted rows, assembly.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows Sec. 3.2 (eq. stdGrad, eq. stdLap, stencils S_Lap and S_Cro, regular
cells), Sec. 3.3 (PLG stencil X(i) = S_PLG(i) u {S_i}, sample matrix
eq. detailedSampleMatrix, weighted minimum-norm coefficients eq. derivedCoefAgain
with weights eq. weightDef, recentred and scaled monomial basis), Sec. 3.4
(L u + N g = f, eq. PoissonLinearDiscretization) and Sec. 2.2 (poisedness).

Readings of the paper:
  * eq. stdLap prints +<phi>_{i-2e}; the weights (-1, 16, -30, 16, -1) must sum to
    zero, so the last sign is read as minus (pinned by polynomial exactness).
  * The cross derivative is stdGrad in x1 applied after stdGrad in x2.
  * The PLG algorithm itself lives in a paper that is not available.  The stencil
    is chosen by a deterministic, exact rule built from transformed principal
    lattices (see plg_stencil): 5 parallel grid lines with 5, 4, 3, 2, 1 cells,
    least integer cost within the Chebyshev ball of radius 3, 4 or 5.  Every
    decision is on integers, so two independent codes pick the same cells.
  * The fit is done in the scaled frame ((x - p)/h) with derivatives taken in that
    frame too (so the weights of eq. weightDef are dimensionless for Neumann rows);
    physical coefficients follow by dividing by h^2 (cells, Dirichlet) or h (Neumann).
  * p is the centre of the bounding box of the stencil's Cartesian cells.
  * With no boundary piece the system is square and beta = M^{-1} L.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass
from typing import Dict, List, Optional, Tuple

import numpy as np
import scipy.sparse as sp

from .geometry import (CutGrid, EXPS, EIDX, PURE, CUT, EMPTY, DIRICHLET, NEUMANN,
                       shift_moments)

RADII = (3, 4, 5)
PERMS = list(itertools.permutations([1, 2, 3, 4, 5]))     # lexicographic order
PERM_ARR = np.array(PERMS)
NCAND = 12


class PLGError(Exception):
    pass


# ------------------------------------------------------------------ regular stencil

def regular_stencil(a: float, b: float, c: float) -> Dict[Tuple[int, int], float]:
    """h^2-scaled weights of a u_xx + b u_xy + c u_yy on cell averages (eq. stdLap, stdGrad)."""
    lap = {-2: -1.0, -1: 16.0, 0: -30.0, 1: 16.0, 2: -1.0}
    grad = {-2: 1.0, -1: -8.0, 1: 8.0, 2: -1.0}
    w: Dict[Tuple[int, int], float] = {}
    for m, v in lap.items():
        w[(m, 0)] = w.get((m, 0), 0.0) + a * v / 12.0
        w[(0, m)] = w.get((0, m), 0.0) + c * v / 12.0
    if b != 0.0:
        for m1, g1 in grad.items():
            for m2, g2 in grad.items():
                w[(m1, m2)] = w.get((m1, m2), 0.0) + b * g1 * g2 / 144.0
    return w


def regular_mask(cg: CutGrid) -> np.ndarray:
    """Regular cells: every cell of S_Lap(i) u S_Cro(i) (the 5x5 box) is pure."""
    pure = cg.status == PURE
    ny, nx = pure.shape
    P = np.zeros((ny + 4, nx + 4), dtype=bool)
    P[2:-2, 2:-2] = pure
    reg = np.ones((ny, nx), dtype=bool)
    for dj in range(-2, 3):
        for di in range(-2, 3):
            reg &= P[2 + dj:2 + dj + ny, 2 + di:2 + di + nx]
    return reg


# ------------------------------------------------------------------ FV sample values

def cell_avg_monomials(cg: CutGrid, i: int, j: int, px: float, py: float) -> np.ndarray:
    """<((x - p)/h)^alpha> over cell (i, j) for the 15 graded monomials."""
    lin = j * cg.nx + i
    xc, yc = cg.centre(i, j)
    m = shift_moments(cg.moments(lin), (xc - px) / cg.h, (yc - py) / cg.h)
    return m / cg.vol[j, i]


def _sample_matrix(cg: CutGrid, cells, px, py) -> np.ndarray:
    """M[alpha, k] = <phi_alpha>_{cell k}."""
    return np.stack([cell_avg_monomials(cg, i, j, px, py) for (i, j) in cells], axis=1)


def _bbox_centre(cg: CutGrid, cells):
    imin = min(c[0] for c in cells)
    imax = max(c[0] for c in cells)
    jmin = min(c[1] for c in cells)
    jmax = max(c[1] for c in cells)
    return (cg.x0 + 0.5 * (imin + imax + 1) * cg.h, cg.y0 + 0.5 * (jmin + jmax + 1) * cg.h)


def plg_candidates(cg: CutGrid, i: int, j: int, kmax: int) -> List[List[Tuple[int, int]]]:
    """Up to kmax poised 15-cell lattices around irregular cell (i, j), best first.

    A candidate is a lattice on 5 distinct parallel grid lines (rows or columns)
    carrying 5, 4, 3, 2 and 1 non-empty cells: such a lattice is poised for Pi_4
    (restricted to the line with 5 nodes an interpolant of zero data vanishes, so it
    is divisible by that line's linear form; repeat with degree 3 on the line with
    4 nodes, and so on), which makes it a transformed principal lattice.  The line
    offsets form a 5-subset of [-R, R] containing 0; on each line the cells closest
    to i are used (order (du^2, du)).  Candidates are ranked by the integer cost
    sum |j_k - i|^2, then rows before columns, then the lexicographic order of the
    5-subset, then the lexicographic order of the assignment of the counts 1..5 to
    the sorted lines.  R is 3; 4 and 5 are used only if no candidate exists.
    """
    nonempty = cg.status != EMPTY
    for R in RADII:
        keys, meta = [], []
        for o in (0, 1):
            lines = {}
            for dv in range(-R, R + 1):
                av = []
                for du in range(-R, R + 1):
                    ii, jj = (i + du, j + dv) if o == 0 else (i + dv, j + du)
                    if 0 <= ii < cg.nx and 0 <= jj < cg.ny and nonempty[jj, ii]:
                        av.append(du)
                av.sort(key=lambda d: (d * d, d))
                lines[dv] = av
            tab = np.full((2 * R + 1, 5), np.inf)
            for dv, av in lines.items():
                for m in range(1, min(5, len(av)) + 1):
                    tab[dv + R, m - 1] = sum(d * d for d in av[:m]) + m * dv * dv
            others = [dv for dv in range(-R, R + 1) if dv != 0]
            subs = [sorted(sub + (0,)) for sub in itertools.combinations(others, 4)]
            rows_ = np.array(subs) + R                                   # [nsub, 5]
            costs = tab[rows_[:, None, :], PERM_ARR[None, :, :] - 1].sum(axis=2)   # [nsub, 120]
            si, pk = np.nonzero(np.isfinite(costs))
            keys.append(np.stack([costs[si, pk], np.full(si.shape, o), si, pk], axis=1))
            meta.append((subs, lines))
        K = np.concatenate(keys, axis=0)
        if len(K):
            order = np.lexsort((K[:, 3], K[:, 2], K[:, 1], K[:, 0]))[:kmax]
            out = []
            for r in order:
                cost, o, si, pk = K[r]
                o, si, pk = int(o), int(si), int(pk)
                subs, lines = meta[o]
                cells = []
                for dv, m in zip(subs[si], PERMS[pk]):
                    for du in lines[dv][:m]:
                        cells.append((i + du, j + dv) if o == 0 else (i + dv, j + du))
                cells.sort(key=lambda c: (c != (i, j), c[1] - j, c[0] - i))
                out.append(cells)
            return out
    raise PLGError(f"no poised stencil for cell ({i},{j})")


# ------------------------------------------------------------------ fitted rows

@dataclass
class Row:
    cells: List[Tuple[int, int]]
    beta: np.ndarray        # physical coefficients of the stencil cells
    beta_b: float           # physical coefficient of the boundary datum (0 if none)
    cond: float


def _fit(cg: CutGrid, i: int, j: int, cells, a: float, b: float, c: float):
    """beta = W M^T (M W M^T)^{-1} L for one stencil; returns (scaled beta, ||beta||_{W^-1}^2, cond)."""
    px, py = _bbox_centre(cg, cells)
    M = _sample_matrix(cg, cells, px, py)
    M15 = M
    lin = j * cg.nx + i
    h = cg.h
    xc, yc = cg.centre(i, j)
    dx, dy = (xc - px) / h, (yc - py) / h
    mi = shift_moments(cg.moments(lin), dx, dy) / cg.vol[j, i]
    Lhat = np.zeros(15)
    for k, (p, q) in enumerate(EXPS):
        v = 0.0
        if p >= 2:
            v += a * p * (p - 1) * mi[EIDX[(p - 2, q)]]
        if p >= 1 and q >= 1:
            v += b * p * q * mi[EIDX[(p - 1, q - 1)]]
        if q >= 2:
            v += c * q * (q - 1) * mi[EIDX[(p, q - 2)]]
        Lhat[k] = v
    w = [max(math.hypot(ci - i, cj - j), 0.5) for (ci, cj) in cells]
    if lin in cg.bpieces:
        S = cg.bm0[lin][0]
        col_d = shift_moments(cg.bm0[lin], dx, dy) / S
        gx = shift_moments(cg.bmx[lin], dx, dy)
        gy = shift_moments(cg.bmy[lin], dx, dy)
        col_n = np.zeros(15)
        for k, (p, q) in enumerate(EXPS):
            v = 0.0
            if p >= 1:
                v += p * gx[EIDX[(p - 1, q)]]
            if q >= 1:
                v += q * gy[EIDX[(p, q - 1)]]
            col_n[k] = v / S
        if cg.bc[lin] == DIRICHLET:
            col = col_d
        elif cg.bc[lin] == NEUMANN:
            col = col_n
        else:
            # Robin, N = gamma1 + gamma2 d/dn (Sec. 3.3): <N phi> in the scaled frame is
            # gamma1 <phi> + (gamma2 / h) <d phi / dn_s>, normalised by |gamma1| + |gamma2| / h
            # so that gamma2 = 0 gives the Dirichlet column and gamma1 = 0 the Neumann one
            g1, g2 = cg.robin[lin]
            col = (g1 * col_d + (g2 / cg.h) * col_n) / _robin_norm(g1, g2, cg.h)
        M = np.concatenate([M, col[:, None]], axis=1)
        w.append(0.5)
    w = np.array(w)
    Wd = 1.0 / w
    MW = M * Wd[None, :]
    beta_s = Wd * (M.T @ np.linalg.solve(MW @ M.T, Lhat))
    return beta_s, float(np.sum(w * beta_s * beta_s)), M15


def _robin_norm(g1: float, g2: float, h: float) -> float:
    """Scale of the Robin boundary column, |gamma1| + |gamma2| / h (see _fit)."""
    return abs(g1) + abs(g2) / h


def fit_row(cg: CutGrid, i: int, j: int, a: float, b: float, c: float) -> Row:
    """Fitted row of irregular cell (i, j) (eq. derivedCoefAgain, weights eq. weightDef).

    Among the first NCAND PLG candidates the stencil whose coefficients have the
    least weighted norm ||beta||_{W^-1} (the objective the fit itself minimises)
    is used; a candidate replaces the best so far only if its norm is smaller by a
    relative 1e-9, so near-ties fall to the earlier candidate."""
    best = None
    for cells in plg_candidates(cg, i, j, NCAND):
        beta_s, nrm, M15 = _fit(cg, i, j, cells, a, b, c)
        if best is None or nrm < best[1] * (1.0 - 1e-9):
            best = (cells, nrm, beta_s, M15)
    cells, nrm, beta_s, M15 = best
    cond = float(np.linalg.cond(M15, 2))
    lin = j * cg.nx + i
    h = cg.h
    beta = beta_s[:15] / h ** 2
    beta_b = 0.0
    if lin in cg.bpieces:
        if cg.bc[lin] == DIRICHLET:
            beta_b = beta_s[15] / h ** 2
        elif cg.bc[lin] == NEUMANN:
            beta_b = beta_s[15] / h
        else:
            g1, g2 = cg.robin[lin]
            beta_b = beta_s[15] / (_robin_norm(g1, g2, h) * h ** 2)
    return Row(cells, beta, beta_b, cond)


# ------------------------------------------------------------------ assembly

@dataclass
class Discretization:
    cg: CutGrid
    a: float
    b: float
    c: float
    L: sp.csr_matrix         # [nx*ny, nx*ny] physical units, empty rows/cols for empty cells
    N: sp.csr_matrix         # [nx*ny, nseg]
    regular: np.ndarray      # [ny, nx] bool
    irregular: np.ndarray    # [ny, nx] bool
    segs: np.ndarray         # linear indices of the cells owning boundary segments
    rows: Dict[int, Row]


def discretize(cg: CutGrid, a: float, b: float, c: float) -> Discretization:
    """Assemble L and N of L u + N g = f (eq. PoissonLinearDiscretization)."""
    if b * b - 4 * a * c >= 0:
        raise ValueError("the operator is not elliptic (b^2 - 4ac >= 0)")
    nx, ny, h = cg.nx, cg.ny, cg.h
    nonempty = cg.status != EMPTY
    reg = regular_mask(cg) & nonempty
    irr = nonempty & ~reg
    segs = np.array(sorted(cg.bpieces.keys()), dtype=np.int64)
    seg_of = {int(s): k for k, s in enumerate(segs)}
    R, C, V = [], [], []
    # regular rows (vectorised)
    st = regular_stencil(a, b, c)
    rj, ri = np.nonzero(reg)
    rl = rj * nx + ri
    for (di, dj), wv in st.items():
        R.append(rl)
        C.append((rj + dj) * nx + (ri + di))
        V.append(np.full(rl.shape, wv / h ** 2))
    # irregular rows
    rows: Dict[int, Row] = {}
    NR, NC, NV = [], [], []
    jj, ii = np.nonzero(irr)
    for (j, i) in zip(jj.tolist(), ii.tolist()):
        row = fit_row(cg, i, j, a, b, c)
        lin = j * nx + i
        rows[lin] = row
        R.append(np.full(15, lin))
        C.append(np.array([cj * nx + ci for (ci, cj) in row.cells]))
        V.append(row.beta)
        if lin in seg_of:
            NR.append(lin)
            NC.append(seg_of[lin])
            NV.append(row.beta_b)
    n = nx * ny
    L = sp.csr_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))), shape=(n, n))
    N = sp.csr_matrix((np.array(NV), (np.array(NR, dtype=np.int64), np.array(NC, dtype=np.int64))),
                      shape=(n, len(segs)))
    return Discretization(cg, a, b, c, L, N, reg, irr, segs, rows)
