"""The product's host setup (C++, through the C ABI's host-only view) against the oracle:
identical discrete choices (cells, merges, classification, stencils) and coefficients equal
to rounding, on every level of the hierarchy.  No GPU needed."""
import numpy as np
import pytest

import workloads as W
from oracle import discretization as D
from oracle import geometry as G
from oracle import multigrid as MG

P = pytest.importorskip("paper_2504_00724_gb300")


def _compare_level(hs, level, prob_level):
    cg = G.cut_cells(prob_level)
    dz = D.discretize(cg, prob_level.a, prob_level.b, prob_level.c)
    st, ow, rg, vol, mom = hs.cell_map(level)
    assert np.array_equal(st, cg.status)
    ne = cg.status != 0
    assert np.array_equal(ow[ne], cg.owner[ne])
    assert np.array_equal(rg.astype(bool), dz.regular)
    assert np.abs(vol - cg.vol).max() < 1e-13
    for lin, m in cg.mom.items():
        j, i = divmod(lin, prob_level.nx)
        assert np.abs(mom[j, i] - m).max() < 1e-12
    cell, cols, beta, nb, seg = hs.rows(level)
    lins = sorted(dz.rows.keys())
    assert sorted(cell.tolist()) == lins          # the product numbers rows in boundary order
    where = {int(c): r for r, c in enumerate(cell)}
    segs = {int(s): k for k, s in enumerate(dz.segs)}
    for lin in lins:
        r = where[lin]
        row = dz.rows[lin]
        assert list(cols[r]) == [cj * prob_level.nx + ci for (ci, cj) in row.cells], lin
        scale = np.abs(row.beta).max()
        assert np.abs(beta[r] - row.beta).max() <= 1e-9 * scale
        assert abs(nb[r] - row.beta_b) <= 1e-9 * scale
        assert seg[r] == segs.get(lin, -1)


@pytest.mark.parametrize("mk", [lambda: W.disk_minus(32), lambda: W.star(64),
                                lambda: W.three_ellipses(64), lambda: W.paper_problem2(32, W.NEUMANN),
                                lambda: W.star(32, (1.25, -0.8660254037844386, 1.75)),
                                lambda: W.paper_problem1(40), lambda: W.disk_robin(32),
                                lambda: W.disk_robin(32, (2.0, -0.3), abc=(1.0, 0.5, 2.0)),
                                lambda: W.paper_problem3_rotated(32), lambda: W.spline_blob(64)])
def test_finest_level_matches_oracle(mk):
    prob = mk()
    hs = P.HostSetup(prob)
    _compare_level(hs, 0, prob)


@pytest.mark.slow
def test_every_level_matches_oracle():
    prob = W.star(128)
    hs = P.HostSetup(prob)
    nl = MG.n_levels(prob)
    for m in range(nl):
        _compare_level(hs, m, MG.coarsen(prob, m))


def test_polygon_every_level_matches_oracle():
    """The rotated box of Problem 3, case (ii): a polygon curve whose corners fall inside cut
    cells, (a, b, c) = (5/4, -sqrt(3)/2, 7/4), on every level."""
    prob = W.paper_problem3_rotated(64)
    hs = P.HostSetup(prob)
    for m in range(MG.n_levels(prob)):
        _compare_level(hs, m, MG.coarsen(prob, m))


def test_spline_every_level_matches_oracle():
    """A cubic-spline boundary (knots at chord lengths, integrals split at the knots)."""
    prob = W.spline_blob(64, seed=3)
    hs = P.HostSetup(prob)
    for m in range(MG.n_levels(prob)):
        _compare_level(hs, m, MG.coarsen(prob, m))


def test_robin_every_level_matches_oracle():
    """The Robin column (scaled by |gamma1| + |gamma2| / h of the level) on every level."""
    prob = W.disk_robin(64, (1.0, 0.5))
    hs = P.HostSetup(prob)
    for m in range(MG.n_levels(prob)):
        _compare_level(hs, m, MG.coarsen(prob, m))


def test_invalid_problems_are_rejected():
    prob = W.star(64)
    bad = W.Problem(1.0, 3.0, 1.0, 0.0, 0.0, 1 / 64, 64, 64, W.NONE, prob.curves)   # b^2 - 4ac > 0
    with pytest.raises(P.CcmError) as e:
        P.HostSetup(bad)
    assert e.value.code == -1
    off = W.Problem(1.0, 0.0, 1.0, 0.0, 0.0, 1 / 64, 64, 64, W.NONE,
                    [W.Curve(W.CIRCLE, (0.95, 0.5, 0.2), +1, W.DIRICHLET)])            # leaves the box
    with pytest.raises(P.CcmError) as e:
        P.HostSetup(off)
    assert e.value.code == -2
    clockwise = (0.2, 0.8, 0.8, 0.8, 0.8, 0.2, 0.2, 0.2)
    for verts in (clockwise, clockwise[:4]):           # clockwise; two vertices only
        bad = W.Problem(1.0, 0.0, 1.0, 0.0, 0.0, 1 / 32, 32, 32, W.NONE, [W.Curve(W.POLYGON, verts, +1, W.DIRICHLET)])
        with pytest.raises(P.CcmError) as e:
            P.HostSetup(bad)
        assert e.value.code == -1
    for gamma in ((0.0, 0.0), (float("nan"), 1.0)):                                 # no Robin operator
        with pytest.raises(P.CcmError) as e:
            P.HostSetup(W.disk_robin(32, gamma))
        assert e.value.code == -1
