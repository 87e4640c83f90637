"""Input averages computed by the library (ccm_cell_averages, ccm_boundary_averages) with
the caller's functions: equal to the oracle's own cubature of the same functions on every
cell and segment, and exact for a polynomial on pure cells."""
import numpy as np
import pytest

import workloads as W
from oracle import cubature as Q
from oracle import discretization as D
from oracle import geometry as G

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2504_00724_gb300")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mk,mms", [(lambda: W.star(96), W.mms_star()), (lambda: W.three_ellipses(64), W.mms_ellipses()),
                                    (lambda: W.paper_problem1(40), W.mms_problem1())])
def test_averages_match_oracle(mk, mms):
    prob = mk()
    cg = G.cut_cells(prob)
    dz = D.discretize(cg, prob.a, prob.b, prob.c)
    fw = Q.cell_averages(cg, mms.f(prob.a, prob.b, prob.c))
    gw = Q.boundary_averages(cg, dz.segs, mms.u, mms.ux, mms.uy)
    s = P.Solver(prob)
    try:
        fg = s.cell_averages(mms.f(prob.a, prob.b, prob.c))
        gg = s.boundary_averages(mms.u, mms.ux, mms.uy)
        assert np.abs(fg - fw).max() <= 1e-12 * np.abs(fw).max()
        assert np.abs(gg - gw).max() <= 1e-12 * np.abs(gw).max()
    finally:
        s.close()


def test_pure_cell_rule_exact_on_polynomial():
    prob = W.star(64)
    s = P.Solver(prob)
    try:
        st = s.cell_map()[0]
        got = s.cell_averages(lambda x, y: x ** 4 * y ** 3)
        h = prob.h
        j, i = np.nonzero(st == 1)
        x0, y0 = prob.x0 + i * h, prob.y0 + j * h
        want = ((x0 + h) ** 5 - x0 ** 5) / 5 * ((y0 + h) ** 4 - y0 ** 4) / 4 / (h * h)
        assert np.abs(got[j, i] - want).max() <= 1e-14
        assert np.all(got[st == 0] == 0.0)
    finally:
        s.close()


def test_callback_errors_propagate():
    s = P.Solver(W.star(64))
    try:
        with pytest.raises(ZeroDivisionError):
            s.cell_averages(lambda x, y: 1 / 0)
    finally:
        s.close()
