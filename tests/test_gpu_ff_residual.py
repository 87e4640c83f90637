"""The outer residual of the mixed solve in float-float arithmetic (pairs of FP32 words, used
for tolerances of 1e-11 and above): the solve must stop only where the residual, evaluated
independently in FP64 (ccm_apply), meets the tolerance, also on the 4096^2 star, and its
solution must equal the oracle's direct solution to the accuracy that tolerance buys."""
import numpy as np
import pytest

import workloads as W
from oracle import cubature as Q
from oracle import discretization as D
from oracle import geometry as G
from oracle import multigrid as MG

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2504_00724_gb300")

pytestmark = pytest.mark.gpu


def fp64_rel_residual(s, f, g, u, ne):
    """||(f - N g) - L u||_inf / ||f - N g||_inf on the non-empty cells, by the FP64 apply."""
    t = (f - s.apply(u, g)).cpu().numpy()
    r = (f - s.apply(torch.zeros_like(u), g)).cpu().numpy()
    return float(np.abs(t[ne]).max() / np.abs(r[ne]).max())


@pytest.mark.parametrize("n,rtol", [(4096, 1e-11), (1024, 1e-11), (1024, 1e-10)])
def test_float_float_residual_is_truthful(n, rtol):
    prob, mms = W.star(n), W.mms_star()
    s = P.Solver(prob, rtol=rtol, max_iter=60, coarsest=64)
    try:
        q = s.quadrature()
        f = torch.tensor(s.cell_averages(mms.f(prob.a, prob.b, prob.c), quad=q), device="cuda")
        g = torch.tensor(s.boundary_averages(mms.u, mms.ux, mms.uy, quad=q), device="cuda")
        ne = s.cell_map()[0] != 0
        u, st = s.solve(f, g)
        assert st.rel_residual <= rtol
        assert fp64_rel_residual(s, f, g, u, ne) <= 1.5 * rtol
    finally:
        s.close()


def test_float_float_solve_matches_direct():
    prob, mms = W.star(288), W.mms_star()
    cg = G.cut_cells(prob)
    dz = D.discretize(cg, prob.a, prob.b, prob.c)
    fa = Q.cell_averages(cg, mms.f(prob.a, prob.b, prob.c))
    ga = Q.boundary_averages(cg, dz.segs, mms.u, mms.ux, mms.uy)
    want = MG.direct_solve(dz, fa.ravel() - dz.N @ ga).reshape(prob.ny, prob.nx)
    s = P.Solver(prob, rtol=1e-11, max_iter=100)
    try:
        u, st = s.solve(torch.tensor(fa, device="cuda"), torch.tensor(ga, device="cuda"))
        assert st.rel_residual <= 1e-11
        got = u.cpu().numpy()
        # a relative residual of 1e-11 leaves an algebraic error of at most cond(L) times that
        assert np.abs(got - want).max() <= 1e-8 * np.abs(want).max()
    finally:
        s.close()
