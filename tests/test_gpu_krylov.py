"""GMRES(m) correction of the mixed outer iteration (ccm_params.krylov): the inner FP32
V-cycles as right preconditioner, the FP64 residual around it.  On the three-ellipse domain
with Neumann data on the ellipses, where the V-cycle's iteration operator has eigenvalues
outside the unit disk from 512^2 cells on, the solution must equal the oracle's sparse direct
solution of the same discretisation; on the star it must too; two solves are bitwise equal;
and a group solve with GMRES members equals their own solves."""
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


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def oracle_case(prob, mms):
    cg = G.cut_cells(prob)
    dz = D.discretize(cg, prob.a, prob.b, prob.c)
    fa = Q.cell_averages(cg, mms.f(prob.a, prob.b, prob.c))
    ga = Q.boundary_averages(cg, dz.segs, mms.u, mms.ux, mms.uy)
    want = MG.direct_solve(dz, fa.ravel() - dz.N @ ga).reshape(prob.ny, prob.nx)
    return fa, ga, want


CASES = {
    "ellipses512": (lambda: (W.three_ellipses(512), W.mms_ellipses()), 16),
    "star128": (lambda: (W.star(128), W.mms_star()), 16),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    mk, coarsest = CASES[request.param]
    prob, mms = mk()
    return (prob, coarsest) + oracle_case(prob, mms)


@pytest.mark.parametrize("m,inner", [(2, 3), (4, 1)])
def test_krylov_solve_matches_direct(case, m, inner):
    prob, coarsest, fa, ga, want = case
    s = P.Solver(prob, rtol=1e-12, max_iter=100, coarsest=coarsest, krylov=m, inner_cycles=inner)
    try:
        assert s.info.batch == 1
        u, st = s.solve(cuda(fa), cuda(ga))
        assert st.rel_residual <= 1e-12
        got = u.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
        u2, st2 = s.solve(cuda(fa), cuda(ga))
        assert st2.iterations == st.iterations and torch.equal(u, u2)
    finally:
        s.close()


def test_krylov_refuses_bad_lengths():
    for m in (-1, 9):
        with pytest.raises(P.CcmError) as e:
            P.Solver(W.star(64), krylov=m)
        assert e.value.code == -1


def test_group_with_krylov_members():
    """Members with and without the GMRES correction in one graph launch, each equal to its
    own solve."""
    members = [(W.three_ellipses(256), W.mms_ellipses(), 2), (W.star(128), W.mms_star(), 0),
               (W.three_ellipses(128, seed=3, min_gap=1.0 / 8), W.mms_ellipses(), 3)]
    solvers, data = [], []
    try:
        for p, m, k in members:
            s = P.Solver(p, rtol=1e-10, max_iter=60, krylov=k, coarsest=32 if k else 16)
            q = s.quadrature()
            data.append((torch.tensor(s.cell_averages(m.f(p.a, p.b, p.c), quad=q), device="cuda"),
                         torch.tensor(s.boundary_averages(m.u, m.ux, m.uy, quad=q), device="cuda")))
            solvers.append(s)
        ref = [s.solve(f, g) for s, (f, g) in zip(solvers, data)]
        grp = P.Group(solvers)
        try:
            us, st, rc = grp.solve([f for f, _ in data], [g for _, g in data])
        finally:
            grp.close()
        assert rc == 0
        for k, ((u0, s0), u, s) in enumerate(zip(ref, us, st)):
            assert s.iterations == s0.iterations, k
            assert s.rel_residual <= 1e-10
            assert (u - u0).abs().max().item() <= 1e-13 * u0.abs().max().item(), k
    finally:
        for s in solvers:
            s.close()
