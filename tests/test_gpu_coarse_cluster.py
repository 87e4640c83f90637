"""The cluster launch that runs the small levels of a V-cycle (parameter coarse_n) against
the multi-launch path on the same hierarchy: one V-cycle in FP64 and FP32 from a random
right-hand side, and full solves against the oracle's direct solution.  Cases put the
cluster's first level at several depths, including the level right below the finest."""
import numpy as np
import pytest

import workloads as W
from oracle import cubature as Q
from oracle import multigrid as MG

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2504_00724_gb300")

pytestmark = pytest.mark.gpu

CASES = {
    "star288_from144": (lambda: W.star(288), 160),
    "star288_from36": (lambda: W.star(288), 40),
    "disk64_from32": (lambda: W.disk_minus(64), 32),
    "ellipses128_from64": (lambda: W.three_ellipses(128), 64),
    "star96_cross0_from48": (lambda: W.star(96, (1.0, 0.0, 1.0)), 48),
}


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module", params=list(CASES))
def pair(request):
    mk, cn = CASES[request.param]
    prob = mk()
    multi = P.Solver(prob, rtol=1e-12, max_iter=200, coarse_n=0)
    clus = P.Solver(prob, rtol=1e-12, max_iter=200, coarse_n=cn)
    yield prob, multi, clus
    multi.close()
    clus.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-5)])
def test_vcycle_cluster_matches_multi_launch(pair, precision, tol):
    prob, multi, clus = pair
    st = multi.cell_map()[0]
    rng = np.random.default_rng(3)
    r = cuda(np.where(st != 0, rng.standard_normal(st.shape), 0.0))
    u0 = cuda(np.where(st != 0, rng.standard_normal(st.shape), 0.0))
    for rep in range(2):       # the second call starts from the buffers the first one left
        want = host(multi.vcycle(u0.clone(), r, precision))
        got = host(clus.vcycle(u0.clone(), r, precision))
        assert np.all(np.isfinite(got))
        assert np.abs(got - want).max() <= tol * np.abs(want).max(), rep


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_with_cluster_matches_direct(pair, precision):
    prob, multi, clus = pair
    mms = W.mms_star()
    H = MG.build_hierarchy(prob)
    lv = H.levels[0]
    fa = Q.cell_averages(lv.cg, mms.f(prob.a, prob.b, prob.c))
    ga = Q.boundary_averages(lv.cg, lv.dz.segs, mms.u, mms.ux, mms.uy)
    want = MG.direct_solve(lv.dz, fa.ravel() - lv.dz.N @ ga).reshape(lv.ny, lv.nx)
    solver = clus if precision == 1 else P.Solver(prob, rtol=1e-12, max_iter=200, precision=0,
                                                    coarse_n=clus.params.coarse_n)
    try:
        u, stats = solver.solve(cuda(fa), cuda(ga))
        assert stats.rel_residual <= 1e-12
        assert np.abs(host(u) - want).max() <= 1e-10 * np.abs(want).max()
    finally:
        if solver is not clus:
            solver.close()
