"""The FMG cycle (ccm_fmg, and ccm_params.cycle = 1 in the mixed solve) against the oracle:
with the exact sequential smoother one FMG cycle equals the oracle's FMG cycle; mixed solves
whose outer iterations start with an FMG cycle reach the oracle's direct solution, one
right-hand side at a time and batched."""
import numpy as np
import pytest

import workloads as W
from oracle import cubature as Q
from oracle import multigrid as MG

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2504_00724_gb300")

pytestmark = pytest.mark.gpu

CASES = {
    "star64": (lambda: W.star(64), W.mms_star),
    "disk32": (lambda: W.disk_minus(32), W.mms_disk),
    "ellipses64": (lambda: W.three_ellipses(64), W.mms_ellipses),
    "star160": (lambda: W.star(160), W.mms_star),
}
OMEGA = 0.8


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    mk, mms = CASES[request.param]
    prob = mk()
    H = MG.build_hierarchy(prob)
    return prob, mms(), H


def test_fmg_cycle_matches_oracle(case):
    prob, mms, H = case
    lv = H.levels[0]
    rng = np.random.default_rng(23)
    r = np.where(lv.ne, rng.standard_normal(lv.nx * lv.ny), 0.0) / lv.h ** 2
    want = MG.fmg(H, r, omega=OMEGA, nu1=3, nu2=3)
    s = P.Solver(prob, omega=OMEGA, ras_passes=40, smoother=0, ras_exact=1024)
    try:
        got = host(s.fmg(cuda(r.reshape(lv.ny, lv.nx)), P.CCM_FP64)).ravel()
        assert np.abs(got - want).max() <= 1e-8 * np.abs(want).max()
    finally:
        s.close()


@pytest.mark.parametrize("batch", [1, 2])
def test_mixed_solve_with_fmg_matches_direct(case, batch):
    prob, mms, H = case
    lv = H.levels[0]
    fa = Q.cell_averages(lv.cg, mms.f(prob.a, prob.b, prob.c))
    ga = Q.boundary_averages(lv.cg, lv.dz.segs, mms.u, mms.ux, mms.uy)
    want = MG.direct_solve(lv.dz, fa.ravel() - lv.dz.N @ ga).reshape(lv.ny, lv.nx)
    s = P.Solver(prob, rtol=1e-12, max_iter=200, cycle=1, batch=batch)
    try:
        F = np.stack([fa, 2.0 * fa, -fa][:max(batch, 1) + 1])
        G = np.stack([ga, 2.0 * ga, -ga][:max(batch, 1) + 1])
        u, st = s.solve(cuda(F), cuda(G))
        assert st.rel_residual <= 1e-12
        got = host(u)
        for k, scale in enumerate((1.0, 2.0, -1.0)[:len(F)]):
            assert np.abs(got[k] - scale * want).max() <= 1e-10 * np.abs(want).max(), k
    finally:
        s.close()
