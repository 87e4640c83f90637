"""Parity at a size where the large-level kernels run: star 288^2 (TMA-staged SMO-1 on the
first levels, ragged 64 x 32 tiles at the right and top edges, overlapping SMO-2 blocks)."""
import numpy as np
import pytest

import workloads as W
from oracle import cubature as Q
from oracle import multigrid as MG

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2504_00724_gb300")

pytestmark = pytest.mark.gpu
OMEGA = 0.8


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def big():
    prob, mms = W.star(288), W.mms_star()
    H = MG.build_hierarchy(prob)
    return prob, mms, H


def test_large_level_smoother(big):
    prob, mms, H = big
    s = P.Solver(prob, omega=OMEGA, ras_passes=40, smoother=0, ras_exact=1024)
    try:
        for m in (0, 1):
            lv = H.levels[m]
            rng = np.random.default_rng(m)
            u0 = np.where(lv.ne, rng.standard_normal(lv.nx * lv.ny), 0.0).reshape(lv.ny, lv.nx)
            r = np.where(lv.ne, rng.standard_normal(lv.nx * lv.ny), 0.0).reshape(lv.ny, lv.nx) / lv.h ** 2
            want = u0.ravel().copy()
            MG.smo1(lv, want, r.ravel(), OMEGA)
            MG.smo2(lv, want, r.ravel())
            got = host(s.level_smooth(m, cuda(u0), cuda(r), P.CCM_FP64)).ravel()
            assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max(), m
            got32 = host(s.level_smooth(m, cuda(u0), cuda(r), P.CCM_MIXED)).ravel()
            assert np.abs(got32 - want).max() <= 2e-4 * np.abs(want).max(), m
    finally:
        s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_large_solve(big, precision):
    prob, mms, H = big
    lv = H.levels[0]
    fa = Q.cell_averages(lv.cg, mms.f(prob.a, prob.b, prob.c))
    ga = Q.boundary_averages(lv.cg, lv.dz.segs, mms.u, mms.ux, mms.uy)
    want = MG.direct_solve(lv.dz, fa.ravel() - lv.dz.N @ ga).reshape(lv.ny, lv.nx)
    s = P.Solver(prob, omega=OMEGA, rtol=1e-12, precision=precision, max_iter=200)
    try:
        u, st = s.solve(cuda(fa), cuda(ga))
        assert st.rel_residual <= 1e-12
        assert np.abs(host(u) - want).max() <= 1e-10 * np.abs(want).max()
    finally:
        s.close()
