"""The Robin condition gamma1 u + gamma2 du/dn = g on a curve (Sec. 3.3 boundary operator)
solved on the GPU: the max-norm error against the exact cell averages falls at fourth order,
and the mixed-precision form reaches the FP64 form's error to two significant digits."""
import math

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2504_00724_gb300")

pytestmark = pytest.mark.gpu


def _error(prob, mms, precision):
    s = P.Solver(prob, rtol=1e-12, max_iter=300, precision=precision)
    try:
        q = s.quadrature()
        gam = s.boundary_operator()
        cell, bc, _ = s.boundary_segments()
        rob = bc == P.CCM_ROBIN
        assert rob.any() and np.all(bc[~rob] == P.CCM_DIRICHLET)
        assert np.array_equal(gam[rob], np.broadcast_to(prob.curves[0].robin, gam[rob].shape))
        assert np.array_equal(gam[~rob], np.broadcast_to((1.0, 0.0), gam[~rob].shape))
        fa = s.cell_averages(mms.f(prob.a, prob.b, prob.c), quad=q)
        ga = s.boundary_averages(mms.u, mms.ux, mms.uy, quad=q)
        ua = s.cell_averages(mms.u, quad=q)
        u, st = s.solve(torch.tensor(fa, device="cuda"), torch.tensor(ga, device="cuda"))
        assert st.rel_residual <= 1e-12
        ne = s.cell_map()[0] != 0
        return float(np.abs(u.cpu().numpy() - ua)[ne].max())
    finally:
        s.close()


@pytest.mark.parametrize("gamma,abc", [((1.0, 0.5), (1.0, 0.0, 1.0)), ((1.0, 2.0), (1.0, 0.5, 2.0))])
def test_robin_fourth_order_fp64_and_mixed(gamma, abc):
    sizes = (64, 128, 256)
    e64 = [_error(W.disk_robin(n, gamma, abc=abc), W.mms_disk(), P.CCM_FP64) for n in sizes]
    em = [_error(W.disk_robin(n, gamma, abc=abc), W.mms_disk(), P.CCM_MIXED) for n in sizes]
    for a, b in zip(e64[1:], e64[:-1]):
        assert math.log2(b / a) > 3.5, e64
    for a, b in zip(e64, em):
        assert float(f"{a:.1e}") == float(f"{b:.1e}"), (e64, em)
