"""A Y_c domain (the interior of a closed cubic spline, Sec. 2) solved on the GPU: the
max-norm error against the exact cell averages falls at fourth order, and the mixed form
reaches the FP64 form's error to two significant digits."""
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
        f = torch.tensor(s.cell_averages(mms.f(prob.a, prob.b, prob.c), quad=q), device="cuda")
        g = torch.tensor(s.boundary_averages(mms.u, mms.ux, mms.uy, quad=q), device="cuda")
        ua = s.cell_averages(mms.u, quad=q)
        u, st = s.solve(f, g)
        assert st.rel_residual <= 1e-12
        ne = s.cell_map()[0] != 0
        return float(np.abs(u.cpu().numpy() - ua)[ne].max())
    finally:
        s.close()


def test_spline_domain_fourth_order_fp64_and_mixed():
    sizes = (64, 128, 256)
    e64 = [_error(W.spline_blob(n), W.mms_star(), P.CCM_FP64) for n in sizes]
    em = [_error(W.spline_blob(n), W.mms_star(), P.CCM_MIXED) for n in sizes]
    for a, b in zip(e64[1:], e64[:-1]):
        assert math.log2(b / a) > 3.5, e64
    for a, b in zip(e64, em):
        assert float(f"{a:.1e}") == float(f"{b:.1e}"), (e64, em)
