"""Failure detection without a GPU fault: a kernel waits, with the solve kernels' bounded-wait
helper, on an mbarrier phase that nothing completes.  The wait runs out, the error word comes
back as CCM_ETIMEOUT, and the same handle then solves normally (the context stays usable)."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2504_00724_gb300")

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_context_survives():
    prob, mms = W.star(128), W.mms_star()
    s = P.Solver(prob, rtol=1e-10)
    try:
        assert s.wait_selftest() == -6          # CCM_ETIMEOUT
        q = s.quadrature()
        f = torch.tensor(s.cell_averages(mms.f(prob.a, prob.b, prob.c), quad=q), device="cuda")
        g = torch.tensor(s.boundary_averages(mms.u, mms.ux, mms.uy, quad=q), device="cuda")
        u, st = s.solve(f, g)
        assert st.rel_residual <= 1e-10
        assert s.wait_selftest() == -6          # again, after a solve
        u2, st2 = s.solve(f, g)
        assert torch.equal(u, u2) and st2.iterations == st.iterations
    finally:
        s.close()
