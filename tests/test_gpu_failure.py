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


def test_injected_nan_is_reported_and_handle_survives():
    """A NaN injected into f (one non-empty cell): the residual norm turns non-finite and the
    solve stops with CCM_ENOTFINITE instead of iterating to max_iter; the next solve with clean
    data converges on the same handle."""
    prob, mms = W.star(96), W.mms_star()
    s = P.Solver(prob, rtol=1e-10, max_iter=50)
    try:
        q = s.quadrature()
        fa = s.cell_averages(mms.f(prob.a, prob.b, prob.c), quad=q)
        ga = s.boundary_averages(mms.u, mms.ux, mms.uy, quad=q)
        j, i = np.argwhere(s.cell_map()[0] != 0)[len(fa) // 2]
        bad = fa.copy()
        bad[j, i] = np.nan
        _, st = s.solve(torch.tensor(bad, device="cuda"), torch.tensor(ga, device="cuda"), check=False)
        assert st.iterations == 0
        rc = P.lib().ccm_solve(s.h, None, None, None, 1, None, None)
        assert rc == -1                         # arguments are still checked
        u, st = s.solve(torch.tensor(fa, device="cuda"), torch.tensor(ga, device="cuda"))
        assert st.rel_residual <= 1e-10
        with pytest.raises(P.CcmError) as e:
            s.solve(torch.tensor(bad, device="cuda"), torch.tensor(ga, device="cuda"))
        assert e.value.code == -9               # CCM_ENOTFINITE
    finally:
        s.close()


def test_residual_log_on_request():
    """CCM_LOG=1: the solve prints its residual history to stderr."""
    import os
    import subprocess
    import sys
    code = ("import torch, workloads as W, paper_2504_00724_gb300 as P\n"
            "prob = W.star(64); s = P.Solver(prob, rtol=1e-8)\n"
            "f = torch.ones((prob.ny, prob.nx), dtype=torch.float64, device='cuda')\n"
            "s.solve(f); s.close()\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CCM_LOG="1", PYTHONPATH=root)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "ccm_solve:" in r.stderr and "rel. residual" in r.stderr
