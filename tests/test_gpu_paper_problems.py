"""The paper's convergence tests solved on the GPU (Sec. 5.1): Problem 1 (the flower
exterior, Dirichlet on the box, Neumann on the flower), Problem 2 (the ellipse hole,
Dirichlet and Neumann on the ellipse) and Problem 3, case (i) (the box with (a, b, c) =
(1, 0, 2)).  Solution errors against the exact cell averages must lie within a factor of
the errors the paper prints (tests/golden) - 5 for Problem 2, whose PLG stencils near the
curve differ from the paper's (the oracle's pin uses the same factor), 3 for the others - fall
at a fourth-order rate, and the mixed form must give the FP64 form's error to two
significant digits."""
import os

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2504_00724_gb300")

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if len(parts) == 4:      # case, h, norm, value
                case, h, norm, val = parts
            else:
                case, (h, norm, val) = "", parts
            if norm == "Linf":
                rows[(case, int(h.split("/")[1]))] = float(val)
    return rows


def _error(prob, mms, precision):
    s = P.Solver(prob, rtol=1e-12, max_iter=300, precision=precision)
    try:
        q = s.quadrature()
        fa = s.cell_averages(mms.f(prob.a, prob.b, prob.c), quad=q)
        ga = s.boundary_averages(mms.u, mms.ux, mms.uy, quad=q)
        ua = s.cell_averages(mms.u, quad=q)
        f = torch.tensor(fa, device="cuda")
        g = torch.tensor(ga, device="cuda")
        u, st = s.solve(f, g)
        assert st.rel_residual <= 1e-12
        ne = s.cell_map()[0] != 0
        return float(np.abs(u.cpu().numpy() - ua)[ne].max())
    finally:
        s.close()


CASES = {
    "problem1_flower": (W.paper_problem1, W.mms_problem1, "paper_problem1.txt", "", 3.0, (40, 80, 160)),
    "problem3_rotated": (W.paper_problem3_rotated, W.mms_problem3_rotated, "paper_problem3_rotated.txt", "", 3.0,
                         (64, 128, 256)),
    "problem2_DD": (lambda n: W.paper_problem2(n, W.DIRICHLET), W.mms_sinsin, "paper_problem2.txt", "DD", 5.0,
                    (64, 128, 256)),
    "problem2_DN": (lambda n: W.paper_problem2(n, W.NEUMANN), W.mms_sinsin, "paper_problem2.txt", "DN", 5.0,
                    (64, 128, 256)),
    "problem3_box": (W.paper_problem3, W.mms_problem3, "paper_problem3.txt", "", 3.0, (64, 128, 256)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_paper_errors_and_rates(name):
    mk, mms, golden, case, factor, sizes = CASES[name]
    paper = _golden(golden)
    errs = {}
    for n in sizes:
        e64 = _error(mk(n), mms(), P.CCM_FP64)
        e32 = _error(mk(n), mms(), P.CCM_MIXED)
        assert abs(e32 - e64) <= 0.05 * e64, (n, e32, e64)     # equal to two significant digits
        errs[n] = e64
        want = paper[(case, n)]
        assert want / factor <= e64 <= want * factor, (n, e64, want)
    n0, n1, n2 = sizes
    assert np.log2(errs[n0] / errs[n1]) > 3.3
    assert np.log2(errs[n1] / errs[n2]) > 3.3
