"""Many geometries of uneven grid sizes advanced by one graph launch (ccm_group_solve): every
member's solution, iteration count and residual history equal those of its own ccm_solve
(the same kernels on the same data; only the convergence test runs on the device), members
retire independently (an iteration limit, an already-converged start), and bad arguments are
rejected."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2504_00724_gb300")

pytestmark = pytest.mark.gpu


def _inputs(s, prob, mms):
    q = s.quadrature()
    f = torch.tensor(s.cell_averages(mms.f(prob.a, prob.b, prob.c), quad=q), device="cuda")
    g = torch.tensor(s.boundary_averages(mms.u, mms.ux, mms.uy, quad=q), device="cuda")
    return f, g


def _members():
    probs = [W.geometry_of_seed(k) for k in range(6)]
    # uneven sizes small enough for a test: the drawn geometry on a 64..256 grid
    sizes = [64, 128, 256, 64, 128, 96]
    out = []
    for p, n in zip(probs, sizes):
        p.nx = p.ny = n
        p.h = 1.0 / n
        out.append(p)
    out.append(W.three_ellipses(128))
    return out


@pytest.fixture(scope="module")
def setups():
    mms = W.mms_star()
    probs = _members()
    precs = [P.CCM_MIXED] * (len(probs) - 2) + [P.CCM_FP64, P.CCM_MIXED]
    solvers = [P.Solver(p, rtol=1e-10, max_iter=60, precision=pr) for p, pr in zip(probs, precs)]
    data = [_inputs(s, p, W.mms_ellipses() if p.name.startswith("three") else mms) for s, p in zip(solvers, probs)]
    yield probs, solvers, data
    for s in solvers:
        s.close()


def test_group_equals_individual_solves(setups):
    probs, solvers, data = setups
    ref = [s.solve(f, g) for s, (f, g) in zip(solvers, data)]
    grp = P.Group(solvers)
    try:
        us, st, rc = grp.solve([f for f, _ in data], [g for _, g in data])
        assert rc == 0
        for k, ((u0, s0), u, s) in enumerate(zip(ref, us, st)):
            assert s.iterations == s0.iterations, k
            assert s.rel_residual <= 1e-10
            assert s.rel_residual == pytest.approx(s0.rel_residual, rel=1e-12, abs=0), k
            hist = np.array(s.history[:s.iterations + 1])
            hist0 = np.array(s0.history[:s0.iterations + 1])
            assert np.allclose(hist, hist0, rtol=1e-12, atol=0), k
            d = (u - u0).abs().max().item()
            assert d <= 1e-13 * u0.abs().max().item(), (k, d)
        # a second solve from the graph captured once gives the same answer
        us2, st2, rc2 = grp.solve([f for f, _ in data], [g for _, g in data])
        assert rc2 == 0
        for u, u2 in zip(us, us2):
            assert torch.equal(u, u2)
    finally:
        grp.close()


def test_members_retire_independently(setups):
    probs, solvers, data = setups
    mk = lambda: W.geometry_of_seed(3)
    p = mk()
    p.nx = p.ny = 64
    p.h = 1.0 / 64
    limited = P.Solver(p, rtol=1e-10, max_iter=2, precision=P.CCM_MIXED)
    try:
        f, g = _inputs(limited, p, W.mms_star())
        members = [solvers[0], limited, solvers[1]]
        zero = torch.zeros_like(data[1][0])
        grp = P.Group(members)
        try:
            us, st, rc = grp.solve([data[0][0], f, zero], [data[0][1], g, torch.zeros_like(data[1][1])], check=False)
        finally:
            grp.close()
        assert rc == -5                          # CCM_ENOCONV: the limited member
        assert st[1].iterations == 2 and st[1].rel_residual > 1e-10
        assert st[0].iterations > 2 and st[0].rel_residual <= 1e-10
        assert st[2].iterations == 0             # zero data: converged before the first pass
        assert us[2].abs().max().item() == 0.0
    finally:
        limited.close()


def test_bad_groups_rejected(setups):
    _, solvers, _ = setups
    with pytest.raises(P.CcmError) as e:
        P.Group([solvers[0], solvers[0]])
    assert e.value.code == -1
    with pytest.raises(P.CcmError):
        P.Group([])
