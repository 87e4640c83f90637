"""Adjoint path: ccm_solve_T against the oracle's transposed system, the dot-product identity
of the device solves, and gradients of a quadratic loss against central finite differences
(exact for a quadratic loss up to rounding) in seeded random directions."""
import numpy as np
import pytest

import workloads as W
from oracle import cubature as Q
from oracle import discretization as D
from oracle import geometry as G
from oracle import multigrid as MG

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2504_00724_gb300")
from paper_2504_00724_gb300 import autograd as AG  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = {
    "star64": lambda: W.star(64, (1.0, 0.3, 1.0)),
    "disk32": lambda: W.disk_minus(32),
    "ellipses64": lambda: W.three_ellipses(64),
    "star288": lambda: W.star(288, (1.0, 0.3, 1.0)),
}


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    prob = CASES[request.param]()
    cg = G.cut_cells(prob)
    dz = D.discretize(cg, prob.a, prob.b, prob.c)
    return prob, cg, dz


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_T_matches_oracle(case, precision):
    prob, cg, dz = case
    ne = (cg.status != 0).ravel()
    idx = np.nonzero(ne)[0]
    rng = np.random.default_rng(5)
    b = np.where(ne, rng.standard_normal(ne.size), 0.0)
    import scipy.sparse.linalg as spla
    want = np.zeros(ne.size)
    want[idx] = spla.spsolve(dz.L[idx][:, idx].T.tocsc(), b[idx])
    s = P.Solver(prob, rtol=1e-12, precision=precision, max_iter=300)
    try:
        lam, st = s.solve_T(cuda(b.reshape(prob.ny, prob.nx)))
        assert st.rel_residual <= 1e-12
        got = host(lam).ravel()
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
    finally:
        s.close()


@pytest.mark.parametrize("eps,tol", [(1e-6, 2e-7), (1e-3, 2e-9)])
def test_adjoint_dot_product_and_fd_gradients(case, eps, tol):
    prob, cg, dz = case
    mms = W.mms_star()
    ne = (cg.status != 0)
    fa = Q.cell_averages(cg, mms.f(prob.a, prob.b, prob.c))
    ga = Q.boundary_averages(cg, dz.segs, mms.u, mms.ux, mms.uy)
    ua = Q.cell_averages(cg, mms.u)
    rng = np.random.default_rng(9)
    uobs = np.where(ne, ua + 1e-3 * rng.standard_normal(ua.shape), 0.0)
    s = P.Solver(prob, rtol=1e-13, precision=0, max_iter=300)
    try:
        # <solve(f), b> = <f, solve_T(b)> for the device pair
        f1 = cuda(np.where(ne, rng.standard_normal(ne.shape), 0.0))
        b1 = cuda(np.where(ne, rng.standard_normal(ne.shape), 0.0))
        u1, _ = s.solve(f1)
        l1, _ = s.solve_T(b1)
        lhs, rhs = float((u1 * b1).sum()), float((f1 * l1).sum())
        assert abs(lhs - rhs) <= 1e-10 * float((u1 * b1).abs().sum())

        f = cuda(fa).requires_grad_(True)
        g = cuda(ga).requires_grad_(True)
        ob = cuda(uobs)

        def loss(ff, gg):
            u = AG.solve(s, ff, gg)
            return 0.5 * ((u - ob) ** 2 * cuda(ne.astype(float))).sum()

        J = loss(f, g)
        J.backward()
        gf, gg = f.grad.detach().clone(), g.grad.detach().clone()
        for k in range(4):
            df = cuda(np.where(ne, rng.standard_normal(ne.shape), 0.0))
            dg = cuda(rng.standard_normal(len(ga)))
            with torch.no_grad():
                jp = loss(f + eps * df, g + eps * dg).item()
                jm = loss(f - eps * df, g - eps * dg).item()
            fd = (jp - jm) / (2 * eps)
            ad = float((gf * df).sum() + (gg * dg).sum())
            # the loss is quadratic in (f, g): central differences carry no truncation error
            # at any step, only J's rounding and the solves' stopping points, divided by eps
            assert abs(fd - ad) <= tol * abs(ad), (k, fd, ad, abs(fd - ad) / abs(ad))
    finally:
        s.close()
