"""Batched right-hand sides (ccm_params.batch): one graph replay advances several right-hand
sides of one geometry, every kernel taking its right-hand side from the grid's y index.
Each solution of a batch must equal the oracle's direct solution for its own right-hand
side.  Five right-hand sides in batches of three leave a second, smaller group, which
takes a second graph capture."""
import numpy as np
import pytest

import workloads as W
from oracle import multigrid as MG

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2504_00724_gb300")

pytestmark = pytest.mark.gpu

CASES = {
    "star96": lambda: W.star(96),
    "disk128": lambda: W.disk_minus(128),
    "ellipses128": lambda: W.three_ellipses(128),
}


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    prob = CASES[request.param]()
    H = MG.build_hierarchy(prob)
    lv = H.levels[0]
    nrhs = 5
    rng = np.random.default_rng(17)
    ne = lv.ne.reshape(lv.ny, lv.nx)
    F = np.stack([np.where(ne, rng.standard_normal(ne.shape), 0.0) for _ in range(nrhs)])
    G = rng.standard_normal((nrhs, lv.dz.N.shape[1]))
    want = np.stack([MG.direct_solve(lv.dz, F[b].ravel() - lv.dz.N @ G[b]).reshape(lv.ny, lv.nx)
                     for b in range(nrhs)])
    return prob, F, G, want


def test_batched_solve_matches_direct(case):
    prob, F, G, want = case
    s = P.Solver(prob, rtol=1e-12, max_iter=200, batch=3)
    try:
        assert s.info.batch == 3
        for rep in range(2):        # the second call reuses both captured groups
            u, st = s.solve(cuda(F), cuda(G))
            assert st.rel_residual <= 1e-12
            got = host(u)
            for b in range(len(F)):
                assert np.abs(got[b] - want[b]).max() <= 1e-10 * np.abs(want[b]).max(), (rep, b)
    finally:
        s.close()


def test_batch_equals_one_at_a_time(case):
    prob, F, G, want = case
    one = P.Solver(prob, rtol=1e-12, max_iter=200)
    many = P.Solver(prob, rtol=1e-12, max_iter=200, batch=5)
    try:
        assert one.info.batch == 1 and many.info.batch == 5
        u1, _ = one.solve(cuda(F), cuda(G))
        u5, _ = many.solve(cuda(F), cuda(G))
        a, b = host(u1), host(u5)
        assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max()
    finally:
        one.close()
        many.close()


def test_batch_needs_the_block_jacobi_smoother(case):
    """With the sequential smoother the handle runs one right-hand side at a time."""
    prob, F, G, want = case
    s = P.Solver(prob, rtol=1e-12, max_iter=300, batch=4, smoother=0)
    try:
        assert s.info.batch == 1
        u, st = s.solve(cuda(F[:2]), cuda(G[:2]))
        got = host(u)
        for b in range(2):
            assert np.abs(got[b] - want[b]).max() <= 1e-10 * np.abs(want[b]).max()
    finally:
        s.close()
