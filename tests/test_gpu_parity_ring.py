"""Parity of the persistent kernels on the path the benchmarked sizes take: every CTA works
through two or more items of its two-stage copy ring (stage reuse, mbarrier phase flips).

The smoothing sweep (SMO-1 tiles and SMO-2 blocks, Sec. 4.1) and the residual + restriction
(Alg. 2) each run as one launch of G CTAs per right-hand side; CTA c takes items c, c + G, ...
ccm_level_launch reports the items and G, and every test asserts items > G (or more), so that
the ring really turns.  Three ways to get there:
  * the launch cap (ccm_set_launch_cap) on star 288^2: a few CTAs take every item, through
    many phase flips, for the sweep, the restriction and whole solves;
  * star 1024^2 at the default launch shape: level 0 has more items than resident CTAs in
    FP64 (in FP32, whose three resident CTAs per SM outnumber them, on half the grid);
  * 64 right-hand sides on star 288^2: 456 / 64 = 8 CTAs per right-hand side.
Expected values come from the oracle: its level-0 operator, the block-Jacobi sweep written out
on it (also from the prolonged iterate, for the first post-smoothing sweep with the
prolongation fused), its restriction and its sparse direct solve."""
from types import SimpleNamespace

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import cubature as Q
from oracle import discretization as D
from oracle import geometry as G
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


def level0(prob):
    """The oracle's finest level (cut cells, operator) and the coarse level's cell map."""
    cg = G.cut_cells(prob)
    dz = D.discretize(cg, prob.a, prob.b, prob.c)
    st = D.regular_stencil(prob.a, prob.b, prob.c)
    lv = SimpleNamespace(cg=cg, dz=dz, nx=prob.nx, ny=prob.ny, h=prob.h,
                         ne=(cg.status != G.EMPTY).ravel(), reg=dz.regular.ravel(),
                         diag=st[(0, 0)] / prob.h ** 2)
    pc = MG.coarsen(prob, 1)
    cc = G.cut_cells(pc)
    coarse = SimpleNamespace(nx=pc.nx, ny=pc.ny, ne=(cc.status != G.EMPTY).ravel())
    return lv, coarse


def block_jacobi_sweep(lv, cells, u, r, omega, block, overlap):
    """One sweep of the default smoother from its definition: SMO-1 on the regular cells and,
    for each run of `block` consecutive fitted rows (product row order = Alg. 3's boundary
    order) widened by `overlap` rows on each side, the exact solve of L22 on the widened rows
    kept on the core rows; all from the old iterate.  Sparse slicing, so that it scales."""
    L = lv.dz.L.tocsr()
    res = r - L @ u
    out = u.copy()
    out[lv.reg] += omega / lv.diag * res[lv.reg]
    n2 = len(cells)
    L22 = L[cells][:, cells].tocsr()
    for cs in range(0, n2, block):
        ce = min(n2, cs + block)
        es, ee = max(0, cs - overlap), min(n2, ce + overlap)
        x = np.linalg.solve(L22[es:ee, es:ee].toarray(), res[cells[es:ee]])
        out[cells[cs:ce]] = u[cells[cs:ce]] + x[cs - es:ce - es]
    return out


def check_sweep(s, lv, seed, precision, tol):
    cells = s.level_rows(0)[0].astype(np.int64)
    rng = np.random.default_rng(seed)
    u0 = np.where(lv.ne, rng.standard_normal(lv.nx * lv.ny), 0.0)
    r = np.where(lv.ne, rng.standard_normal(lv.nx * lv.ny), 0.0) / lv.h ** 2
    want = block_jacobi_sweep(lv, cells, u0, r, OMEGA, s.params.ras_block, s.params.ras_overlap)
    got = host(s.level_smooth(0, cuda(u0.reshape(lv.ny, lv.nx)), cuda(r.reshape(lv.ny, lv.nx)),
                              precision)).ravel()
    assert np.abs(got - want).max() <= tol * np.abs(want).max()


def check_prolong_sweep(s, lv, coarse, seed, precision, tol):
    """The first post-smoothing sweep with the prolongation fused (what the V-cycle runs)
    against the oracle's prolongation followed by the block-Jacobi sweep."""
    cells = s.level_rows(0)[0].astype(np.int64)
    rng = np.random.default_rng(seed)
    u0 = np.where(lv.ne, rng.standard_normal(lv.nx * lv.ny), 0.0)
    uc = np.where(coarse.ne, rng.standard_normal(coarse.nx * coarse.ny), 0.0)
    r = np.where(lv.ne, rng.standard_normal(lv.nx * lv.ny), 0.0) / lv.h ** 2
    start = u0 + MG.prolong(lv, coarse, uc)
    assert np.abs(start - u0).max() > 0.5          # the correction reaches the regular cells
    want = block_jacobi_sweep(lv, cells, start, r, OMEGA, s.params.ras_block, s.params.ras_overlap)
    got = host(s.level_prolong_smooth(0, cuda(u0.reshape(lv.ny, lv.nx)), cuda(uc.reshape(coarse.ny, coarse.nx)),
                                      cuda(r.reshape(lv.ny, lv.nx)), precision)).ravel()
    assert np.abs(got - want).max() <= tol * np.abs(want).max()


def check_restrict(s, lv, coarse, seed):
    rng = np.random.default_rng(seed)
    u = np.where(lv.ne, rng.standard_normal(lv.nx * lv.ny), 0.0)
    r = np.where(lv.ne, rng.standard_normal(lv.nx * lv.ny), 0.0) / lv.h ** 2
    got = host(s.level_restrict(0, cuda(u.reshape(lv.ny, lv.nx)), cuda(r.reshape(lv.ny, lv.nx)))).ravel()
    res = np.where(lv.ne, r - lv.dz.L @ u, 0.0)
    want = MG.restrict(lv, coarse, res)
    scale = MG.restrict(lv, coarse, np.abs(r) + abs(lv.dz.L) @ np.abs(u))
    assert np.all(np.abs(got - want) <= 1e-10 * scale + 1e-300)


# ------------------------------------------------------------ launch cap on star 288^2

CAP = 4


@pytest.fixture(scope="module")
def star288():
    prob, mms = W.star(288), W.mms_star()
    lv, coarse = level0(prob)
    fa = Q.cell_averages(lv.cg, mms.f(prob.a, prob.b, prob.c))
    ga = Q.boundary_averages(lv.cg, lv.dz.segs, mms.u, mms.ux, mms.uy)
    want = MG.direct_solve(lv.dz, fa.ravel() - lv.dz.N @ ga).reshape(lv.ny, lv.nx)
    return prob, lv, coarse, fa, ga, want


@pytest.mark.parametrize("precision,tol", [(P.CCM_FP64, 1e-10), (P.CCM_MIXED, 2e-4)])
def test_capped_sweep_matches_block_jacobi(star288, precision, tol):
    prob, lv, coarse, *_ = star288
    s = P.Solver(prob, omega=OMEGA)
    try:
        s.set_launch_cap(CAP)
        li = s.level_launch(0, precision)
        assert li.sweep_ctas == CAP and li.sweep_items >= 3 * CAP and li.sweep_blocks > CAP
        check_sweep(s, lv, 41, precision, tol)
    finally:
        s.close()


@pytest.mark.parametrize("precision,tol", [(P.CCM_FP64, 1e-10), (P.CCM_MIXED, 2e-4)])
def test_capped_prolong_sweep_matches_oracle(star288, precision, tol):
    prob, lv, coarse, *_ = star288
    s = P.Solver(prob, omega=OMEGA)
    try:
        s.set_launch_cap(CAP)
        li = s.level_launch(0, precision)
        assert li.sweep_ctas == CAP and li.sweep_items >= 3 * CAP and li.sweep_blocks > CAP
        check_prolong_sweep(s, lv, coarse, 47, precision, tol)
    finally:
        s.close()


def test_capped_restrict_matches_oracle(star288):
    prob, lv, coarse, *_ = star288
    s = P.Solver(prob)
    try:
        s.set_launch_cap(CAP)
        li = s.level_launch(0, P.CCM_FP64)
        assert li.restrict_ctas == CAP and li.restrict_items >= 3 * CAP
        check_restrict(s, lv, coarse, 43)
    finally:
        s.close()


@pytest.mark.parametrize("precision", [P.CCM_FP64, P.CCM_MIXED])
def test_capped_solve_matches_direct(star288, precision):
    """Whole solves with every persistent launch of every level on CAP CTAs."""
    prob, lv, coarse, fa, ga, want = star288
    s = P.Solver(prob, rtol=1e-12, precision=precision, max_iter=200)
    try:
        s.set_launch_cap(CAP)
        for m in range(s.info.levels - 1):
            li = s.level_launch(m, precision)
            assert li.sweep_ctas <= CAP and li.restrict_ctas <= CAP
        assert s.level_launch(0, precision).sweep_items > 10 * CAP
        u, st = s.solve(cuda(fa), cuda(ga))
        assert st.rel_residual <= 1e-12
        assert np.abs(host(u) - want).max() <= 1e-10 * np.abs(want).max()
    finally:
        s.close()


@pytest.mark.parametrize("block,overlap", [(32, 16), (96, 8)])
def test_rebuilt_smo2_blocks(star288, block, overlap):
    """ccm_set_smo2_blocks on a set-up handle: the sweep equals the block-Jacobi sweep with the
    new blocks, under the launch cap, and a solve still equals the direct solution."""
    prob, lv, coarse, fa, ga, want = star288
    s = P.Solver(prob, omega=OMEGA, rtol=1e-12, max_iter=200)
    try:
        s.set_smo2_blocks(block, overlap)
        s.set_launch_cap(CAP)
        assert s.level_launch(0, P.CCM_MIXED).sweep_items > 3 * CAP
        check_sweep(s, lv, 47, P.CCM_FP64, 1e-10)
        check_sweep(s, lv, 48, P.CCM_MIXED, 2e-4)
        u, st = s.solve(cuda(fa), cuda(ga))
        assert st.rel_residual <= 1e-12
        assert np.abs(host(u) - want).max() <= 1e-10 * np.abs(want).max()
    finally:
        s.close()


def test_cap_does_not_change_results(star288):
    prob, lv, coarse, fa, ga, want = star288
    s = P.Solver(prob, rtol=1e-12, max_iter=200)
    try:
        u0, st0 = s.solve(cuda(fa), cuda(ga))
        s.set_launch_cap(3)
        u1, st1 = s.solve(cuda(fa), cuda(ga))
        assert st1.iterations == st0.iterations
        assert torch.equal(u0, u1)
        s.set_launch_cap(0)
        assert s.level_launch(0, P.CCM_MIXED).sweep_ctas > 3
    finally:
        s.close()


# ------------------------------------------------------------ star 1024^2, default launch shape

@pytest.fixture(scope="module")
def star1024():
    prob = W.star(1024)
    lv, coarse = level0(prob)
    return prob, lv, coarse


@pytest.mark.parametrize("precision,tol", [(P.CCM_FP64, 1e-10), (P.CCM_MIXED, 2e-4)])
def test_star1024_level0_sweep(star1024, precision, tol):
    prob, lv, coarse = star1024
    s = P.Solver(prob, omega=OMEGA)
    try:
        li = s.level_launch(0, precision)
        if li.sweep_items <= li.sweep_ctas:
            # FP32 keeps 3 CTAs per SM resident, more than this level's items: halve the grid
            s.set_launch_cap(li.sweep_items // 2)
            li = s.level_launch(0, precision)
        assert li.sweep_items > li.sweep_ctas > 0
        check_sweep(s, lv, 51, precision, tol)
    finally:
        s.close()


@pytest.mark.parametrize("precision,tol", [(P.CCM_FP64, 1e-10), (P.CCM_MIXED, 2e-4)])
def test_star1024_level0_prolong_sweep(star1024, precision, tol):
    prob, lv, coarse = star1024
    s = P.Solver(prob, omega=OMEGA)
    try:
        li = s.level_launch(0, precision)
        if li.sweep_items <= li.sweep_ctas:
            s.set_launch_cap(li.sweep_items // 2)
            li = s.level_launch(0, precision)
        assert li.sweep_items > li.sweep_ctas > 0
        check_prolong_sweep(s, lv, coarse, 57, precision, tol)
    finally:
        s.close()


def test_star1024_level0_restrict(star1024):
    prob, lv, coarse = star1024
    s = P.Solver(prob)
    try:
        li = s.level_launch(0, P.CCM_FP64)
        assert li.restrict_items > li.restrict_ctas > 0
        check_restrict(s, lv, coarse, 53)
    finally:
        s.close()


# ------------------------------------------------------------ 64 right-hand sides on star 288^2

def test_batch64_each_rhs_matches_direct(star288):
    prob, lv, coarse, fa, ga, want = star288
    nrhs = 64
    rng = np.random.default_rng(61)
    ne = lv.ne.reshape(lv.ny, lv.nx)
    F = np.stack([np.where(ne, rng.standard_normal(ne.shape), 0.0) for _ in range(nrhs)])
    Gb = rng.standard_normal((nrhs, lv.dz.N.shape[1]))
    idx = np.nonzero(lv.ne)[0]
    lu = spla.splu(lv.dz.L[idx][:, idx].tocsc())
    s = P.Solver(prob, rtol=1e-12, max_iter=200, batch=nrhs)
    try:
        assert s.info.batch == nrhs
        for m in range(s.info.levels - 1):
            li = s.level_launch(m, P.CCM_MIXED, nrhs)
            if li.sweep_items:
                assert li.sweep_ctas <= 8
        li = s.level_launch(0, P.CCM_MIXED, nrhs)
        assert li.sweep_items > 2 * li.sweep_ctas and li.restrict_items > 2 * li.restrict_ctas
        u, st = s.solve(cuda(F), cuda(Gb))
        assert st.rel_residual <= 1e-12
        got = host(u)
        for b in range(nrhs):
            rhs = F[b].ravel() - lv.dz.N @ Gb[b]
            w = np.zeros(lv.nx * lv.ny)
            w[idx] = lu.solve(rhs[idx])
            assert np.abs(got[b].ravel() - w).max() <= 1e-10 * np.abs(w).max(), b
    finally:
        s.close()
