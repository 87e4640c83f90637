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


def test_large_level_restrict(big):
    """Residual + restriction of the TMA-staged kernel (level 0 here) against the oracle."""
    prob, mms, H = big
    s = P.Solver(prob)
    try:
        f, c = H.levels[0], H.levels[1]
        rng = np.random.default_rng(21)
        u = np.where(f.ne, rng.standard_normal(f.nx * f.ny), 0.0).reshape(f.ny, f.nx)
        r = np.where(f.ne, rng.standard_normal(f.nx * f.ny), 0.0).reshape(f.ny, f.nx) / f.h ** 2
        got = host(s.level_restrict(0, cuda(u), cuda(r))).ravel()
        want = MG.restrict(f, c, MG.residual(f, u.ravel(), r.ravel()))
        scale = MG.restrict(f, c, np.abs(r.ravel()) + abs(f.dz.L) @ np.abs(u.ravel()))
        assert np.all(np.abs(got - want) <= 1e-10 * scale + 1e-300)
    finally:
        s.close()


def _composed_vcycle(s, levels, m, u, r, nu1=3, nu2=3, precision=P.CCM_FP64):
    """Alg. 2 spelled out through the per-level entry points (separate prolongation, no
    coarse-level cluster launch, every sweep reading its iterate)."""
    if m == levels - 1:
        return s.bottom_solve(r)
    for _ in range(nu1):
        u = s.level_smooth(m, u, r, precision)
    rc = s.level_restrict(m, u, r)
    uc = _composed_vcycle(s, levels, m + 1, torch.zeros_like(rc), rc, nu1, nu2, precision)
    u = s.level_prolong(m, uc, u)
    for _ in range(nu2):
        u = s.level_smooth(m, u, r, precision)
    return u


@pytest.mark.parametrize("n,coarse_n", [(576, 0), (576, 80), (288, 150)])
def test_vcycle_equals_composed_level_calls(n, coarse_n):
    """ccm_vcycle (prolongation fused into the first post-smoothing sweep on TMA levels, the
    small levels in one cluster launch) equals the same V-cycle built from the per-level
    calls, in FP64, with the default block-Jacobi smoother."""
    prob = W.star(n)
    s = P.Solver(prob, coarse_n=coarse_n)
    try:
        st = s.cell_map()[0]
        rng = np.random.default_rng(n + coarse_n)
        u0 = cuda(np.where(st != 0, rng.standard_normal(st.shape), 0.0))
        r = cuda(np.where(st != 0, rng.standard_normal(st.shape), 0.0) * n * n)
        want = host(_composed_vcycle(s, s.info.levels, 0, u0.clone(), r))
        got = host(s.vcycle(u0.clone(), r, P.CCM_FP64))
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    finally:
        s.close()


def test_mixed_vcycle_close_to_composed_level_calls():
    """The FP32 V-cycle (every coarse level's first sweep starting from the zero iterate the
    restriction leaves, without reading it) against the same cycle composed from FP32 level
    calls that read their iterates (and restrict in FP64): the two differ by FP32 rounding."""
    prob = W.star(576)
    s = P.Solver(prob)
    try:
        st = s.cell_map()[0]
        rng = np.random.default_rng(577)
        u0 = cuda(np.where(st != 0, rng.standard_normal(st.shape), 0.0))
        r = cuda(np.where(st != 0, rng.standard_normal(st.shape), 0.0) * 576 * 576)
        want = host(_composed_vcycle(s, s.info.levels, 0, u0.clone(), r, precision=P.CCM_MIXED))
        got = host(s.vcycle(u0.clone(), r, P.CCM_MIXED))
        assert np.abs(got - want).max() <= 1e-4 * np.abs(want).max()
    finally:
        s.close()


def _block_jacobi_sweep(lv, cells, u, r, omega, block, overlap):
    """One sweep of the device's default smoother written out from its definition: SMO-1 on
    the regular cells and, for each block of `block` consecutive fitted rows (in the product's
    row order, which is Alg. 3's boundary order) widened by `overlap` rows on each side, the
    exact solve of L22 on the widened rows, kept on the core rows; both from the old iterate."""
    L = lv.dz.L.tocsr()
    res = r - L @ u
    out = u.copy()
    out[lv.reg] += omega / lv.diag * res[lv.reg]
    n2 = len(cells)
    L22 = L[cells][:, cells].toarray()
    for cs in range(0, n2, block):
        ce = min(n2, cs + block)
        es, ee = max(0, cs - overlap), min(n2, ce + overlap)
        x = np.linalg.solve(L22[es:ee, es:ee], res[cells[es:ee]])
        out[cells[cs:ce]] = u[cells[cs:ce]] + x[cs - es:ce - es]
    return out


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 2e-4)])
def test_large_default_smoother_matches_block_jacobi(big, precision, tol):
    """The persistent sweep kernel (SMO-2 block items and TMA tile items in one launch) on the
    first level of star 288 equals the block-Jacobi sweep computed on the oracle's operator."""
    prob, mms, H = big
    hs = P.HostSetup(prob)
    s = P.Solver(prob, omega=OMEGA)
    try:
        lv = H.levels[0]
        cells = hs.rows(0)[0].astype(np.int64)
        rng = np.random.default_rng(31)
        u0 = np.where(lv.ne, rng.standard_normal(lv.nx * lv.ny), 0.0)
        r = np.where(lv.ne, rng.standard_normal(lv.nx * lv.ny), 0.0) / lv.h ** 2
        want = _block_jacobi_sweep(lv, cells, u0, r, OMEGA, s.params.ras_block, s.params.ras_overlap)
        got = host(s.level_smooth(0, cuda(u0.reshape(lv.ny, lv.nx)), cuda(r.reshape(lv.ny, lv.nx)),
                                  precision)).ravel()
        assert np.abs(got - want).max() <= tol * np.abs(want).max()
    finally:
        s.close()
        hs.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_bottom_64_cluster_split(precision):
    """A 64^2 bottom level (about 1.2k unknowns on the star, the hierarchy of the benchmark):
    the dense bottom inverse applied by a cluster of CTAs over column chunks, partial sums added
    in rank order through distributed shared memory, against the oracle's LU solve of the same
    level; and a V-cycle through that bottom level against the oracle's (FP64)."""
    prob = W.star(128)
    H = MG.build_hierarchy(prob, coarsest=64)
    assert len(H.levels) == 2 and int(H.levels[-1].ne.sum()) >= 256
    s = P.Solver(prob, omega=OMEGA, coarsest=64, ras_passes=40, smoother=0, ras_exact=1024)
    try:
        last = H.levels[-1]
        rng = np.random.default_rng(11)
        r = np.where(last.ne, rng.standard_normal(last.nx * last.ny), 0.0).reshape(last.ny, last.nx) / last.h ** 2
        want = MG.bottom(H, r.ravel())
        got = host(s.bottom_solve(cuda(r))).ravel()
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
        if precision == 0:
            lv = H.levels[0]
            u0 = np.where(lv.ne, rng.standard_normal(lv.nx * lv.ny), 0.0).reshape(lv.ny, lv.nx)
            rr = np.where(lv.ne, rng.standard_normal(lv.nx * lv.ny), 0.0).reshape(lv.ny, lv.nx) / lv.h ** 2
            want = MG.vcycle(H, 0, u0.ravel().copy(), rr.ravel(), omega=OMEGA, nu1=3, nu2=3)
            got = host(s.vcycle(cuda(u0), cuda(rr), P.CCM_FP64)).ravel()
            assert np.abs(got - want).max() <= 1e-8 * np.abs(want).max()
        else:
            # the FP32 bottom inside the mixed solve: converged to the FP64 tolerance
            mms = W.mms_star()
            q = s.quadrature()
            f = torch.tensor(s.cell_averages(mms.f(prob.a, prob.b, prob.c), quad=q), device="cuda")
            g = torch.tensor(s.boundary_averages(mms.u, mms.ux, mms.uy, quad=q), device="cuda")
            _, st = s.solve(f, g)
            assert st.rel_residual <= 1e-10
    finally:
        s.close()
