"""Pins of the oracle's multigrid (Sec. 4): smoother error property, transfers,
V-cycle convergence, agreement with a direct solve, and Alg. 3 bandwidth."""
import numpy as np
import pytest

import workloads as W
from oracle import cubature as Q
from oracle import discretization as D
from oracle import geometry as G
from oracle import multigrid as MG


def _rhs(H, prob, mms):
    lv = H.levels[0]
    fa = Q.cell_averages(lv.cg, mms.f(prob.a, prob.b, prob.c)).ravel()
    ga = Q.boundary_averages(lv.cg, lv.dz.segs, mms.u, mms.ux, mms.uy)
    r = fa - lv.dz.N @ ga
    r[~lv.ne] = 0.0
    return r


@pytest.fixture(scope="module")
def star64():
    prob = W.star(64)
    H = MG.build_hierarchy(prob)
    return prob, H, _rhs(H, prob, W.mms_star())


def test_smo2_zeroes_irregular_residual(star64):
    """eq. errorOfE2: after SMO-2 the residual of every irregular row vanishes."""
    prob, H, r = star64
    lv = H.levels[0]
    rng = np.random.default_rng(0)
    u = np.where(lv.ne, rng.standard_normal(r.shape), 0.0)
    MG.smo1(lv, u, r, 0.5)
    MG.smo2(lv, u, r)
    res = MG.residual(lv, u, r)
    assert np.abs(res[lv.irr]).max() <= 1e-12 * np.abs(r).max() * 1e3
    assert np.abs(res[lv.reg]).max() > 1e-6


def test_smo1_is_weighted_jacobi(star64):
    """SMO-1 on one regular cell equals u + w (r - L u)/D with D the stencil centre."""
    prob, H, r = star64
    lv = H.levels[0]
    rng = np.random.default_rng(1)
    u = np.where(lv.ne, rng.standard_normal(r.shape), 0.0)
    u0 = u.copy()
    MG.smo1(lv, u, r, 0.5)
    k = int(lv.reg_idx[len(lv.reg_idx) // 2])
    row = lv.dz.L.getrow(k)
    Lu = float((row @ u0)[0])
    assert abs(u[k] - (u0[k] + 0.5 * (r[k] - Lu) / row[0, k])) < 1e-12 * abs(u0[k] + 1)
    assert np.array_equal(u[lv.irr], u0[lv.irr])


def test_transfers_preserve_constants(star64):
    prob, H, r = star64
    f, c = H.levels[0], H.levels[1]
    one = np.where(f.ne, 1.0, 0.0)
    rc = MG.restrict(f, c, one)
    assert np.allclose(rc[c.ne], 1.0)
    up = MG.prolong(f, c, np.where(c.ne, 2.0, 0.0))
    assert np.allclose(up[f.reg], 2.0) and np.all(up[~f.reg] == 0.0)


def test_bottom_solve_is_exact(star64):
    prob, H, r = star64
    last = H.levels[-1]
    rng = np.random.default_rng(2)
    rr = np.where(last.ne, rng.standard_normal(last.nx * last.ny), 0.0)
    u = MG.bottom(H, rr)
    assert np.abs((last.dz.L @ u - rr)[last.ne]).max() < 1e-10 * np.abs(rr).max() / last.h ** 0


def test_vcycles_converge_to_direct_solution(star64):
    prob, H, r = star64
    hist = []
    u = MG.solve(H, r, rtol=1e-12, max_iter=80, history=hist)
    assert hist[-1] <= 1e-12
    ud = MG.direct_solve(H.levels[0].dz, r)
    ne = H.levels[0].ne
    assert np.abs(u - ud)[ne].max() <= 1e-9 * np.abs(ud[ne]).max()


@pytest.mark.slow
def test_convergence_factor_h_independent():
    """V-cycle convergence factor (paper parameters omega = 0.5, nu = 3) stays bounded and
    roughly h-independent (Sec. 4.3); measured as the geometric mean over cycles 4-10."""
    rhos = []
    for n in (64, 128):
        prob = W.star(n)
        H = MG.build_hierarchy(prob)
        r = _rhs(H, prob, W.mms_star())
        hist = []
        MG.solve(H, r, rtol=0.0, max_iter=10, history=hist)
        f = np.array(hist[1:]) / np.array(hist[:-1])
        rhos.append(float(np.exp(np.mean(np.log(f[3:])))))
    assert max(rhos) < 0.8
    assert rhos[1] < rhos[0] * 1.6


def _component_bandwidths(L, order):
    """Per connected component of the coupling graph of L22 (rows and columns in `order`):
    (size, cyclic bandwidth within the component, whether the component is contiguous)."""
    import scipy.sparse.csgraph as csg
    L22 = L[order][:, order].tocsr()
    ncomp, lab = csg.connected_components(L22 != 0, directed=False)
    out = []
    for c in range(ncomp):
        idx = np.nonzero(lab == c)[0]
        sub = L22[idx][:, idx].tocoo()
        n = len(idx)
        d = np.abs(sub.row - sub.col)
        out.append((n, int(np.minimum(d, n - d).max()) if n > 1 else 0, idx.max() - idx.min() + 1 == n))
    return out


@pytest.mark.parametrize("mk,sizes", [(W.star, (64, 128, 256)), (W.disk_minus, (128,)), (W.three_ellipses, (128,))])
def test_alg3_cyclic_bandwidth_of_assembled_L22(mk, sizes):
    """Sec. 4.2, Alg. 3: with the irregular cells numbered along the boundary, L22 is cyclic
    banded with a bandwidth that does not grow with 1/h.  Measured on the assembled L22 of
    the oracle's operator, in the oracle's Alg. 3 order and in the product's row order (the
    order its SMO-2 blocks follow): one diagonal block per boundary component, each contiguous
    in the order, with a cyclic bandwidth of at most 26 (the paper's stencils give at most 20,
    ours reach up to 26 with their radius-3 lattices), flat in h."""
    P = pytest.importorskip("paper_2504_00724_gb300")
    claims = _paper_claims()
    assert claims["cyclic_bandwidth"] == 20
    per_size = []
    for n in sizes:
        prob = mk(n)
        cg = G.cut_cells(prob)
        dz = D.discretize(cg, prob.a, prob.b, prob.c)
        lvl = MG.Level(prob, cg, dz, prob.h, n, n, (cg.status != 0).ravel(), dz.regular.ravel(),
                       dz.irregular.ravel(), 0.0, None, None)
        o = MG.alg3_order(lvl)
        hs = P.HostSetup(prob)
        try:
            cells = hs.rows(0)[0].astype(np.int64)
        finally:
            hs.close()
        L = dz.L.tocsr()
        ncomp = 1 + len(prob.curves) if prob.box_bc != W.NONE else len(prob.curves)
        for order in (o, cells):
            assert sorted(order.tolist()) == sorted(np.nonzero(lvl.irr)[0].tolist())
            comps = _component_bandwidths(L, order)
            assert len(comps) == ncomp
            assert all(contiguous for _, _, contiguous in comps)
            assert max(bw for _, bw, _ in comps) <= 26
        per_size.append(max(bw for _, bw, _ in _component_bandwidths(L, cells)))
    assert per_size[-1] <= per_size[0] + 3


def _paper_claims():
    import os
    claims = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_conditioning.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, val = line.split()
            claims[key] = float(val)
    return claims


def test_fmg_iterations_converge_to_direct_solution(star64):
    """FMG cycles iterated on the residual equation reach the direct solution."""
    prob, H, r = star64
    hist = []
    u = MG.fmg_solve(H, r, rtol=1e-12, max_iter=40, history=hist)
    assert hist[-1] <= 1e-12
    ud = MG.direct_solve(H.levels[0].dz, r)
    ne = H.levels[0].ne
    assert np.abs(u - ud)[ne].max() <= 1e-9 * np.abs(ud[ne]).max()


def test_fmg_cycle_is_one_vcycle_per_level_from_the_prolonged_coarse_solution(star64):
    """The FMG cycle written out: restricted right-hand sides, bottom solve, then per level a
    V-cycle whose initial guess is the prolonged coarse result."""
    prob, H, r = star64
    M = len(H.levels) - 1
    rs = [r]
    for m in range(M):
        rs.append(MG.restrict(H.levels[m], H.levels[m + 1], rs[m]))
    want = MG.bottom(H, rs[M])
    for m in range(M - 1, -1, -1):
        guess = MG.prolong(H.levels[m], H.levels[m + 1], want)
        want = MG.vcycle(H, m, guess, rs[m])
    got = MG.fmg(H, r)
    assert np.array_equal(got, want)
    # and it is a better start than the zero guess a V-cycle would take
    lv = H.levels[0]
    v = MG.vcycle(H, 0, np.zeros_like(r), r)
    assert MG.rel_residual(lv, got, r) < MG.rel_residual(lv, v, r)


def test_fmg_reduction_matches_paper_problem2():
    """Sec. 5.2, Fig. fig:reduction: on Problem 2 at h = 1/128 with omega = 0.5 and
    nu1 = nu2 = 3, from the zero guess, the relative residual falls by a factor 11.3 per FMG
    cycle before it stagnates.  Geometric mean of the reduction over the first 8 cycles,
    within a factor 2 of the printed value (the readings of the transfers differ in detail)."""
    paper = _paper_claims()["fmg_reduction"]
    prob, mms = W.paper_problem2(128), W.mms_sinsin()
    H = MG.build_hierarchy(prob)
    lv = H.levels[0]
    fa = Q.cell_averages(lv.cg, mms.f(prob.a, prob.b, prob.c))
    ga = Q.boundary_averages(lv.cg, lv.dz.segs, mms.u, mms.ux, mms.uy)
    r = fa.ravel() - lv.dz.N @ ga
    hist = []
    MG.fmg_solve(H, r, rtol=0.0, max_iter=8, omega=0.5, nu1=3, nu2=3, history=hist)
    factor = (hist[0] / hist[8]) ** (1.0 / 8.0)
    assert paper / 2 <= factor <= paper * 2, factor
