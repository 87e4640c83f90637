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


def test_alg3_cyclic_bandwidth_small_and_flat():
    """Sec. 4.2: the cyclic bandwidth of L22 in the Alg. 3 order does not grow with 1/h
    (the paper reports <= 20 with its stencils; ours reach a few more)."""
    bws = []
    for n in (64, 128, 256):
        prob = W.star(n)
        cg = G.cut_cells(prob)
        lvl = MG.Level(prob, cg, None, prob.h, n, n, (cg.status != 0).ravel(), None, None, 0.0, None, None)
        reg = D.regular_mask(cg) & (cg.status != 0)
        lvl.irr = ((cg.status != 0) & ~reg).ravel()
        o = MG.alg3_order(lvl)
        assert len(o) == int(lvl.irr.sum()) and len(set(o.tolist())) == len(o)
        # bandwidth of the coupling pattern: PLG stencils lie within the Chebyshev ball
        # of radius 3 for these cells, so use that pattern (no fit needed)
        pos = -np.ones(n * n, dtype=np.int64)
        pos[o] = np.arange(len(o))
        N = len(o)
        bw = 0
        for q in o:
            j, i = divmod(int(q), n)
            for dj in range(-3, 4):
                for di in range(-3, 4):
                    ii, jj = i + di, j + dj
                    if 0 <= ii < n and 0 <= jj < n and pos[jj * n + ii] >= 0:
                        d = abs(pos[q] - pos[jj * n + ii])
                        bw = max(bw, min(d, N - d))
        bws.append(bw)
    assert max(bws) <= 60
    assert bws[-1] <= bws[0] + 8
