"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Tolerances: the two codes build their operators independently; their coefficients agree to
about 1e-11 relative (rounding of independent fits), so operator applications are compared
per row against the row's own magnitude sum |L_ij| |u_j| with a 1e-10 factor.  Solutions
solved to a 1e-12 residual are compared at 1e-10 relative to max |u| (FP64), and the mixed
form's discretisation error against the exact solution must equal the FP64 form's to two
significant digits."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import cubature as Q
from oracle import discretization as D
from oracle import geometry as G
from oracle import multigrid as MG

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2504_00724_gb300")

pytestmark = pytest.mark.gpu

CASES = {
    "star64": (lambda: W.star(64), W.mms_star),
    "disk32": (lambda: W.disk_minus(32), W.mms_disk),
    "ellipses64": (lambda: W.three_ellipses(64), W.mms_ellipses),
    "robin32": (lambda: W.disk_robin(32, (1.0, 0.5)), W.mms_disk),
    "robin_cross64": (lambda: W.disk_robin(64, (1.0, 2.0), abc=(1.0, 0.5, 2.0)), W.mms_disk),
    "spline64": (lambda: W.spline_blob(64), W.mms_star),
    "rotated_box64": (lambda: W.paper_problem3_rotated(64), W.mms_problem3_rotated),
}
OMEGA = 0.8


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    mk, mms = CASES[request.param]
    prob = mk()
    H = MG.build_hierarchy(prob)
    solver = P.Solver(prob, omega=OMEGA, rtol=1e-12, precision=P.CCM_FP64, max_iter=200)
    yield prob, mms(), H, solver
    solver.close()


def rand_field(lv, seed):
    rng = np.random.default_rng(seed)
    return np.where(lv.ne, rng.standard_normal(lv.nx * lv.ny), 0.0).reshape(lv.ny, lv.nx)


def test_apply_matches_oracle(case):
    prob, mms, H, s = case
    lv = H.levels[0]
    u = rand_field(lv, 1)
    g = np.random.default_rng(2).standard_normal(len(lv.dz.segs))
    out = host(s.apply(cuda(u), cuda(g)))
    want = (lv.dz.L @ u.ravel() + lv.dz.N @ g).reshape(lv.ny, lv.nx)
    scale = (abs(lv.dz.L) @ np.abs(u.ravel()) + abs(lv.dz.N) @ np.abs(g)).reshape(lv.ny, lv.nx)
    assert np.all(np.abs(out - want) <= 1e-10 * scale + 1e-300)
    assert np.all(out[~lv.ne.reshape(lv.ny, lv.nx)] == 0.0)


def test_apply_transposed_matches_oracle(case):
    prob, mms, H, s = case
    lv = H.levels[0]
    v = rand_field(lv, 3)
    ou, og = s.apply_T(cuda(v))
    ou, og = host(ou), host(og)
    want_u = (lv.dz.L.T @ v.ravel()).reshape(lv.ny, lv.nx)
    want_g = lv.dz.N.T @ v.ravel()
    scale = (abs(lv.dz.L).T @ np.abs(v.ravel())).reshape(lv.ny, lv.nx)
    ne = lv.ne.reshape(lv.ny, lv.nx)
    assert np.all(np.abs(ou - want_u)[ne] <= 1e-10 * scale[ne] + 1e-300)
    assert np.abs(og - want_g).max() <= 1e-10 * (abs(lv.dz.N).T @ np.abs(v.ravel())).max()
    # dot-product identity of the device pair: <L u, v> = <u, L^T v>
    u = rand_field(lv, 4)
    Lu = host(s.apply(cuda(u)))
    lhs, rhs = float((Lu * v).sum()), float((u * ou).sum())
    assert abs(lhs - rhs) <= 1e-11 * (np.abs(Lu * v).sum())


def test_level_apply_every_level(case):
    prob, mms, H, s = case
    for m, lv in enumerate(H.levels):
        u = rand_field(lv, 10 + m)
        out = host(s.level_apply(m, cuda(u)))
        want = (lv.dz.L @ u.ravel()).reshape(lv.ny, lv.nx)
        scale = (abs(lv.dz.L) @ np.abs(u.ravel())).reshape(lv.ny, lv.nx)
        assert np.all(np.abs(out - want) <= 1e-10 * scale + 1e-300), m


def test_smoother_step_matches_oracle(case):
    """SMO-1 + SMO-2; with enough passes the block solve is the exact L22 solve."""
    prob, mms, H, _ = case
    s = P.Solver(prob, omega=OMEGA, ras_passes=40, smoother=0, ras_exact=1024)
    try:
        for m in range(len(H.levels) - 1):
            lv = H.levels[m]
            u0 = rand_field(lv, 20 + m)
            r = rand_field(lv, 30 + m) / lv.h ** 2
            want = u0.ravel().copy()
            MG.smo1(lv, want, r.ravel(), OMEGA)
            MG.smo2(lv, want, r.ravel())
            got = host(s.level_smooth(m, cuda(u0), cuda(r), P.CCM_FP64)).ravel()
            assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max(), m
            got32 = host(s.level_smooth(m, cuda(u0), cuda(r), P.CCM_MIXED)).ravel()
            assert np.abs(got32 - want).max() <= 2e-4 * np.abs(want).max(), m
    finally:
        s.close()


def test_default_smoother_step(case):
    """The default smoother step (block-Jacobi form: SMO-1 and one pass of the overlapping
    block solve, both from the old iterate).  Regular cells equal the oracle's SMO-1 of the old
    iterate; on the irregular cells the step removes most of the residual of the SMO-2
    equation L22 u2 = r2 - L21 u1_old (one pass of the block solve is not exact)."""
    prob, mms, H, s = case
    lv = H.levels[0]
    u0 = rand_field(lv, 40).ravel()
    r = (rand_field(lv, 41) / lv.h ** 2).ravel()
    s1 = P.Solver(prob, omega=OMEGA)
    try:
        got = host(s1.level_smooth(0, cuda(u0.reshape(lv.ny, lv.nx)), cuda(r.reshape(lv.ny, lv.nx)),
                                   P.CCM_FP64)).ravel()
    finally:
        s1.close()
    ref = u0.copy()
    MG.smo1(lv, ref, r, OMEGA)
    assert np.abs(got - ref)[lv.reg].max() <= 1e-10 * np.abs(ref).max()
    L22 = lv.dz.L[lv.irr_idx][:, lv.irr_idx]
    rhs = r[lv.irr_idx] - lv.L21 @ u0[lv.reg_idx]
    before = np.linalg.norm(rhs - L22 @ u0[lv.irr_idx])
    after = np.linalg.norm(rhs - L22 @ got[lv.irr_idx])
    assert after <= 0.1 * before


def test_restrict_prolong_bottom(case):
    prob, mms, H, s = case
    for m in range(len(H.levels) - 1):
        f, c = H.levels[m], H.levels[m + 1]
        u = rand_field(f, 50 + m)
        r = rand_field(f, 60 + m) / f.h ** 2
        got = host(s.level_restrict(m, cuda(u), cuda(r))).ravel()
        want = MG.restrict(f, c, MG.residual(f, u.ravel(), r.ravel()))
        # the residual cancels: scale by the restriction of |r| + |L| |u|
        scale = MG.restrict(f, c, np.abs(r.ravel()) + abs(f.dz.L) @ np.abs(u.ravel()))
        assert np.all(np.abs(got - want) <= 1e-10 * scale + 1e-300), m
        uc = rand_field(c, 70 + m)
        got = host(s.level_prolong(m, cuda(uc), cuda(u))).ravel()
        want = u.ravel() + MG.prolong(f, c, uc.ravel())
        assert np.abs(got - want).max() <= 1e-14 * np.abs(want).max(), m
    last = H.levels[-1]
    r = rand_field(last, 80) / last.h ** 2
    got = host(s.bottom_solve(cuda(r))).ravel()
    want = MG.bottom(H, r.ravel())
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


def test_vcycle_matches_oracle(case):
    """One V-cycle (Alg. 2) with exact SMO-2 equals the oracle's V-cycle."""
    prob, mms, H, _ = case
    s = P.Solver(prob, omega=OMEGA, ras_passes=40, smoother=0, ras_exact=1024)
    try:
        lv = H.levels[0]
        u0 = rand_field(lv, 90)
        r = rand_field(lv, 91) / lv.h ** 2
        want = MG.vcycle(H, 0, u0.ravel().copy(), r.ravel(), omega=OMEGA, nu1=3, nu2=3)
        got = host(s.vcycle(cuda(u0), cuda(r), P.CCM_FP64)).ravel()
        assert np.abs(got - want).max() <= 1e-8 * np.abs(want).max()
    finally:
        s.close()


def _rhs(prob, mms, lv):
    fa = Q.cell_averages(lv.cg, mms.f(prob.a, prob.b, prob.c))
    ga = Q.boundary_averages(lv.cg, lv.dz.segs, mms.u, mms.ux, mms.uy)
    return fa, ga


def test_fp64_solve_matches_oracle_solution(case):
    prob, mms, H, s = case
    lv = H.levels[0]
    fa, ga = _rhs(prob, mms, lv)
    u, st = s.solve(cuda(fa), cuda(ga))
    u = host(u)
    assert st.rel_residual <= 1e-12
    want = MG.direct_solve(lv.dz, fa.ravel() - lv.dz.N @ ga).reshape(lv.ny, lv.nx)
    assert np.abs(u - want).max() <= 1e-10 * np.abs(want).max()


def test_mixed_solve_same_discretisation_error(case):
    prob, mms, H, s64 = case
    lv = H.levels[0]
    fa, ga = _rhs(prob, mms, lv)
    ua = Q.cell_averages(lv.cg, mms.u)
    ne = lv.ne.reshape(lv.ny, lv.nx)
    u64, st64 = s64.solve(cuda(fa), cuda(ga))
    sm = P.Solver(prob, omega=OMEGA, rtol=1e-12, precision=P.CCM_MIXED, max_iter=200)
    try:
        um, stm = sm.solve(cuda(fa), cuda(ga))
    finally:
        sm.close()
    assert stm.rel_residual <= 1e-12
    e64 = np.abs(host(u64) - ua)[ne].max()
    em = np.abs(host(um) - ua)[ne].max()
    assert float(f"{e64:.1e}") == float(f"{em:.1e}")
    want = MG.direct_solve(lv.dz, fa.ravel() - lv.dz.N @ ga).reshape(lv.ny, lv.nx)
    assert np.abs(host(um) - want).max() <= 1e-10 * np.abs(want).max()


def test_library_quadrature_matches_oracle_cubature(case):
    prob, mms, H, s = case
    lv = H.levels[0]
    fa, ga = _rhs(prob, mms, lv)
    f = mms.f(prob.a, prob.b, prob.c)
    fl = s.cell_averages(f)
    gl = s.boundary_averages(mms.u, mms.ux, mms.uy)
    assert np.abs(fl - fa).max() <= 1e-12 * np.abs(fa).max()
    assert np.abs(gl - ga).max() <= 1e-12 * max(1.0, np.abs(ga).max())
