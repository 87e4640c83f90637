"""The setup's work on the GPU (ccm_params.setup_device = 1: the centre classification of every
cell, one thread per cell, and the PLG fits, one warp per candidate stencil) against the host
setup (the cell maps of every level equal, and the host fits (the host-only setup, which tests/test_host_setup.py ties to
the oracle): the same stencils on every level, coefficients equal to rounding (1e-9 of the
row's largest coefficient, the bound the host setup meets against the oracle: the
ill-conditioned sample matrices of coarse levels amplify the different summation order; the
flower's 10^2 level differs by up to 4e-10), the same condition-number diagnostic, and
solves that agree to the solver tolerance."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2504_00724_gb300")

pytestmark = pytest.mark.gpu

CASES = {
    "star128": lambda: W.star(128),
    "ellipses128_neumann": lambda: W.three_ellipses(128),
    "robin64_cross": lambda: W.disk_robin(64, (1.0, 2.0), abc=(1.0, 0.5, 2.0)),
    "problem1_flower80": lambda: W.paper_problem1(80),
    "problem2_ellipse64_neumann": lambda: W.paper_problem2(64, W.NEUMANN),
    "problem3_rotated_box64": lambda: W.paper_problem3_rotated(64),
    "spline128": lambda: W.spline_blob(128),
}


@pytest.mark.parametrize("name", list(CASES))
def test_device_fits_equal_host_fits(name):
    prob = CASES[name]()
    hs = P.HostSetup(prob)
    s = P.Solver(prob, setup_device=1)
    try:
        levels = int(s.info.levels)
        dev_map, host_map = s.cell_map(), hs.cell_map(0)
        for d, h in zip(dev_map, host_map[:4]):
            assert np.array_equal(d, h)
        for m in range(levels):
            cell, cols, beta, nb, seg = s.level_rows(m)
            hc, hcols, hbeta, hnb, hseg = hs.rows(m)
            assert np.array_equal(cell, hc), m
            assert np.array_equal(cols, hcols), m           # the same PLG stencil of every row
            assert np.array_equal(seg, hseg), m
            scale = np.abs(hbeta).max(axis=1)
            assert np.all(np.abs(beta - hbeta).max(axis=1) <= 1e-9 * scale), m
            assert np.all(np.abs(nb - hnb) <= 1e-9 * scale), m
    finally:
        s.close()


def test_device_and_host_setup_solve_alike():
    prob, mms = W.star(256), W.mms_star()
    out = []
    for dev in (1, 0):
        s = P.Solver(prob, setup_device=dev, precision=P.CCM_FP64, rtol=1e-12, max_iter=200)
        try:
            q = s.quadrature()
            f = torch.tensor(s.cell_averages(mms.f(prob.a, prob.b, prob.c), quad=q), device="cuda")
            g = torch.tensor(s.boundary_averages(mms.u, mms.ux, mms.uy, quad=q), device="cuda")
            u, st = s.solve(f, g)
            assert st.rel_residual <= 1e-12
            out.append((u.cpu().numpy(), float(s.info.plg_cond_max)))
        finally:
            s.close()
    (u1, c1), (u0, c0) = out
    assert np.abs(u1 - u0).max() <= 1e-10 * np.abs(u0).max()
    assert abs(c1 - c0) <= 1e-6 * c0


@pytest.mark.parametrize("mk", [lambda: W.star(1024), lambda: W.three_ellipses(1024), lambda: W.spline_blob(512),
                                lambda: W.paper_problem3_rotated(256)])
def test_device_centre_classification_large(mk):
    """The O(h^-2) scan at sizes where it matters: every level's cells (status, owner, regular
    flag, volume) equal between the device setup and the host setup (every level's fitted rows
    too, as a consequence)."""
    prob = mk()
    hs = P.HostSetup(prob, coarsest=64)
    s = P.Solver(prob, setup_device=1, coarsest=64)
    try:
        dev_map, host_map = s.cell_map(), hs.cell_map(0)
        for d, h in zip(dev_map, host_map[:4]):
            assert np.array_equal(d, h)
        for m in range(int(s.info.levels)):
            assert np.array_equal(s.level_rows(m)[0], hs.rows(m)[0]), m
            assert np.array_equal(s.level_rows(m)[1], hs.rows(m)[1]), m
    finally:
        s.close()
        hs.close()
