"""ccm_solve_host: the solve with host buffers (pinned: read and written by the kernels over the
host link; pageable: the device's own access or staging copies) gives the device-buffer
solve's result bit for bit on the non-empty cells, for one and for several right-hand sides,
and leaves the cells outside the domain as the caller's buffer held them."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2504_00724_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    prob, mms = W.star(256), W.mms_star()
    s = P.Solver(prob, rtol=1e-10)
    q = s.quadrature()
    fa = s.cell_averages(mms.f(prob.a, prob.b, prob.c), quad=q)
    ga = s.boundary_averages(mms.u, mms.ux, mms.uy, quad=q)
    yield s, fa, ga
    s.close()


def test_pinned_host_buffers_equal_device_buffers(setup):
    s, fa, ga = setup
    u_dev, st_dev = s.solve(torch.tensor(fa, device="cuda"), torch.tensor(ga, device="cuda"))
    fh = torch.tensor(fa).pin_memory()
    gh = torch.tensor(ga).pin_memory()
    uh = torch.zeros_like(fh).pin_memory()
    u_host, st = s.solve_host(fh, gh, uh)
    assert u_host.data_ptr() == uh.data_ptr()
    assert st.iterations == st_dev.iterations and st.rel_residual == st_dev.rel_residual
    assert torch.equal(uh, u_dev.cpu())


def test_pageable_host_buffers_and_several_rhs(setup):
    s, fa, ga = setup
    rng = np.random.default_rng(5)
    F = np.stack([fa, fa * 0.5 + rng.standard_normal(fa.shape) * (s.cell_map()[0] != 0)])
    G = np.stack([ga, ga * 0.5])
    u_dev, _ = s.solve(torch.tensor(F, device="cuda"), torch.tensor(G, device="cuda"))
    U = np.zeros_like(F)
    s.solve_host(F, G, U)                        # numpy arrays: pageable memory
    assert np.array_equal(U, u_dev.cpu().numpy())


def test_host_solve_keeps_cells_outside_the_domain(setup):
    """Only the non-empty cells cross the host link back: the cells outside the domain keep
    whatever the caller's buffer held there, the non-empty cells hold the device solve's
    solution bit for bit (pinned and pageable buffers)."""
    s, fa, ga = setup
    ne = s.cell_map()[0] != 0
    assert (~ne).any()
    u_dev, _ = s.solve(torch.tensor(fa, device="cuda"), torch.tensor(ga, device="cuda"))
    ud = u_dev.cpu().numpy()
    fh = torch.tensor(fa).pin_memory()
    gh = torch.tensor(ga).pin_memory()
    uh = torch.full(fh.shape, 7.0, dtype=torch.float64).pin_memory()
    uh[torch.from_numpy(ne)] = 0.0
    s.solve_host(fh, gh, uh)
    assert np.all(uh.numpy()[~ne] == 7.0)
    assert np.array_equal(uh.numpy()[ne], ud[ne])
    U = np.where(ne, 0.0, -3.0)
    s.solve_host(np.array(fa), np.array(ga), U)
    assert np.all(U[~ne] == -3.0)
    assert np.array_equal(U[ne], ud[ne])
