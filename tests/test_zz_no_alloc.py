"""The allocation-free operator application (ccm_apply_noalloc), called through the C ABI.

Callers that must not allocate device memory at call time (a framework whose caching
allocator owns the device, or a loop that cannot afford cudaMalloc's device synchronisation)
use this entry point: its scratch is a fixed device array inside the library.  Its result must equal ccm_apply's, also on the
second of two calls in a row (the scratch keeps the previous call's contents), and grids
beyond the fixed scratch must be refused cleanly."""
import ctypes

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2504_00724_gb300")

pytestmark = pytest.mark.gpu


def _field(st, seed):
    rng = np.random.default_rng(seed)
    return np.where(st != 0, rng.standard_normal(st.shape), 0.0)


def _noalloc(solver, u, g, out):
    stream = torch.cuda.current_stream().cuda_stream
    return P.lib().ccm_apply_noalloc(solver.h, ctypes.c_void_p(u.data_ptr()),
                                     ctypes.c_void_p(g.data_ptr()) if g is not None else None,
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


@pytest.mark.parametrize("mk", [lambda: W.star(128), lambda: W.disk_minus(64)])
def test_noalloc_apply_matches_apply_twice(mk):
    prob = mk()
    s = P.Solver(prob)
    try:
        st = s.cell_map()[0]
        for call, seed in enumerate((11, 12)):
            u = torch.tensor(_field(st, seed), dtype=torch.float64, device="cuda")
            g = None
            if call == 0:
                g = torch.tensor(np.random.default_rng(seed + 100).standard_normal(s.nseg),
                                 dtype=torch.float64, device="cuda")
            ref = s.apply(u, g)
            out = torch.full_like(u, float("nan"))
            rc = _noalloc(s, u, g, out)
            assert rc == 0, P.lib().ccm_strerror(rc)
            torch.cuda.synchronize()
            a, b = out.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(a))
            assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()
    finally:
        s.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    s = P.Solver(W.star(1024))
    try:
        u = torch.zeros((1024, 1024), dtype=torch.float64, device="cuda")
        out = torch.full_like(u, 7.0)
        assert _noalloc(s, u, None, out) == -10     # CCM_ETOOLARGE, nothing queued
        torch.cuda.synchronize()
        assert bool((out == 7.0).all())             # out untouched
    finally:
        s.close()
