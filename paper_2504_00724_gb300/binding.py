"""ctypes marshalling for libccm.so (include/ccm.h).  No arithmetic of the method here."""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libccm.so")

CCM_CIRCLE, CCM_ELLIPSE, CCM_STAR, CCM_POLYGON, CCM_SPLINE = 1, 2, 3, 4, 5
CCM_NONE, CCM_DIRICHLET, CCM_NEUMANN, CCM_ROBIN = 0, 1, 2, 3
CCM_FP64, CCM_MIXED = 0, 1
CCM_PROF_OFF, CCM_PROF_RESID_FP64, CCM_PROF_SMO1_FP32, CCM_PROF_SMO1_FP64, CCM_PROF_VCYCLE = 0, 1, 2, 3, 4
CCM_PROF_SMO2_FP32, CCM_PROF_PROLONG_SMO1_FP32, CCM_PROF_RESTRICT_FP32 = 5, 6, 7


class CcmError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {lib().ccm_strerror(code).decode()} ({code})")


class ccm_curve(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("p", ctypes.c_double * 8), ("orient", ctypes.c_int),
                ("bc", ctypes.c_int), ("robin", ctypes.c_double * 2), ("npts", ctypes.c_int),
                ("pts", ctypes.POINTER(ctypes.c_double))]


class ccm_problem(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("h", ctypes.c_double),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("box_bc", ctypes.c_int),
                ("ncurves", ctypes.c_int), ("curves", ctypes.POINTER(ccm_curve))]


class ccm_params(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("theta", ctypes.c_double), ("coarsest", ctypes.c_int), ("precision", ctypes.c_int),
                ("rtol", ctypes.c_double), ("max_iter", ctypes.c_int), ("ras_passes", ctypes.c_int),
                ("ras_block", ctypes.c_int), ("ras_overlap", ctypes.c_int), ("nthreads", ctypes.c_int),
                ("ras_exact", ctypes.c_int), ("inner_cycles", ctypes.c_int), ("smoother", ctypes.c_int),
                ("coarse_n", ctypes.c_int), ("batch", ctypes.c_int),
                ("cycle", ctypes.c_int), ("setup_device", ctypes.c_int), ("krylov", ctypes.c_int)]


class ccm_info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("levels", ctypes.c_int),
                ("n_cells", ctypes.c_int64), ("n_regular", ctypes.c_int64),
                ("n_irregular", ctypes.c_int64), ("n_segments", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("setup_ms", ctypes.c_double),
                ("plg_cond_max", ctypes.c_double), ("batch", ctypes.c_int),
                ("setup_geometry_ms", ctypes.c_double), ("setup_fits_ms", ctypes.c_double),
                ("setup_blocks_ms", ctypes.c_double), ("setup_bottom_ms", ctypes.c_double),
                ("setup_upload_ms", ctypes.c_double)]


class ccm_launch_info(ctypes.Structure):
    _fields_ = [("sweep_items", ctypes.c_int), ("sweep_blocks", ctypes.c_int), ("sweep_ctas", ctypes.c_int),
                ("restrict_items", ctypes.c_int), ("restrict_ctas", ctypes.c_int),
                ("block_inv_entries", ctypes.c_int64)]


class ccm_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("history", ctypes.c_double * 64)]


_LIB = None

DP = ctypes.POINTER(ctypes.c_double)
FIELD_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int64, DP, DP, DP)
GRAD_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int64, DP, DP, DP, DP, DP)

P = ctypes.c_void_p
I = ctypes.c_int
I64P = ctypes.POINTER(ctypes.c_int64)

_SIGS = {
    "ccm_default_params": (I, [ctypes.POINTER(ccm_params)]),
    "ccm_setup": (I, [ctypes.POINTER(ccm_problem), ctypes.POINTER(ccm_params), ctypes.POINTER(P)]),
    "ccm_query": (I, [P, ctypes.POINTER(ccm_info)]),
    "ccm_cell_map": (I, [P, P, P, P, P]),
    "ccm_boundary_segments": (I, [P, P, P, P]),
    "ccm_boundary_robin": (I, [P, P]),
    "ccm_level_rows": (I, [P, I, I64P, P, P, P, P, P]),
    "ccm_quadrature": (I, [P, I64P, I64P, P, P, P, P, P, P, P]),
    "ccm_cell_averages": (I, [P, FIELD_FN, P, P]),
    "ccm_boundary_averages": (I, [P, GRAD_FN, P, P]),
    "ccm_apply": (I, [P, P, P, P, I, P]),
    "ccm_apply_T": (I, [P, P, P, P, I, P]),
    "ccm_solve": (I, [P, P, P, P, I, P, ctypes.POINTER(ccm_stats)]),
    "ccm_solve_host": (I, [P, P, P, P, I, P, ctypes.POINTER(ccm_stats)]),
    "ccm_solve_T": (I, [P, P, P, I, P, ctypes.POINTER(ccm_stats)]),
    "ccm_level_apply": (I, [P, I, P, P, P]),
    "ccm_level_smooth": (I, [P, I, P, P, I, P]),
    "ccm_level_restrict": (I, [P, I, P, P, P, P]),
    "ccm_level_prolong": (I, [P, I, P, P, P]),
    "ccm_level_prolong_smooth": (I, [P, I, P, P, P, I, P]),
    "ccm_bottom_solve": (I, [P, P, P, P]),
    "ccm_vcycle": (I, [P, P, P, I, P]),
    "ccm_fmg": (I, [P, P, P, I, P]),
    "ccm_set_cycle_params": (I, [P, ctypes.c_double, I, I, I, I]),
    "ccm_set_launch_cap": (I, [P, I]),
    "ccm_set_smo2_blocks": (I, [P, I, I]),
    "ccm_level_launch": (I, [P, I, I, I, ctypes.POINTER(ccm_launch_info)]),
    "ccm_free": (None, [P]),
    "ccm_strerror": (ctypes.c_char_p, [I]),
    "ccm_host_build": (I, [ctypes.POINTER(ccm_problem), ctypes.POINTER(ccm_params), ctypes.POINTER(P)]),
    "ccm_host_level_sizes": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I), I64P, I64P]),
    "ccm_host_rows": (I, [P, I, P, P, P, P, P]),
    "ccm_host_cell_map": (I, [P, I, P, P, P, P, P]),
    "ccm_host_free": (None, [P]),
    "ccm_launch_count": (ctypes.c_int64, []),
    "ccm_apply_noalloc": (I, [P, P, P, P, P]),
    "ccm_profile": (I, [P, I]),
    "ccm_wait_selftest": (I, [P, P]),
    "ccm_profile_read": (I, [P, ctypes.POINTER(ctypes.c_double), I64P]),
    "ccm_group_create": (I, [P, I, P, ctypes.POINTER(P)]),
    "ccm_group_solve": (I, [P, P, P, P, P, ctypes.POINTER(ccm_stats)]),
    "ccm_group_query": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
    "ccm_group_free": (None, [P]),
}


def load_library(path: str = LIBPATH) -> ctypes.CDLL:
    """Load libccm.so and declare every entry point of include/ccm.h; raises if absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise ImportError(f"libccm.so not built ({path}); run paper_2504_00724_gb300/build.py")
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


def lib() -> ctypes.CDLL:
    return load_library()


def launch_count() -> int:
    """Kernels launched by libccm.so in this process so far."""
    return int(lib().ccm_launch_count())


def _check(rc: int, what: str):
    if rc != 0:
        raise CcmError(rc, what)


def default_params(**kw) -> ccm_params:
    p = ccm_params()
    _check(lib().ccm_default_params(ctypes.byref(p)), "ccm_default_params")
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def problem_struct(prob) -> tuple:
    """ccm_problem from a workloads.Problem-like object (keeps the curve array alive)."""
    n = len(prob.curves)
    arr = (ccm_curve * max(1, n))()
    keep = [arr]
    for k, c in enumerate(prob.curves):
        arr[k].kind = int(c.kind)
        if int(c.kind) in (CCM_POLYGON, CCM_SPLINE):
            pts = (ctypes.c_double * len(c.params))(*[float(v) for v in c.params])
            keep.append(pts)
            arr[k].npts = len(c.params) // 2
            arr[k].pts = ctypes.cast(pts, ctypes.POINTER(ctypes.c_double))
        else:
            for m, v in enumerate(c.params):
                arr[k].p[m] = float(v)
        arr[k].orient = int(c.orient)
        arr[k].bc = int(c.bc)
        g = getattr(c, "robin", (1.0, 0.0))
        arr[k].robin[0], arr[k].robin[1] = float(g[0]), float(g[1])
    s = ccm_problem(float(prob.a), float(prob.b), float(prob.c), float(prob.x0), float(prob.y0),
                    float(prob.h), int(prob.nx), int(prob.ny), int(prob.box_bc), n, arr)
    return s, keep


def _ptr(t) -> int:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Solver:
    """A set-up problem on the current CUDA device (one handle of the C ABI)."""

    def __init__(self, prob, **params):
        self.prob = prob
        self._ps, self._curves = problem_struct(prob)
        self.params = default_params(**params)
        h = P()
        _check(lib().ccm_setup(ctypes.byref(self._ps), ctypes.byref(self.params), ctypes.byref(h)), "ccm_setup")
        self.h = h
        self.info = ccm_info()
        _check(lib().ccm_query(self.h, ctypes.byref(self.info)), "ccm_query")
        self.nx, self.ny = prob.nx, prob.ny
        self.nseg = int(self.info.n_segments)

    def close(self):
        if getattr(self, "h", None):
            lib().ccm_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- host queries
    def cell_map(self):
        n = self.nx * self.ny
        st = np.zeros(n, np.int8)
        ow = np.zeros(n, np.int32)
        rg = np.zeros(n, np.int8)
        vol = np.zeros(n, np.float64)
        _check(lib().ccm_cell_map(self.h, st.ctypes.data, ow.ctypes.data, rg.ctypes.data, vol.ctypes.data),
               "ccm_cell_map")
        sh = (self.ny, self.nx)
        return st.reshape(sh), ow.reshape(sh), rg.reshape(sh), vol.reshape(sh)

    def boundary_segments(self):
        cell = np.zeros(self.nseg, np.int32)
        bc = np.zeros(self.nseg, np.int32)
        ln = np.zeros(self.nseg, np.float64)
        _check(lib().ccm_boundary_segments(self.h, cell.ctypes.data, bc.ctypes.data, ln.ctypes.data),
               "ccm_boundary_segments")
        return cell, bc, ln

    def level_rows(self, level=0):
        """Fitted rows of a level: (cell, cols[n,15], beta[n,15], nb, seg), physical units."""
        n = ctypes.c_int64(0)
        _check(lib().ccm_level_rows(self.h, level, ctypes.byref(n), None, None, None, None, None), "ccm_level_rows")
        n2 = n.value
        cell = np.zeros(n2, np.int32)
        cols = np.zeros((n2, 15), np.int32)
        beta = np.zeros((n2, 15))
        nb = np.zeros(n2)
        seg = np.zeros(n2, np.int32)
        _check(lib().ccm_level_rows(self.h, level, None, cell.ctypes.data, cols.ctypes.data, beta.ctypes.data,
                                    nb.ctypes.data, seg.ctypes.data), "ccm_level_rows")
        return cell, cols, beta, nb, seg

    def boundary_operator(self) -> np.ndarray:
        """(gamma1, gamma2) per segment [n_segments, 2]: the segment's boundary operator is
        gamma1 u + gamma2 du/dn."""
        gam = np.zeros((self.nseg, 2))
        _check(lib().ccm_boundary_robin(self.h, gam.ctypes.data), "ccm_boundary_robin")
        return gam

    def quadrature(self):
        nc, nb = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib().ccm_quadrature(self.h, ctypes.byref(nc), ctypes.byref(nb), None, None, None, None, None,
                                    None, None), "ccm_quadrature")
        n, m = nc.value, nb.value
        cell = np.zeros(n, np.int32)
        cxy = np.zeros((n, 2))
        cw = np.zeros(n)
        seg = np.zeros(m, np.int32)
        bxy = np.zeros((m, 2))
        bw = np.zeros(m)
        bn = np.zeros((m, 2))
        _check(lib().ccm_quadrature(self.h, ctypes.byref(nc), ctypes.byref(nb), cell.ctypes.data, cxy.ctypes.data,
                                    cw.ctypes.data, seg.ctypes.data, bxy.ctypes.data, bw.ctypes.data,
                                    bn.ctypes.data), "ccm_quadrature")
        return cell, cxy, cw, seg, bxy, bw, bn

    # ---- device operations (torch float64 CUDA tensors, C-contiguous)
    def apply(self, u, g=None, out=None, stream=None):
        import torch
        nrhs = u.numel() // (self.nx * self.ny)
        out = torch.empty_like(u) if out is None else out
        _check(lib().ccm_apply(self.h, _ptr(u), _ptr(g), _ptr(out), nrhs, _stream(stream)), "ccm_apply")
        return out

    def apply_T(self, v, stream=None, want_u=True, want_g=True):
        import torch
        nrhs = v.numel() // (self.nx * self.ny)
        ou = torch.empty_like(v) if want_u else None
        og = torch.empty(v.shape[:-2] + (self.nseg,), dtype=v.dtype, device=v.device) if want_g else None
        _check(lib().ccm_apply_T(self.h, _ptr(v), _ptr(ou), _ptr(og), nrhs, _stream(stream)), "ccm_apply_T")
        return ou, og

    def solve(self, f, g=None, u0=None, stream=None, check=True):
        import torch
        nrhs = f.numel() // (self.nx * self.ny)
        u = torch.zeros_like(f) if u0 is None else u0.clone()
        st = ccm_stats()
        rc = lib().ccm_solve(self.h, _ptr(f), _ptr(g), _ptr(u), nrhs, _stream(stream), ctypes.byref(st))
        if check:
            _check(rc, "ccm_solve")
        return u, st

    def solve_host(self, f, g=None, u=None, stream=None, check=True):
        """solve() with host arrays (CPU torch tensors, pinned for the direct path, or numpy
        float64 arrays); u, if given, is the initial guess and receives the solution in place.
        Returns (u, stats)."""
        import torch

        def ptr(a):
            if a is None:
                return None
            return a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data

        nrhs = (f.numel() if isinstance(f, torch.Tensor) else f.size) // (self.nx * self.ny)
        if u is None:
            u = torch.zeros(f.shape, dtype=torch.float64)
        st = ccm_stats()
        rc = lib().ccm_solve_host(self.h, ptr(f), ptr(g), ptr(u), nrhs, _stream(stream), ctypes.byref(st))
        if check:
            _check(rc, "ccm_solve_host")
        return u, st

    def solve_T(self, rhs, lam0=None, stream=None, check=True):
        """lambda with L^T lambda = rhs (adjoint solve)."""
        import torch
        nrhs = rhs.numel() // (self.nx * self.ny)
        lam = torch.zeros_like(rhs) if lam0 is None else lam0.clone()
        st = ccm_stats()
        rc = lib().ccm_solve_T(self.h, _ptr(rhs), _ptr(lam), nrhs, _stream(stream), ctypes.byref(st))
        if check:
            _check(rc, "ccm_solve_T")
        return lam, st

    def level_apply(self, level, u, stream=None):
        import torch
        out = torch.empty_like(u)
        _check(lib().ccm_level_apply(self.h, level, _ptr(u), _ptr(out), _stream(stream)), "ccm_level_apply")
        return out

    def level_smooth(self, level, u, r, precision=CCM_FP64, stream=None):
        u = u.clone()
        _check(lib().ccm_level_smooth(self.h, level, _ptr(u), _ptr(r), precision, _stream(stream)),
               "ccm_level_smooth")
        return u

    def level_restrict(self, level, u, r, stream=None):
        import torch
        nc, mc = self.nx >> (level + 1), self.ny >> (level + 1)
        rc = torch.zeros((mc, nc), dtype=u.dtype, device=u.device)
        _check(lib().ccm_level_restrict(self.h, level, _ptr(u), _ptr(r), _ptr(rc), _stream(stream)),
               "ccm_level_restrict")
        return rc

    def level_prolong(self, level, uc, u, stream=None):
        u = u.clone()
        _check(lib().ccm_level_prolong(self.h, level, _ptr(uc), _ptr(u), _stream(stream)), "ccm_level_prolong")
        return u

    def level_prolong_smooth(self, level, u, uc, r, precision=CCM_FP64, stream=None):
        """The first post-smoothing sweep with the prolongation fused: one sweep from u + P uc."""
        u = u.clone()
        _check(lib().ccm_level_prolong_smooth(self.h, level, _ptr(u), _ptr(uc), _ptr(r), precision, _stream(stream)),
               "ccm_level_prolong_smooth")
        return u

    def bottom_solve(self, r, stream=None):
        import torch
        u = torch.zeros_like(r)
        _check(lib().ccm_bottom_solve(self.h, _ptr(r), _ptr(u), _stream(stream)), "ccm_bottom_solve")
        return u

    def vcycle(self, u, r, precision=CCM_FP64, stream=None):
        u = u.clone()
        _check(lib().ccm_vcycle(self.h, _ptr(u), _ptr(r), precision, _stream(stream)), "ccm_vcycle")
        return u

    def set_cycle_params(self, omega=None, nu1=None, nu2=None, inner_cycles=None, cycle=None):
        """Change omega, nu1, nu2, inner_cycles, cycle without a new setup
        (ccm_set_cycle_params); unspecified ones keep their values."""
        p = self.params
        vals = [p.omega if omega is None else omega, p.nu1 if nu1 is None else nu1,
                p.nu2 if nu2 is None else nu2, p.inner_cycles if inner_cycles is None else inner_cycles,
                p.cycle if cycle is None else cycle]
        _check(lib().ccm_set_cycle_params(self.h, float(vals[0]), *[int(v) for v in vals[1:]]),
               "ccm_set_cycle_params")
        p.omega, p.nu1, p.nu2, p.inner_cycles, p.cycle = vals

    def set_smo2_blocks(self, block: int, overlap: int):
        """Rebuild the SMO-2 blocks: cores of `block` rows widened by `overlap` on each side."""
        _check(lib().ccm_set_smo2_blocks(self.h, int(block), int(overlap)), "ccm_set_smo2_blocks")
        self.params.ras_block, self.params.ras_overlap = int(block), int(overlap)

    def set_launch_cap(self, max_ctas: int):
        """At most max_ctas CTAs per right-hand side in the persistent kernels (0: no cap)."""
        _check(lib().ccm_set_launch_cap(self.h, int(max_ctas)), "ccm_set_launch_cap")

    def level_launch(self, level, precision=CCM_FP64, nrhs=1) -> ccm_launch_info:
        """Items and CTAs of level `level`'s persistent sweep and restriction launches."""
        out = ccm_launch_info()
        _check(lib().ccm_level_launch(self.h, level, precision, nrhs, ctypes.byref(out)), "ccm_level_launch")
        return out

    def fmg(self, r, precision=CCM_FP64, stream=None):
        """One FMG cycle for L u = r from the zero guess (ccm_fmg)."""
        import torch
        u = torch.zeros_like(r)
        _check(lib().ccm_fmg(self.h, _ptr(u), _ptr(r), precision, _stream(stream)), "ccm_fmg")
        return u

    def wait_selftest(self, stream=None) -> int:
        """ccm_wait_selftest: the bounded-wait failure path; returns the status code."""
        return lib().ccm_wait_selftest(self.h, _stream(stream))

    # ---- accounting
    def profile(self, kernel_class: int):
        _check(lib().ccm_profile(self.h, kernel_class), "ccm_profile")

    def profile_read(self):
        ms, n = ctypes.c_double(0), ctypes.c_int64(0)
        _check(lib().ccm_profile_read(self.h, ctypes.byref(ms), ctypes.byref(n)), "ccm_profile_read")
        return ms.value, n.value

    # ---- input averages: the library's rules, the caller's functions (marshalled through
    # ctypes callbacks that only evaluate them at the nodes the library passes)
    def cell_averages(self, fn, quad=None) -> np.ndarray:
        """<fn> over every non-empty cell [ny, nx] (host), by ccm_cell_averages; fn(x, y) is
        vectorised over numpy arrays.  `quad` is accepted for compatibility and unused."""
        err = []

        def cb(ctx, n, x, y, out):
            try:
                X = np.ctypeslib.as_array(x, shape=(n,))
                Y = np.ctypeslib.as_array(y, shape=(n,))
                np.ctypeslib.as_array(out, shape=(n,))[:] = fn(X, Y)
            except Exception as e:      # re-raised after the call
                err.append(e)

        out = np.zeros((self.ny, self.nx))
        c = FIELD_FN(cb)
        _check(lib().ccm_cell_averages(self.h, c, None, out.ctypes.data), "ccm_cell_averages")
        if err:
            raise err[0]
        return out

    def boundary_averages(self, u, ux, uy, quad=None) -> np.ndarray:
        """<<N u>> over every boundary segment (host), by ccm_boundary_averages: u (Dirichlet),
        grad u . n (Neumann) or gamma1 u + gamma2 grad u . n (Robin).  `quad` is unused."""
        err = []

        def cb(ctx, n, x, y, pu, pux, puy):
            try:
                X = np.ctypeslib.as_array(x, shape=(n,))
                Y = np.ctypeslib.as_array(y, shape=(n,))
                np.ctypeslib.as_array(pu, shape=(n,))[:] = u(X, Y)
                np.ctypeslib.as_array(pux, shape=(n,))[:] = ux(X, Y)
                np.ctypeslib.as_array(puy, shape=(n,))[:] = uy(X, Y)
            except Exception as e:
                err.append(e)

        out = np.zeros(self.nseg)
        c = GRAD_FN(cb)
        _check(lib().ccm_boundary_averages(self.h, c, None, out.ctypes.data), "ccm_boundary_averages")
        if err:
            raise err[0]
        return out


class Group:
    """Many set-up problems advanced together by one CUDA graph launch per solve
    (ccm_group_create / ccm_group_solve).  The solvers must outlive the group."""

    def __init__(self, solvers, stream=None):
        self.solvers = list(solvers)
        n = len(self.solvers)
        arr = (P * max(1, n))(*[s.h for s in self.solvers])
        g = P()
        _check(lib().ccm_group_create(arr, n, _stream(stream), ctypes.byref(g)), "ccm_group_create")
        self.g = g

    @property
    def programmatic(self) -> bool:
        m, p = I(0), I(0)
        _check(lib().ccm_group_query(self.g, ctypes.byref(m), ctypes.byref(p)), "ccm_group_query")
        return bool(p.value)

    def solve(self, fs, gs=None, us=None, stream=None, check=True):
        """fs[k], gs[k], us[k]: member k's cell averages, boundary data (or None) and initial
        guess (None: zero).  Returns (solutions, per-member ccm_stats, return code)."""
        import torch
        n = len(self.solvers)
        us = [torch.zeros_like(f) if (us is None or us[k] is None) else us[k].clone() for k, f in enumerate(fs)]
        fa = (P * n)(*[_ptr(f) for f in fs])
        ua = (P * n)(*[_ptr(u) for u in us])
        ga = None if gs is None else (P * n)(*[_ptr(g) for g in gs])
        st = (ccm_stats * n)()
        rc = lib().ccm_group_solve(self.g, fa, ga, ua, _stream(stream), st)
        if check:
            _check(rc, "ccm_group_solve")
        return us, list(st), rc

    def close(self):
        if getattr(self, "g", None):
            lib().ccm_group_free(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostSetup:
    """Host-only setup (ccm_host_build): the discrete choices of every level, no GPU needed."""

    def __init__(self, prob, **params):
        self._ps, self._curves = problem_struct(prob)
        self.params = default_params(**params)
        h = P()
        _check(lib().ccm_host_build(ctypes.byref(self._ps), ctypes.byref(self.params), ctypes.byref(h)),
               "ccm_host_build")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().ccm_host_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sizes(self, level=0):
        nx, ny = I(0), I(0)
        n2, ns = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib().ccm_host_level_sizes(self.h, level, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(n2),
                                          ctypes.byref(ns)), "ccm_host_level_sizes")
        return nx.value, ny.value, n2.value, ns.value

    def rows(self, level=0):
        nx, ny, n2, ns = self.sizes(level)
        cell = np.zeros(n2, np.int32)
        cols = np.zeros((n2, 15), np.int32)
        beta = np.zeros((n2, 15))
        nb = np.zeros(n2)
        seg = np.zeros(n2, np.int32)
        _check(lib().ccm_host_rows(self.h, level, cell.ctypes.data, cols.ctypes.data, beta.ctypes.data,
                                   nb.ctypes.data, seg.ctypes.data), "ccm_host_rows")
        return cell, cols, beta, nb, seg

    def cell_map(self, level=0):
        nx, ny, n2, ns = self.sizes(level)
        n = nx * ny
        st = np.zeros(n, np.int8)
        ow = np.zeros(n, np.int32)
        rg = np.zeros(n, np.int8)
        vol = np.zeros(n)
        mom = np.zeros((n, 15))
        _check(lib().ccm_host_cell_map(self.h, level, st.ctypes.data, ow.ctypes.data, rg.ctypes.data,
                                       vol.ctypes.data, mom.ctypes.data), "ccm_host_cell_map")
        sh = (ny, nx)
        return st.reshape(sh), ow.reshape(sh), rg.reshape(sh), vol.reshape(sh), mom.reshape(ny, nx, 15)
