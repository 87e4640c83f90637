"""Autotuner for the cycle parameters of a set-up solver.

The multigrid's free parameters (the shape of the SMO-2 blocks, the smoothing weight omega,
the sweep counts nu1 and nu2, the FP32 cycles per outer iteration and the cycle type, V or
FMG-first) change both the cost of an outer iteration and the number of iterations the solve
needs, and which combination is fastest depends on the domain, the grid and the GPU.  The
block shape sets the work items and the shared-memory stage of the persistent sweep kernel.
`autotune` times complete solves to the solver's tolerance on the caller's right-hand side,
first for every SMO-2 block shape (ccm_set_smo2_blocks: the block inverses are recomputed,
nothing else), keeping the fastest, then for every cycle candidate on that shape
(ccm_set_cycle_params; no new setup), and leaves the solver on the fastest combination that
converged.  Each candidate's first solve captures its graphs and is not timed."""
from __future__ import annotations

import itertools
from typing import Callable, Dict, Iterable, List, Optional, Tuple


def default_candidates() -> List[Dict]:
    """omega in {0.7, 0.8}; nu1 = nu2 in {1, 2, 3, 4}; inner cycles in {2, 3, 4}; V or FMG first."""
    out = []
    for omega, nu, inner, cycle in itertools.product((0.7, 0.8), (1, 2, 3, 4), (2, 3, 4), (0, 1)):
        out.append({"omega": omega, "nu1": nu, "nu2": nu, "inner_cycles": inner, "cycle": cycle})
    return out


def default_block_candidates() -> List[Tuple[int, int]]:
    """(core rows, overlap) of the SMO-2 blocks."""
    return [(64, 24), (64, 16), (64, 32), (48, 16), (32, 16)]


def _event_timer(solver, f, g, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    u, st = solver.solve(f, g, stream=stream, check=False)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), st


def _time(solver, f, g, stream, timer, repeats, rtol):
    _, st = timer(solver, f, g, stream)              # graph capture, not timed
    times, ok, iters = [], st.rel_residual <= rtol, st.iterations
    for _ in range(max(1, repeats)):
        ms, st = timer(solver, f, g, stream)
        times.append(ms)
        ok = ok and st.rel_residual <= rtol
    times.sort()
    return times[len(times) // 2], iters, bool(ok)


def autotune(solver, f, g=None, candidates: Optional[Iterable[Dict]] = None, repeats: int = 3,
             timer: Optional[Callable] = None, stream=None,
             block_candidates: Optional[Iterable[Tuple[int, int]]] = None) -> Tuple[Dict, List[Dict]]:
    """Time `repeats` solves (median, ms) for every SMO-2 block shape (none: keep the
    solver's), keep the fastest that met the tolerance, then every cycle candidate on it, and
    keep the fastest of those.  Returns (best parameters, one record per candidate: the
    parameters, 'ms', 'iterations', 'converged').  The solver is left on the best set.
    `timer(solver, f, g, stream) -> (ms, stats)` replaces the CUDA-event timing."""
    if timer is None:
        import torch
        stream = stream if stream is not None else torch.cuda.current_stream()
        timer = _event_timer
    rtol = solver.params.rtol
    records = []
    blocks = list(block_candidates) if block_candidates is not None else []
    if blocks:
        brec = []
        for (b, o) in blocks:
            solver.set_smo2_blocks(b, o)
            ms, iters, ok = _time(solver, f, g, stream, timer, repeats, rtol)
            brec.append({"ras_block": b, "ras_overlap": o, "ms": ms, "iterations": iters, "converged": ok})
        records += brec
        good = [r for r in brec if r["converged"]]
        if not good:
            raise RuntimeError("autotune: no SMO-2 block shape met the tolerance")
        bb = min(good, key=lambda r: r["ms"])
        solver.set_smo2_blocks(bb["ras_block"], bb["ras_overlap"])
    crec = []
    for cand in (default_candidates() if candidates is None else list(candidates)):
        solver.set_cycle_params(**cand)
        ms, iters, ok = _time(solver, f, g, stream, timer, repeats, rtol)
        crec.append(dict(cand, ms=ms, iterations=iters, converged=ok))
    records += crec
    good = [r for r in crec if r["converged"]]
    if not good:
        raise RuntimeError("autotune: no candidate met the tolerance")
    best = min(good, key=lambda r: r["ms"])
    params = {k: best[k] for k in ("omega", "nu1", "nu2", "inner_cycles", "cycle")}
    solver.set_cycle_params(**params)
    if blocks:
        params["ras_block"], params["ras_overlap"] = solver.params.ras_block, solver.params.ras_overlap
    return params, records
