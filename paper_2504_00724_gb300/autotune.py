"""Autotuner for the cycle parameters of a set-up solver.

The multigrid's free parameters (the smoothing weight omega, the sweep counts nu1 and nu2,
the FP32 cycles per outer iteration and the cycle type, V or FMG-first) change both the cost
of an outer iteration and the number of iterations the solve needs, and which combination
is fastest depends on the domain, the grid and the GPU.  `autotune` times complete solves
to the solver's tolerance on the caller's right-hand side for every candidate, on the same
handle (ccm_set_cycle_params; no new setup), and leaves the solver on the fastest candidate
that converged.  Each candidate's first solve captures its graphs and is not timed."""
from __future__ import annotations

import itertools
from typing import Callable, Dict, Iterable, List, Optional, Tuple


def default_candidates() -> List[Dict]:
    """omega in {0.7, 0.8}; nu1 = nu2 in {1, 2, 3, 4}; inner cycles in {2, 3, 4}; V or FMG first."""
    out = []
    for omega, nu, inner, cycle in itertools.product((0.7, 0.8), (1, 2, 3, 4), (2, 3, 4), (0, 1)):
        out.append({"omega": omega, "nu1": nu, "nu2": nu, "inner_cycles": inner, "cycle": cycle})
    return out


def _event_timer(solver, f, g, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    u, st = solver.solve(f, g, stream=stream, check=False)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), st


def autotune(solver, f, g=None, candidates: Optional[Iterable[Dict]] = None, repeats: int = 3,
             timer: Optional[Callable] = None, stream=None) -> Tuple[Dict, List[Dict]]:
    """Time `repeats` solves (median, ms) for every candidate parameter set and keep the fastest
    whose solves met the tolerance.  Returns (best parameters, one record per candidate:
    the parameters, 'ms', 'iterations', 'converged').  The solver is left on the best set.
    `timer(solver, f, g, stream) -> (ms, stats)` replaces the CUDA-event timing."""
    if timer is None:
        import torch
        stream = stream if stream is not None else torch.cuda.current_stream()
        timer = _event_timer
    rtol = solver.params.rtol
    records = []
    for cand in (default_candidates() if candidates is None else list(candidates)):
        solver.set_cycle_params(**cand)
        _, st = timer(solver, f, g, stream)              # graph capture, not timed
        times, ok, iters = [], st.rel_residual <= rtol, st.iterations
        for _ in range(max(1, repeats)):
            ms, st = timer(solver, f, g, stream)
            times.append(ms)
            ok = ok and st.rel_residual <= rtol
        times.sort()
        records.append(dict(cand, ms=times[len(times) // 2], iterations=iters, converged=bool(ok)))
    good = [r for r in records if r["converged"]]
    if not good:
        raise RuntimeError("autotune: no candidate met the tolerance")
    best = min(good, key=lambda r: r["ms"])
    params = {k: best[k] for k in ("omega", "nu1", "nu2", "inner_cycles", "cycle")}
    solver.set_cycle_params(**params)
    return params, records
