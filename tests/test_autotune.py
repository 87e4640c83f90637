"""The autotuner's selection logic on a stand-in solver (no GPU): the fastest candidate that
met the tolerance wins, candidates that did not converge are skipped, the untimed first
solve of each candidate is discarded, and the solver is left on the winner."""
import types

import pytest

from paper_2504_00724_gb300 import autotune as AT


class FakeSolver:
    def __init__(self):
        self.params = types.SimpleNamespace(rtol=1e-10, omega=0.7, nu1=3, nu2=3, inner_cycles=3, cycle=0,
                                            ras_block=64, ras_overlap=24)
        self.calls = []

    def set_cycle_params(self, **kw):
        for k, v in kw.items():
            setattr(self.params, k, v)

    def set_smo2_blocks(self, block, overlap):
        self.calls.append((block, overlap))
        self.params.ras_block, self.params.ras_overlap = block, overlap


def fake_timer(costs, diverge=()):
    seen = {}

    def timer(solver, f, g, stream):
        p = solver.params
        key = (p.omega, p.nu1, p.inner_cycles, p.cycle)
        n = seen.get(key, 0)
        seen[key] = n + 1
        ms = 1000.0 if n == 0 else costs[key]          # the capture solve is slow and ignored
        rel = 1e-3 if key in diverge else 1e-11
        return ms, types.SimpleNamespace(rel_residual=rel, iterations=6)
    return timer


def test_picks_fastest_converged_candidate():
    cands = [{"omega": 0.7, "nu1": 3, "nu2": 3, "inner_cycles": 3, "cycle": 0},
             {"omega": 0.8, "nu1": 2, "nu2": 2, "inner_cycles": 3, "cycle": 0},
             {"omega": 0.8, "nu1": 1, "nu2": 1, "inner_cycles": 2, "cycle": 1}]
    costs = {(0.7, 3, 3, 0): 10.0, (0.8, 2, 3, 0): 8.0, (0.8, 1, 2, 1): 5.0}
    s = FakeSolver()
    best, rec = AT.autotune(s, None, candidates=cands, timer=fake_timer(costs, diverge={(0.8, 1, 2, 1)}))
    assert best == {"omega": 0.8, "nu1": 2, "nu2": 2, "inner_cycles": 3, "cycle": 0}
    assert (s.params.omega, s.params.nu1, s.params.inner_cycles) == (0.8, 2, 3)
    assert [r["converged"] for r in rec] == [True, True, False]
    assert [r["ms"] for r in rec] == [10.0, 8.0, 5.0]


def test_no_converged_candidate_raises():
    s = FakeSolver()
    cands = [{"omega": 0.7, "nu1": 3, "nu2": 3, "inner_cycles": 3, "cycle": 0}]
    with pytest.raises(RuntimeError):
        AT.autotune(s, None, candidates=cands, timer=fake_timer({(0.7, 3, 3, 0): 1.0}, diverge={(0.7, 3, 3, 0)}))


def test_default_candidates_cover_the_grid():
    c = AT.default_candidates()
    assert len(c) == 2 * 4 * 3 * 2
    assert {"omega": 0.7, "nu1": 3, "nu2": 3, "inner_cycles": 3, "cycle": 0} in c


def test_block_shapes_tuned_first():
    """The SMO-2 block shapes are timed on the solver's cycle parameters, the fastest converged
    shape is kept, then the cycle candidates run on it."""
    s = FakeSolver()
    seen = {}

    def timer(solver, f, g, stream):
        p = solver.params
        key = (p.ras_block, p.ras_overlap, p.nu1)
        n = seen.get(key, 0)
        seen[key] = n + 1
        cost = {(64, 24): 9.0, (32, 16): 7.0, (48, 16): 6.0}[(p.ras_block, p.ras_overlap)] + p.nu1
        rel = 1e-3 if (p.ras_block, p.ras_overlap) == (48, 16) else 1e-11
        return (1000.0 if n == 0 else cost), types.SimpleNamespace(rel_residual=rel, iterations=6)

    cands = [{"omega": 0.7, "nu1": 3, "nu2": 3, "inner_cycles": 3, "cycle": 0},
             {"omega": 0.7, "nu1": 2, "nu2": 2, "inner_cycles": 3, "cycle": 0}]
    best, rec = AT.autotune(s, None, candidates=cands, timer=timer,
                            block_candidates=[(64, 24), (32, 16), (48, 16)])
    assert (best["ras_block"], best["ras_overlap"]) == (32, 16)
    assert best["nu1"] == 2 and s.params.nu1 == 2
    assert s.calls[-1] == (32, 16) and (s.params.ras_block, s.params.ras_overlap) == (32, 16)
    assert [r["converged"] for r in rec[:3]] == [True, True, False]
