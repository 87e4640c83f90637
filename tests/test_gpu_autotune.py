"""The autotuner on a real handle: it re-parameterises the set-up solver (no new setup), the
winner converges, and a solve with the tuned parameters still reaches the direct solution."""
import numpy as np
import pytest

import workloads as W
from oracle import cubature as Q
from oracle import multigrid as MG

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2504_00724_gb300")
from paper_2504_00724_gb300 import autotune as AT  # noqa: E402

pytestmark = pytest.mark.gpu


def test_autotune_star128():
    prob, mms = W.star(128), W.mms_star()
    H = MG.build_hierarchy(prob)
    lv = H.levels[0]
    fa = Q.cell_averages(lv.cg, mms.f(prob.a, prob.b, prob.c))
    ga = Q.boundary_averages(lv.cg, lv.dz.segs, mms.u, mms.ux, mms.uy)
    want = MG.direct_solve(lv.dz, fa.ravel() - lv.dz.N @ ga).reshape(lv.ny, lv.nx)
    s = P.Solver(prob, rtol=1e-12, max_iter=200)
    try:
        f, g = torch.tensor(fa, device="cuda"), torch.tensor(ga, device="cuda")
        cands = [c for c in AT.default_candidates() if c["omega"] == 0.7 and c["inner_cycles"] in (2, 3)]
        blocks = [(64, 24), (32, 16)]
        best, rec = AT.autotune(s, f, g, candidates=cands, repeats=2, block_candidates=blocks)
        assert len(rec) == len(blocks) + len(cands) and all(r["ms"] > 0 for r in rec)
        assert (best.pop("ras_block"), best.pop("ras_overlap")) in blocks
        assert best in [{k: c[k] for k in best} for c in cands]
        assert s.params.nu1 == best["nu1"] and s.params.cycle == best["cycle"]
        u, st = s.solve(f, g)
        assert st.rel_residual <= 1e-12
        assert np.abs(u.cpu().numpy() - want).max() <= 1e-10 * np.abs(want).max()
    finally:
        s.close()
