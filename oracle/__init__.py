"""CPU oracle for the fourth-order cut-cell elliptic solver (arxiv 2504.00724).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
the paper's method, written from the paper and independent of the CUDA path:
it shares no code, tables or helpers with ``paper_2504_00724_gb300`` and never
imports it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it; the
product path must never route through it.

Modules:
  geometry        cut cells, Green-formula moments, Alg. 1 merging (Sec. 2.4, 3.1)
  discretization  regular stencils, PLG stencils, weighted min-norm fits,
                  assembly of L and N (Sec. 3.2 - 3.4)
  multigrid       the paper's V-cycle, smoother SMO-1/SMO-2, transfers,
                  bottom solve, Alg. 3 ordering (Sec. 4)
  cubature        cell and boundary averages of given functions (Sec. 2.4)

Pins (tests/test_oracle_*.py) tie each part to something other than itself:
closed-form polygon and ellipse moments, exactness of every row on Pi_4,
fourth-order convergence, dense brute-force solves and dot-product identities.
The PLG stencil choice is a deterministic reading of an algorithm the paper
only cites; its parity against the paper is unpinned beyond poisedness,
exactness and agreement between the two independent codes.
"""
