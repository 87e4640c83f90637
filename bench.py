#!/usr/bin/env python
"""Benchmark: fine-grid unknowns solved per second to a 1e-10 relative residual.

Workload: the interior of the 5-petal star r(t) = 0.3 + 0.08 cos 5t centred at (0.5, 0.5),
(a, b, c) = (1, 0.5, 2), Dirichlet data and cell averages of f from the manufactured solution
u = exp(x) sin(pi y) + x^4 (inputs synthetic, computed once before timing).  One step = one
full solve (V-cycles of Alg. 2 with SMO-1/SMO-2, residual, restriction, prolongation, bottom
solve, outer FP64 residual) from the resident right-hand side to ||r - L u|| <= rtol ||r||.

value:  mixed form (FP32 cycles in FP64 refinement), inputs resident in HBM, CUDA events.
e2e:    the same through the C ABI with pinned host buffers (ccm_solve_host): the kernels read f,
        g and the initial guess from host memory and write the solution's non-empty cells back,
        inside the timing.
fp64:   the plain FP64 form, same workload and tolerance.
roofline: the dominant kernel class, timed live with CUDA events during the timed steps;
        algorithmic bytes per unit as in the method's byte model (12 B per regular cell per
        FP32 sweep; 16 x 12 B of fitted row plus 2 x 20 x 4 B of banded L22 factors per
        irregular row), the dense SMO-2 block inverses this build reads instead of the banded
        factors reported beside them as design overhead.
vcycle: one FP32 V-cycle, event-timed, against the unfused (120 B per fine cell) and the
        method-minimum (35 B per fine cell) byte models.
equal_accuracy: both forms against the exact cell averages and against the discrete solution
        (solved to rel. residual 1e-13), at rel. residuals 1e-10 and 1e-12.
configs: the other workloads of the benchmark definition (disk 64^2 FP64; star 256^2 and
        1024^2 in both forms; three ellipses 2048^2 mixed; the adjoint workload on the star
        2048^2 with central finite differences in 16 seeded directions).
cpu_baseline / --impl reference: the CPU oracle (NumPy/SciPy) on a bounded sample of the
same workload (same domain, coefficients and data at a smaller grid); the baseline also runs
one oracle process per host core and reports the oracle's setup time separately.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "fine-grid unknowns solved/s to 1e-10 rel. residual"
UNIT = "unknowns/s"
RTOL = 1e-10
SM_COUNT = 152
FP64_FMA_PER_CLK_SM = 2          # FP64 FMA issue rate per SM (4 flop / clk / SM)

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a reported kernel
# class on the default 4096^2 workload, from one ncu capture (the command is in profiles/).
# A figure is reported only while the device sources hash to the value it was taken on.
KERNEL_SOURCES = ("kernels.cuh", "smooth.cuh", "outer.cuh")
NCU_TRAFFIC = {        # class name -> (source hash, bytes per launch)
    "fp32 sweep, level 0 (SMO-1 regular cells + SMO-2 blocks)": ("e9d37767504660f2", 69.69e6),
    "fp32 residual + restriction, level 0": ("e9d37767504660f2", 76.64e6),
    "outer residual, level 0 (regular cells, float-float)": ("e9d37767504660f2", 95.72e6),
}


def source_hash():
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2504_00724_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_of(name, n):
    if n != 4096 or name not in NCU_TRAFFIC:
        return None
    sha, byts = NCU_TRAFFIC[name]
    return byts if sha == source_hash() else None


def sweep_class_bytes(n_reg, n_irr, launches, iters, nu1, nu2, cycle):
    """Algorithmic bytes per launch of the level-0 FP32 sweep class, averaged over its
    `launches` per solve: a regular cell reads u and r and writes u (12 B), an irregular row
    reads its fitted row (16 x 12 B) and the banded L22 factors of its SMO-2 solve (2 x 20 x
    4 B).  Per outer iteration (`iters`) the first sweep starts from zero and reads no u (when
    nu1 >= 1 and V-cycles) and the last one also reads and writes the FP64 solution, 16 B per
    non-empty cell (when nu2 >= 2; with nu2 = 1 that sweep is the prolongation sweep, another
    class).  Returns (bytes per launch, bytes per regular cell, bytes per irregular row)."""
    n_zero = iters if (nu1 >= 1 and cycle == 0) else 0
    n_fold = iters if nu2 >= 2 else 0
    reg_b = (12.0 * launches - 4.0 * n_zero + 16.0 * n_fold) / launches
    irr_b = 16 * 12.0 + 2 * 20 * 4.0 + 16.0 * n_fold / launches
    return n_reg * reg_b + n_irr * irr_b, reg_b, irr_b


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--sample-n", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the equal-accuracy comparison and the other workloads (disk 64^2, star 256^2 "
                         "and 1024^2, three ellipses 2048^2, the adjoint workload)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched workloads (disk 512^2 with 256 right-hand sides; 64 geometries)")
    ap.add_argument("--coarsest", type=int, default=64,
                    help="the hierarchy stops at the first level with at most this many cells per side "
                         "(64: the bottom level's dense inverse, ~1.2k unknowns on the star, replaces the "
                         "launch-bound 32^2 and 16^2 levels)")
    ap.add_argument("--profile-run", action="store_true",
                    help="only setup, warm-up and the timed solves (for an ncu launch list)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([v.strip() for v in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if len(s) > 2 + k and s[2 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ------------------------------------------------------------------ CPU oracle leg

def oracle_sample(n: int, steps: int, min_seconds: float = 10.0, max_solves: int = 400):
    """Time the oracle's multigrid solve (paper parameters) on the star workload at n x n:
    at least `steps` solves and at least `min_seconds` of solve time (at most max_solves).
    The oracle's setup (cut cells, stencils, fits, hierarchy) is timed separately."""
    import workloads as W
    from oracle import cubature as Q
    from oracle import multigrid as MG
    prob, mms = W.star(n), W.mms_star()
    t0 = time.perf_counter()
    H = MG.build_hierarchy(prob)
    setup_s = time.perf_counter() - t0
    lv = H.levels[0]
    fa = Q.cell_averages(lv.cg, mms.f(prob.a, prob.b, prob.c)).ravel()
    ga = Q.boundary_averages(lv.cg, lv.dz.segs, mms.u, mms.ux, mms.uy)
    r = fa - lv.dz.N @ ga
    r[~lv.ne] = 0.0
    ncell = int(lv.ne.sum())
    times, iters = [], []
    while len(times) < max_solves and (len(times) < steps or sum(times) < min_seconds):
        hist = []
        t0 = time.perf_counter()
        MG.solve(H, r, rtol=RTOL, max_iter=400, history=hist)
        times.append(time.perf_counter() - t0)
        iters.append(len(hist) - 1)
    tot = sum(times)
    return {"value": ncell * len(times) / tot, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"star {n}x{n} ({ncell} unknowns), oracle V-cycles (omega 0.5, nu 3) to rtol {RTOL}, "
                      f"{len(times)} solve(s), {np.mean(iters):.0f} cycles each, {tot:.1f} s",
            "seconds": tot, "solves": len(times), "setup_s": setup_s, "unknowns": ncell}


def _oracle_worker(args):
    n, seconds = args
    out = oracle_sample(n, 1, min_seconds=seconds)
    return out["unknowns"] * out["solves"], out["seconds"]


def oracle_all_cores(n: int, seconds: float = 8.0):
    """The oracle on every host core: one process per core (spawned, one BLAS thread each),
    each solving the sample repeatedly for about `seconds`; throughput = unknowns solved by
    all processes / wall time of the slowest."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(n, seconds)] * cores)
    wall = time.perf_counter() - t0
    done = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    return {"value": done / busy, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"star {n}x{n}, {cores} processes x 1 BLAS thread, {busy:.1f} s of solves each "
                      f"({wall:.1f} s wall with setup)"}


def workload_name(n: int) -> str:
    return f"star r=0.3+0.08cos5t, (a,b,c)=(1,0.5,2), {n}x{n} cells, Dirichlet, u=exp(x)sin(pi y)+x^4"


def run_reference(args, rank: int):
    if rank != 0:
        return
    steps = max(1, args.steps)
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_sample(args.sample_n, 1, min_seconds=0.0)
    cb = oracle_sample(args.sample_n, steps, min_seconds=6.0 * steps)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1000 * cb["seconds"] / cb["solves"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(args.n), "rtol": RTOL,
                                            "oracle_sample": f"the same star on {args.sample_n}x{args.sample_n} cells"},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU leg

def batched_workload(stream, flush, nrhs=256, n=512, one_sample=16):
    """Many right-hand sides on one geometry: the disk domain at n^2, nrhs smoothed N(0,1)
    right-hand sides, homogeneous Dirichlet data, mixed precision to rel. residual 1e-10.
    Timed with all right-hand sides advanced together (ccm_params.batch = nrhs) and, for
    comparison, one at a time on a sample of them."""
    import torch
    import paper_2504_00724_gb300 as P
    import workloads as W
    prob = W.disk_minus(n)
    sv = P.Solver(prob, rtol=RTOL, batch=nrhs)
    mask = sv.cell_map()[0] != 0
    F = torch.tensor(W.smoothed_normal_rhs(n, nrhs, mask, seed=0), device="cuda")
    ncell = int(sv.info.n_cells)

    def timed(solver, f, reps):
        per = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            u, st = solver.solve(f, None, stream=stream)
            e1.record(stream)
            e1.synchronize()
            per.append(e0.elapsed_time(e1))
        return float(np.median(per)), st

    solver_batch = sv.info.batch
    sv.solve(F, None, stream=stream)                       # captures the batched graph
    ms, st = timed(sv, F, 3)
    sv.close()
    one = P.Solver(prob, rtol=RTOL)
    one.solve(F[:1], None, stream=stream)
    ms1, st1 = timed(one, F[:one_sample], 2)
    one.close()
    return {"workload": f"Poisson on [0,1]^2 minus the disk r=0.2, {n}x{n} cells, homogeneous Dirichlet, "
                        f"{nrhs} right-hand sides (N(0,1) cell values, 3 smoothing sweeps, seed 0)",
            "value": nrhs * ncell / (ms / 1000.0), "unit": UNIT, "ms_per_solve": ms, "batch": solver_batch,
            "iterations": st.iterations, "rel_residual": st.rel_residual,
            "one_at_a_time": {"value": one_sample * ncell / (ms1 / 1000.0), "ms": ms1,
                              "sample": f"{one_sample} of the right-hand sides, batch 1"}}


def many_geometries_workload(stream, flush, count=64):
    """Many geometries of uneven grid sizes in one graph launch: the independent geometries of
    seeds 0 .. count-1 (stars with (a,b,c) = (1,0.5,2), Dirichlet, and three-ellipse domains
    with (1,0,1), Neumann on the ellipses; grids drawn from {128, 256, 512, 1024}^2; f and g from
    the manufactured solutions of those workloads), mixed precision to rel. residual 1e-10
    each, advanced together by one group solve (one graph launch); beside it the same problems
    solved one after another with their own solves."""
    import torch
    import paper_2504_00724_gb300 as P
    import workloads as W
    drawn = W.many_geometries(count)
    probs = [p for p, _ in drawn]
    t0 = time.time()
    # bottom levels of about a thousand unknowns (dense inverse): 64^2 cells for a star (the
    # 32^2 level of some 6- and 7-petal stars has an eigenvalue with positive real part), 32^2
    # for a three-ellipse domain, which also takes the GMRES(2) correction (the V-cycle alone
    # diverges on its larger grids)
    # independent setups, four at a time on host threads (ccm_setup releases the interpreter)
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(4) as ex:
        solvers = list(ex.map(lambda p: P.Solver(p, rtol=RTOL, max_iter=200, coarsest=64 if "star" in p.name else 32,
                                                 krylov=0 if "star" in p.name else 2), probs))
    setup_s = time.time() - t0
    fs, gs, exact = [], [], []
    for s, (p, m) in zip(solvers, drawn):
        q = s.quadrature()
        fs.append(torch.tensor(s.cell_averages(m.f(p.a, p.b, p.c), quad=q), device="cuda"))
        gs.append(torch.tensor(s.boundary_averages(m.u, m.ux, m.uy, quad=q), device="cuda"))
        exact.append((s.cell_averages(m.u, quad=q), s.cell_map()[0] != 0))
    ncell = int(sum(s.info.n_cells for s in solvers))
    grid_cells = int(sum(p.nx * p.ny for p in probs))

    def timed(fn, reps):
        per = []
        out = None
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            per.append(e0.elapsed_time(e1))
        return float(np.median(per)), out

    grp = P.Group(solvers, stream=stream)
    grp.solve(fs, gs, stream=stream)                       # warm-up
    ms, (us, st, rc) = timed(lambda: grp.solve(fs, gs, stream=stream), 3)
    programmatic = grp.programmatic
    grp.close()
    err = max(float(np.abs(u.cpu().numpy() - ue)[ne].max()) for u, (ue, ne) in zip(us, exact))
    for s, f, g in zip(solvers, fs, gs):
        s.solve(f, g, stream=stream)                       # captures each solver's own graph
    ms1, sts = timed(lambda: [s.solve(f, g, stream=stream)[1] for s, f, g in zip(solvers, fs, gs)], 2)
    for s in solvers:
        s.close()
    nstar = sum(1 for p in probs if "star" in p.name)
    return {"workload": f"{count} independent geometries (seeds 0..{count - 1}): {nstar} stars "
                        "r0~U[0.25,0.32], amp~U[0.05,0.1], k in 3..7, (a,b,c)=(1,0.5,2), Dirichlet, "
                        "u=exp(x)sin(pi y)+x^4, and "
                        f"{count - nstar} three-ellipse domains, (1,0,1), Neumann on the ellipses, "
                        "u=cos(pi x)cos(pi y)+x y^3, GMRES(2) correction; grids drawn from "
                        f"{{128,256,512,1024}}^2 ({grid_cells} grid cells), mixed precision",
            "max_error_vs_exact": err,
            "value": ncell / (ms / 1000.0), "unit": UNIT, "ms_per_solve": ms, "unknowns": ncell,
            "setup_s": setup_s, "graph_launches_per_solve": 1, "programmatic_edges": programmatic,
            "iterations_max": int(max(x.iterations for x in st)), "iterations_min": int(min(x.iterations for x in st)),
            "rel_residual_max": float(max(x.rel_residual for x in st)),
            "one_after_another": {"value": ncell / (ms1 / 1000.0), "ms": ms1,
                                  "iterations_max": int(max(x.iterations for x in sts))}}


def solve_case(prob, mms, precision, stream, flush, rtol=RTOL, coarsest=16, reps=3, **params):
    """Set up one workload, solve it `reps` times (after one untimed solve that captures the
    iteration graph) and report unknowns/s (median time), iterations and the max-norm error
    against the exact cell averages."""
    import torch
    import paper_2504_00724_gb300 as P
    t0 = time.time()
    sv = P.Solver(prob, precision=precision, rtol=rtol, max_iter=400, coarsest=coarsest, **params)
    setup_s = time.time() - t0
    q = sv.quadrature()
    f = torch.tensor(sv.cell_averages(mms.f(prob.a, prob.b, prob.c), quad=q), device="cuda")
    g = torch.tensor(sv.boundary_averages(mms.u, mms.ux, mms.uy, quad=q), device="cuda")
    ua = sv.cell_averages(mms.u, quad=q)
    ne = sv.cell_map()[0] != 0
    sv.solve(f, g, stream=stream)
    per = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        u, st = sv.solve(f, g, stream=stream)
        e1.record(stream)
        e1.synchronize()
        per.append(e0.elapsed_time(e1))
    ms = float(np.median(per))
    out = {"value": int(sv.info.n_cells) / (ms / 1000.0), "unit": UNIT, "ms": ms, "unknowns": int(sv.info.n_cells),
           "levels": int(sv.info.levels), "iterations": st.iterations, "rel_residual": st.rel_residual,
           "max_error_vs_exact": float(np.abs(u.cpu().numpy() - ua)[ne].max()), "setup_s": setup_s}
    sv.close()
    return out


def other_configs(stream, flush):
    """The benchmark definition's other workloads, each in the form(s) it names."""
    import paper_2504_00724_gb300 as P
    import workloads as W
    out = {}
    out["disk64_fp64"] = dict(workload="(1,0,1), [0,1]^2 minus the disk r=0.2, 64x64, Dirichlet, "
                                       "u=sin(2pi x)cos(3pi y)exp(xy), FP64 V-cycles to 16^2",
                              **solve_case(W.disk_minus(64), W.mms_disk(), P.CCM_FP64, stream, flush))
    for n in (256, 1024):
        for prec, tag in ((P.CCM_MIXED, "mixed"), (P.CCM_FP64, "fp64")):
            out[f"star{n}_{tag}"] = dict(workload=workload_name(n), **solve_case(
                W.star(n), W.mms_star(), prec, stream, flush, coarsest=64 if n >= 1024 else 16))
    out["ellipses2048_mixed"] = dict(
        workload="(1,0,1), [0,1]^2 minus three ellipses (seed 0), 2048x2048, Neumann on the ellipses, "
                 "Dirichlet on the box, u=cos(pi x)cos(pi y)+x y^3, mixed",
        krylov="GMRES(2) correction, 3 V-cycles per preconditioner application (the V-cycle alone diverges here)",
        **solve_case(W.three_ellipses(2048), W.mms_ellipses(), P.CCM_MIXED, stream, flush, coarsest=32, krylov=2))
    out["star2048_adjoint"] = adjoint_case(stream)
    return out


def adjoint_case(stream, n=2048, ndir=16, eps=1e-6):
    """The adjoint workload: star at n^2 with (a,b,c) = (1,0.3,1), loss 0.5 ||u - u_obs||^2 with
    u_obs the exact cell averages plus N(0, (1e-3)^2) noise; the gradient with respect to f and
    the boundary data by one forward and one adjoint solve (timed), and its agreement with
    central finite differences in ndir seeded directions (FP64 solves to rel. residual 1e-13)."""
    import torch
    import paper_2504_00724_gb300 as P
    import workloads as W
    from paper_2504_00724_gb300 import autograd as AG
    prob, mms = W.star(n, (1.0, 0.3, 1.0)), W.mms_star()
    s = P.Solver(prob, precision=P.CCM_FP64, rtol=1e-13, max_iter=400)
    try:
        q = s.quadrature()
        fa = s.cell_averages(mms.f(prob.a, prob.b, prob.c), quad=q)
        ga = s.boundary_averages(mms.u, mms.ux, mms.uy, quad=q)
        ne = s.cell_map()[0] != 0
        rng = np.random.Generator(np.random.PCG64(5))
        uobs = np.where(ne, s.cell_averages(mms.u, quad=q) + 1e-3 * rng.standard_normal(ne.shape), 0.0)
        ob = torch.tensor(uobs, device="cuda")
        mask = torch.tensor(ne.astype(np.float64), device="cuda")

        def loss(ff, gg):
            u = AG.solve(s, ff, gg)
            return 0.5 * ((u - ob) ** 2 * mask).sum()

        f = torch.tensor(fa, device="cuda", requires_grad=True)
        g = torch.tensor(ga, device="cuda", requires_grad=True)
        J = loss(f, g)                 # captures both graphs, untimed
        J.backward()
        f.grad = None
        g.grad = None
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        J = loss(f, g)
        J.backward()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        gf, gg = f.grad.detach(), g.grad.detach()
        # the loss is quadratic, so central differences have no truncation error at any step;
        # what remains is rounding: at eps = 1e-6 the change of u (eps |L^-1 d|, about 1e-13
        # here) is only a thousand times the rounding of u itself, at eps = 1 it dominates
        worst = {eps: 0.0, 1.0: 0.0}
        for _ in range(ndir):
            df = torch.tensor(np.where(ne, rng.standard_normal(ne.shape), 0.0), device="cuda")
            dg = torch.tensor(rng.standard_normal(len(ga)), device="cuda")
            ad = float((gf * df).sum() + (gg * dg).sum())
            for e in worst:
                with torch.no_grad():
                    jp = loss(f + e * df, g + e * dg).item()
                    jm = loss(f - e * df, g - e * dg).item()
                worst[e] = max(worst[e], abs((jp - jm) / (2 * e) - ad) / abs(ad))
        return {"workload": f"star {n}x{n}, (a,b,c)=(1,0.3,1), loss 0.5||u-u_obs||^2, u_obs = exact cell "
                            "averages + N(0,1e-3^2) (seed 5), FP64 solves to rel. residual 1e-13",
                "value": int(s.info.n_cells) / (ms / 1000.0), "unit": "unknowns/s (forward + adjoint solve)",
                "ms_forward_and_gradient": ms, "fd_directions": ndir, "fd_eps": eps,
                "fd_max_rel_diff": worst[eps], "fd_max_rel_diff_eps_1": worst[1.0],
                "fd_note": "the loss is quadratic in (f, g): central differences are exact at any step, "
                           "so the difference at eps 1e-6 is rounding (the change of u is ~1e-13, the "
                           "rounding of u ~1e-16); at eps 1 it measures the adjoint's own accuracy"}
    finally:
        s.close()


def equal_accuracy(prob, mms, stream, flush, coarsest, rtols=(1e-10, 1e-12, 1e-13)):
    """Both forms at equal accuracy: the discrete solution (FP64 to rel. residual 1e-13), each
    form's time and its max-norm errors against that solution and against the exact cell
    averages at each rtol; mixed/FP64 at the smallest rtol where the two exact-solution errors
    agree to two significant digits."""
    import torch
    import paper_2504_00724_gb300 as P
    ref = P.Solver(prob, precision=P.CCM_FP64, rtol=1e-13, max_iter=400, coarsest=coarsest)
    q = ref.quadrature()
    f = torch.tensor(ref.cell_averages(mms.f(prob.a, prob.b, prob.c), quad=q), device="cuda")
    g = torch.tensor(ref.boundary_averages(mms.u, mms.ux, mms.uy, quad=q), device="cuda")
    ua = ref.cell_averages(mms.u, quad=q)
    ne = ref.cell_map()[0] != 0
    ud, std = ref.solve(f, g, stream=stream)
    ud = ud.cpu().numpy()
    ref.close()
    disc = float(np.abs(ud - ua)[ne].max())
    rows = []
    for rtol in rtols:
        row = {"rtol": rtol}
        for prec, tag in ((P.CCM_MIXED, "mixed"), (P.CCM_FP64, "fp64")):
            sv = P.Solver(prob, precision=prec, rtol=rtol, max_iter=400, coarsest=coarsest)
            sv.solve(f, g, stream=stream)
            per = []
            for _ in range(2):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                u, st = sv.solve(f, g, stream=stream)
                e1.record(stream)
                e1.synchronize()
                per.append(e0.elapsed_time(e1))
            uu = u.cpu().numpy()
            row[tag] = {"ms": float(np.median(per)), "iterations": st.iterations, "rel_residual": st.rel_residual,
                        "err_vs_exact": float(np.abs(uu - ua)[ne].max()),
                        "err_vs_discrete": float(np.abs(uu - ud)[ne].max())}
            sv.close()
        a, b = row["mixed"]["err_vs_exact"], row["fp64"]["err_vs_exact"]
        row["exact_errors_agree_2_digits"] = float(f"{a:.1e}") == float(f"{b:.1e}")
        row["both_within_20pct_of_discretisation_error"] = max(row["mixed"]["err_vs_discrete"],
                                                               row["fp64"]["err_vs_discrete"]) <= 0.2 * disc
        row["mixed_over_fp64"] = row["fp64"]["ms"] / row["mixed"]["ms"]
        rows.append(row)
    agree = [r for r in rows if r["both_within_20pct_of_discretisation_error"]]
    return {"discrete_rel_residual": std.rel_residual, "discrete_err_vs_exact": disc, "by_rtol": rows,
            "criterion": "both forms' max-norm errors against the discrete solution below 20 % of the "
                         "discretisation error",
            "mixed_over_fp64_at_equal_accuracy": agree[0]["mixed_over_fp64"] if agree else None,
            "equal_accuracy_rtol": agree[0]["rtol"] if agree else None}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import torch
    import paper_2504_00724_gb300 as P
    import workloads as W

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    prob, mms = W.star(args.n), W.mms_star()
    t0 = time.time()
    solver = P.Solver(prob, precision=P.CCM_MIXED, rtol=RTOL, max_iter=200, coarsest=args.coarsest)
    setup_s = time.time() - t0
    info = solver.info
    q = solver.quadrature()
    fa = solver.cell_averages(mms.f(prob.a, prob.b, prob.c), quad=q)
    ga = solver.boundary_averages(mms.u, mms.ux, mms.uy, quad=q)
    ua = solver.cell_averages(mms.u, quad=q)
    ne = solver.cell_map()[0] != 0
    f = torch.tensor(fa, dtype=torch.float64, device="cuda")
    g = torch.tensor(ga, dtype=torch.float64, device="cuda")
    ncell = int(info.n_cells)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 256 MB > L2

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_solves(sv, steps, profile_class=0):
        per, stats = [], None
        sv.profile(profile_class)
        sv.solve(f, g, stream=stream)            # (re)captures the iteration graph, untimed
        sv.profile(profile_class)                # same class: graphs kept, counters cleared
        torch.cuda.synchronize()
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            u, st = sv.solve(f, g, stream=stream)
            e1.record(stream)
            e1.synchronize()
            per.append(e0.elapsed_time(e1))
            stats = (u, st)
        prof = sv.profile_read() if profile_class else (0.0, 0)
        return per, stats, prof

    # warm-up (no kernel-class profiling: the timed graph carries no profiling events)
    solver.profile(0)
    for _ in range(args.warmup):
        solver.solve(f, g)
    barrier()
    launches0 = P.binding.launch_count()
    clocks = Clocks(local)
    with clocks:
        per, (u, st), _ = timed_solves(solver, args.steps, 0)
    launches = P.binding.launch_count() - launches0
    barrier()
    ms_step = float(np.mean(per))
    from paper_2504_00724_gb300.replicas import replica_throughput
    value, _, _ = replica_throughput(float(ncell * args.steps), sum(per) / 1000.0)
    err = float(np.abs(u.cpu().numpy() - ua)[ne].max())
    iters = st.iterations

    if args.profile_run:
        if rank == 0:
            print(json.dumps({"profile_run": True, "ms_per_step": ms_step, "launches": int(launches)}), flush=True)
        solver.close()
        return

    # kernel-class profiles on extra solves (events around the class's launches; not part of
    # value): the level-0 sweep for the roofline, the other classes, the V-cycle
    _, _, prof_sweep = timed_solves(solver, args.steps, P.binding.CCM_PROF_SMO1_FP32)
    _, _, prof_res = timed_solves(solver, 1, P.binding.CCM_PROF_RESID_FP64)
    _, _, prof_rst = timed_solves(solver, 1, P.binding.CCM_PROF_RESTRICT_FP32)
    _, _, prof_vc = timed_solves(solver, 1, P.binding.CCM_PROF_VCYCLE)

    # e2e: host buffers through the C ABI (ccm_solve_host): the packing kernels read f, g and
    # the initial guess from pinned host memory and write the non-empty cells of u back over
    # the host link, inside the timing (the buffer is zeroed before each step)
    fh = torch.tensor(fa, dtype=torch.float64).pin_memory()
    gh = torch.tensor(ga, dtype=torch.float64).pin_memory()
    uh = torch.zeros_like(fh).pin_memory()
    e2e = []
    for _ in range(max(1, args.steps)):
        flush.zero_()
        uh.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.solve_host(fh, gh, uh, stream=stream)
        e1.record(stream)
        e1.synchronize()
        e2e.append(e0.elapsed_time(e1))
    e2e_value = world * ncell / (float(np.mean(e2e)) / 1000.0)
    e2e_err = float(np.abs(uh.numpy() - ua)[ne].max())

    # plain FP64 form, same workload and tolerance
    fp64 = None
    if not args.no_fp64:
        s64 = P.Solver(prob, precision=P.CCM_FP64, rtol=RTOL, max_iter=200, coarsest=args.coarsest)
        s64.solve(f, g)
        per64, (u64, st64), _ = timed_solves(s64, max(1, min(args.steps, 2)))
        err64 = float(np.abs(u64.cpu().numpy() - ua)[ne].max())
        fp64 = {"value": ncell / (float(np.mean(per64)) / 1000.0), "ms_per_step": float(np.mean(per64)),
                "iterations": st64.iterations, "rel_residual": st64.rel_residual, "max_error": err64}
        s64.close()

    batched = None
    geometries = None
    if not args.no_batched and world == 1:
        batched = batched_workload(stream, flush)
        geometries = many_geometries_workload(stream, flush)

    # the autotuner on this workload (V-cycles; omega, sweeps, inner cycles), then the tuned
    # solve timed like the headline; the headline keeps the default parameters
    tuned = None
    if not args.no_autotune:
        from paper_2504_00724_gb300 import autotune as AT
        defaults = {k: getattr(solver.params, k) for k in ("omega", "nu1", "nu2", "inner_cycles", "cycle")}
        dblock = (solver.params.ras_block, solver.params.ras_overlap)
        cands = [c for c in AT.default_candidates() if c["cycle"] == 0 and c["nu1"] >= 2]
        best, rec = AT.autotune(solver, f, g, candidates=cands, repeats=3, stream=stream,
                                block_candidates=AT.default_block_candidates())
        per_t, (_, st_t), _ = timed_solves(solver, args.steps)
        value_t, _, _ = replica_throughput(float(ncell * args.steps), sum(per_t) / 1000.0)
        tuned = {"params": best, "value": value_t, "ms_per_step": float(np.mean(per_t)),
                 "iterations": st_t.iterations, "candidates": len(rec),
                 "default_params": dict(defaults, ras_block=dblock[0], ras_overlap=dblock[1])}
        solver.set_cycle_params(**defaults)
        solver.set_smo2_blocks(*dblock)

    # roofline of the dominant kernel class (largest total time per step).  Algorithmic bytes
    # per unit follow the method's byte model: an FP32 sweep reads u and r and writes u per
    # regular cell (12 B) and per irregular row reads its fitted row (16 x 12 B: 15 coefficients,
    # columns and gathered values, plus the cell's own) and the banded L22 factors of its SMO-2
    # solve (2 x 20 x 4 B, cyclic bandwidth 20); the residual + restriction reads u, r and the
    # volume per fine cell and writes the coarse r and u (12 + 2 x 4 / 4 B); the FP64 residual is
    # bound by the FP64 pipe.  The dense block inverses read instead of banded factors are this
    # build's design overhead and are reported beside the sweep, not counted in it.
    hbm, sm_max, src = peaks()
    clk = clocks.summary()
    n_reg = int(info.n_regular)
    n_irr = int(info.n_irregular)
    li0 = solver.level_launch(0, P.CCM_MIXED)
    classes = []     # (name, ms per step, avg ms per launch, launches per step, bound, work per launch, unit)
    ms, nl = prof_sweep
    if nl:
        # per outer iteration one of these launches starts from the zero correction (it reads
        # no iterate: 8 B per regular cell) and one, the last, also adds its values to the FP64
        # solution (u_hat read and written: 16 B more per non-empty cell); averaged per launch
        per_step_l = nl / args.steps
        pr = solver.params
        byts, reg_b, irr_b = sweep_class_bytes(n_reg, n_irr, per_step_l, iters, pr.nu1, pr.nu2, pr.cycle)
        classes.append(("fp32 sweep, level 0 (SMO-1 regular cells + SMO-2 blocks)", ms / args.steps, ms / nl,
                        per_step_l, "hbm", byts, "GB/s"))
    ms, nl = prof_rst
    if nl:
        classes.append(("fp32 residual + restriction, level 0", ms, ms / nl, nl, "hbm", ncell * 14.0, "GB/s"))
    ms, nl = prof_res
    if nl:
        # the outer residual reads u_hat, r_hat (FP64) and the class byte and writes the FP32
        # image of the residual per regular cell (8 + 8 + 1 + 4 B); it runs in float-float
        # arithmetic at this tolerance
        classes.append(("outer residual, level 0 (regular cells, float-float)", ms, ms / nl, nl, "hbm",
                        n_reg * 21.0, "GB/s"))
    roof = None
    if classes:
        name, ms_step_cls, avg_ms, per_step, bound, work, unit = max(classes, key=lambda c: c[1])
        if bound == "alu":
            peak = SM_COUNT * FP64_FMA_PER_CLK_SM * 2 * sm_max * 1e6 / 1e12
            achieved = work / (avg_ms / 1000.0) / 1e12
        else:
            peak = hbm
            achieved = work / (avg_ms / 1000.0) / 1e9
        traffic = traffic_of(name, args.n)
        roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": traffic, "kernel": name, "avg_launch_us": avg_ms * 1000.0,
                "launches_per_step": per_step, "algorithmic_per_launch": work,
                "peak_source": ("derived: 152 SMs x 4 FP64 flop/clk x max SM clock" if bound == "alu"
                                else f"{src} copy bandwidth"),
                "dram_frac": (traffic / (avg_ms / 1000.0) / 1e9 / peak) if (traffic and bound == "hbm") else None,
                "others": [{"kernel": c[0], "ms_per_step": c[1], "avg_launch_us": c[2] * 1000.0, "bound": c[4],
                            "achieved": (c[5] / (c[2] / 1000.0) / (1e12 if c[4] == "alu" else 1e9)),
                            "traffic": traffic_of(c[0], args.n)}
                           for c in classes if c[0] != name]}
        if name.startswith("fp32 sweep"):
            roof["bytes_per_regular_cell"] = reg_b
            roof["bytes_per_irregular_row"] = irr_b
            roof["design_overhead_bytes_per_launch"] = {
                "smo2_dense_block_inverse_rows": int(li0.block_inv_entries) * 4,
                "class_bytes": n_reg * 1}

    # the whole V-cycle against the two byte models (N0 fine cells, hierarchy factor 4/3 inside)
    vc_ms, vc_n = prof_vc
    vcycle = None
    if vc_n:
        t = vc_ms / vc_n / 1000.0
        vcycle = {"ms": vc_ms / vc_n, "cells": ncell,
                  "unfused_model": {"bytes_per_cell": 120, "GBs": 120.0 * ncell / t / 1e9,
                                    "frac": 120.0 * ncell / t / 1e9 / hbm},
                  "method_minimum_model": {"bytes_per_cell": 35, "GBs": 35.0 * ncell / t / 1e9,
                                           "frac": 35.0 * ncell / t / 1e9 / hbm},
                  "peak": hbm, "peak_source": f"{src} copy bandwidth"}

    configs = None
    eq = None
    if not args.no_configs and world == 1:
        eq = equal_accuracy(prob, mms, stream, flush, args.coarsest)
        configs = other_configs(stream, flush)

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        one = oracle_sample(args.sample_n, 1)
        cpu = {k: one[k] for k in ("value", "unit", "cores", "kind", "sample")}
        cpu["setup_s"] = one["setup_s"]
        cpu["all_cores"] = oracle_all_cores(args.sample_n)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": workload_name(args.n), "unknowns": ncell, "irregular": int(info.n_irregular),
                       "levels": int(info.levels), "coarsest": args.coarsest, "rtol": RTOL,
                       "precision": "FP32 V-cycles in FP64 refinement",
                       "l2": "flushed (256 MB write) before every step", "parallelism": f"replicas x{world}"},
            "iterations": iters, "rel_residual": st.rel_residual, "max_error_vs_exact": err,
            "vcycle_ms": (vc_ms / vc_n) if vc_n else None, "vcycle": vcycle, "setup_s": setup_s,
            "setup_phases_ms": {k: getattr(info, "setup_" + k + "_ms") for k in ("geometry", "fits", "blocks",
                                                                              "bottom", "upload")},
            "fp64": fp64, "mixed_over_fp64": (value / world / fp64["value"]) if fp64 else None,
            "equal_accuracy": eq,
            "configs": configs,
            "batched": batched,
            "many_geometries": geometries,
            "autotuned": tuned,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(2 * ncell * 8 + gh.numel() * 8),
                    "d2h_bytes_per_step": int(ncell * 8), "ms_per_step": float(np.mean(e2e)),
                    "api": "ccm_solve_host, pinned host buffers read and written by the kernels",
                    "max_error_vs_exact": e2e_err},
            "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": cpu, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
