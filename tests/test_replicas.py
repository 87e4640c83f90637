"""The multi-replica aggregation of bench.py on two gloo ranks (CPU)."""
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("replicas", os.path.join(root, "paper_2504_00724_gb300", "replicas.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    units = [100.0, 300.0][rank]
    secs = [2.0, 4.0][rank]
    out[rank] = mod.replica_throughput(units, secs)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_units_over_slowest_time():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29600 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        value, tmax, units = out[r]
        assert tmax == 4.0 and units == 400.0 and abs(value - 100.0) < 1e-12
