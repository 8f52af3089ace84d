"""The multi-rank path of bench.py on CPU: two gloo ranks aggregate their replicas' figures
with aggregate_over_ranks (timed region = max over ranks, work = sum over ranks), as the
NCCL ranks of `torchrun --nproc-per-node N bench.py` do on GPUs."""
import importlib.util
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        ms, tot = b.aggregate_over_ranks(dist, [10.0, 12.5][rank], {"applies": [100, 80][rank], "solves": [7, 9][rank],
                                                                     "steps": 10}, "cpu")
        q.put((rank, ms, tot))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, tot in res:
        assert ms == 12.5
        assert tot == {"applies": 180.0, "solves": 16.0, "steps": 20.0}


def test_single_rank_passthrough():
    ms, tot = _bench().aggregate_over_ranks(None, 3.0, {"applies": 5}, "cpu")
    assert ms == 3.0 and tot == {"applies": 5.0}
