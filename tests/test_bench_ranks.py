"""The multi-rank path of bench.py (replicas, one process per GPU) on CPU:
two gloo ranks check the job time (the slowest rank's), the whole-job value,
per-rank action streams, and that only rank 0 of the reference arm prints."""
import io
import os
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = bench.max_over_ranks(1.0 + 0.5 * rank, dist, "cpu")
    value = bench.job_value(4096, 20, world, elapsed)
    seed = bench.replica_seed(rank)

    class Args:
        gpus, steps, warmup = world, 1, 0
    buf = io.StringIO()
    calls = []
    orig = bench.oracle_sample
    bench.oracle_sample = lambda n, k, cores: (calls.append(n) or (n * k, 1.0, 100.0))
    try:
        with redirect_stdout(buf):
            bench.reference_arm(Args)
    finally:
        bench.oracle_sample = orig
    dist.destroy_process_group()
    out.put((rank, elapsed, value, seed, buf.getvalue(), len(calls)))


@pytest.mark.timeout(120)
def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=100) for _ in range(world))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    (_, e0, v0, s0, o0, c0), (_, e1, v1, s1, o1, c1) = res
    assert e0 == e1 == 1.5                      # the slowest rank's time, on every rank
    assert v0 == v1 == 2 * 4096 * 20 / 1.5      # whole-job env-steps over that time
    assert s0 != s1                             # independent action streams
    assert '"impl": "reference"' in o0 and c0 > 0
    assert o1 == "" and c1 == 0                 # rank 1 of the reference arm does no work
