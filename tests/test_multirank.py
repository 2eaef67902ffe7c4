"""The multi-rank path of bench.py on CPU: two gloo ranks (one process per
GPU in a real run) take disjoint shards of the batched workload, and the
job's throughput is the cell-steps of all ranks over the slowest rank's
time.  The reference arm runs on rank 0 only."""
import importlib.util
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        insts = b.make_instances(3, rank)
        names = [i.name for i in insts]
        cells = sum(i.cells for i in insts) * b.STEPS_PER_CALL
        ms_local = 10.0 + 5.0 * rank  # the slower rank sets the job's time
        value, ms, units = b.job_throughput(cells, ms_local, "cpu")
        everyone = [None] * world
        dist.all_gather_object(everyone, (names, cells))
        # the reference arm: ranks other than 0 leave at once and print nothing
        printed = io.StringIO()
        with redirect_stdout(printed):
            rc = b.run_reference(b.parse_args_for_test(["--impl", "reference", "--steps", "1", "--warmup", "0",
                                                        "--instances", "2"])) if rank != 0 else 0
            if rank != 0:  # the 3-D workload's reference arm as well
                rc |= b.run_reference_3d(b.parse_args_for_test(["--impl", "reference", "--workload", "random3d",
                                                                "--steps", "1", "--warmup", "0"]))
        out.put((rank, value, ms, units, everyone, rc, printed.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, v0, ms0, u0, all0, _, _), (r1, v1, ms1, u1, all1, rc1, out1) = res
    names0, cells0 = all0[0]
    names1, cells1 = all0[1]
    assert not set(names0) & set(names1)                      # disjoint shards
    b = _bench()
    assert names0 + names1 == [i.name for i in b.make_instances(6, 0)]  # = the single-rank workload
    assert ms0 == ms1 == 15.0                                  # max over ranks
    assert u0 == u1 == cells0 + cells1                         # sum over ranks
    assert v0 == pytest.approx((cells0 + cells1) / 15e-3 / 1e9)
    assert rc1 == 0 and out1 == ""
    # the 3-D workload gives each rank its own grid (seed base + rank)
    import workloads as W
    assert b.W3_N == 256 and b.make_instance3d.__defaults__ == (0,)
    i0 = W.random_instance3d(8, 8, 8, seed=W.BASE_SEED + 0)
    i1 = W.random_instance3d(8, 8, 8, seed=W.BASE_SEED + 1)
    assert not (i0.bx == i1.bx).all()
