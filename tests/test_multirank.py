"""The multi-GPU arm of bench.py is "replicas only": every rank advances its
own independent replica (seeded by rank) and the job time is the maximum over
ranks.  Its host-side logic runs here as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    cfg = bench.workload("liquid_n1000", r)
    # every rank reports a different "time"; the job takes the slowest
    t = bench.max_over_ranks(1.5 + r, "cpu")
    ref = bench.run_reference(type("A", (), dict(workload="liquid_n1000", trav="3c08",
                                                 trunc="pair", steps=1, warmup=0))())
    out.put((r, ws, float(cfg["x"][0, 0]), cfg["x"].shape, t, ref is None))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ws0, x0, sh0, t0, ref0), (r1, ws1, x1, sh1, t1, ref1) = res
    assert ws0 == ws1 == 2
    assert sh0 == sh1 == (3, 1000)
    assert x0 != x1                     # independent replicas (seed + rank)
    assert t0 == t1 == 2.5              # max over ranks
    assert ref1 and not ref0            # the reference arm runs on rank 0 only
