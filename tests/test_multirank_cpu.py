"""The benchmark's multi-rank plumbing on CPU (gloo, world size 2): process
group set-up from the torchrun environment, barrier, max over ranks, and the
reference arm's rule that only rank 0 works and prints."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    dist, r, ws = bench._dist()
    assert (r, ws) == (rank, world) and dist.get_backend() == "gloo"
    bench._barrier(dist)
    m = bench._max_over_ranks(dist, float(10 * rank + 3))
    out = {"rank": r, "max": m}
    if rank == 1:
        # the reference arm returns at once on ranks other than 0
        class A:
            steps, warmup, gpus = 1, 3, world
        out["ref_rc"] = bench.run_reference(A(), None)
    bench._barrier(dist)
    dist.destroy_process_group()
    q.put(out)


def test_two_rank_barrier_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    by = {r["rank"]: r for r in res}
    assert by[0]["max"] == by[1]["max"] == 13.0
    assert by[1]["ref_rc"] == 0
