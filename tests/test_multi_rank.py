"""The multi-rank path of the benchmark on CPU ranks (gloo, world size 2): replicas
only, so the one exchange is the final reduction of the step time (slowest rank) and
the work (all ranks) that the bench reports for N > 1."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench
    seconds, work = bench.reduce_over_ranks(1.5 + rank, 10.0 * (rank + 1), "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, seconds, work))


def test_bench_reduction_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time and the sum of the work
    assert got == [(0, 2.5, 30.0), (1, 2.5, 30.0)]
