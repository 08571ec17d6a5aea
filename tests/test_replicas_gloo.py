"""The multi-GPU form of the bench is replicas only: each rank evaluates its own designs
and the ranks exchange nothing but the timing.  This checks that host logic with two gloo
ranks on the CPU: disjoint design seeds, the barrier, the max over ranks and the whole-job
value every rank derives from it."""
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=ws)
    try:
        bench._barrier(ws)
        slowest = bench._max_over_ranks(100.0 + 25.0 * rank, ws)     # this rank's "time"
        out.put((rank, slowest, bench._replica_value(ws, 40, slowest),
                 bench._replica_seeds(rank, 5)))
        bench._barrier(ws)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_agree_on_the_whole_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [125.0, 125.0]               # both see the slowest rank
    assert res[0][2] == res[1][2] == pytest.approx(2 * 40 / 0.125)
    assert not set(res[0][3]) & set(res[1][3])                  # disjoint designs
