"""Host-side logic of the N-GPU bench path (independent replicas, weak
scaling) on CPU: two gloo ranks set up the process group the way bench.py
does under torchrun, agree on the slowest rank's time, and aggregate the
whole-job rate; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, _ = bench.dist_setup(world)
    assert (r, w) == (rank, world) and dist.get_backend() == "gloo"
    bench.barrier(w)
    ms = bench.max_over_ranks(10.0 * (rank + 1), w)   # rank 1 is the slowest
    rate = bench.whole_job_rate(1e6, w, ms)
    out.put((rank, ms, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_rank():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [20.0, 20.0]
    # 2 ranks x 1e6 units in 20 ms -> 100 million units per second
    assert got[0][2] == pytest.approx(100.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup, gpus, prec = 1, 1, 2, "f32"

    assert bench.run_reference(Args(), None, rank=1, world=2) == 0
    assert capsys.readouterr().out == ""
