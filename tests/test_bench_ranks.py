"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
timing; both see the largest (the job is as slow as its slowest rank), and
the reference arm prints on rank 0 only."""
import contextlib
import io
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.sync_ranks()
    got = bench.max_over_ranks(10.0 + 5.0 * rank)
    dist.destroy_process_group()
    q.put((rank, got))


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 15.0, 1: 15.0}


def test_single_process_is_its_own_maximum():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5


def test_reference_arm_prints_on_rank_zero_only():
    import bench
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_reference(type("A", (), dict(workload="single_sphere_128", warmup=0, steps=1, tol=1e-10,
                                                smoother="gs"))(), 1, 2)
    assert out.getvalue() == ""
