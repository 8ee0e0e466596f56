"""The multi-GPU path is replicas only (ECB needs no exchange): check its host
logic with two gloo ranks on the CPU: the slowest rank's time wins, the
throughput sums both ranks' bytes, and a rank that never reaches the barrier
is detected by a deadline instead of hanging the others."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _timing_worker(rank, world, port, q):
    from paper_1305_4376_gb300 import replicas
    _init(rank, world, port)
    try:
        replicas.barrier(timeout_s=30)
        my_ms = 10.0 + 5.0 * rank
        mx = replicas.max_over_ranks(my_ms)
        r, w = replicas.world()
        q.put((r, w, mx, replicas.aggregate_gbs(1 << 30, mx, w)))
        replicas.barrier(timeout_s=30)
    finally:
        dist.destroy_process_group()


def _missing_worker(rank, world, port, q):
    from paper_1305_4376_gb300 import replicas
    _init(rank, world, port)
    if rank == 1:
        # this rank fails before the timed region: it never reaches the barrier
        q.put((rank, "left"))
        return
    try:
        replicas.barrier(timeout_s=3)
        q.put((rank, "no error"))
    except RuntimeError as e:
        q.put((rank, "detected: %s" % str(e)[:80]))


def _run(fn, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=fn, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return out


def test_two_rank_timing_takes_the_slowest_and_sums_the_work():
    res = sorted(_run(_timing_worker))
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == 2 for r in res)
    assert all(r[2] == 15.0 for r in res)
    gbs = (2 * (1 << 30)) / 15e-3 / 1e9
    assert all(abs(r[3] - gbs) < 1e-9 for r in res)


def test_missing_rank_is_detected_by_the_barrier_deadline():
    res = dict(_run(_missing_worker))
    assert res[1] == "left"
    assert res[0].startswith("detected"), res[0]
