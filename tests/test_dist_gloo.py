"""Two gloo ranks on the CPU exercise the replica plumbing bench.py uses on N GPUs."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    from paper_2109_07073_b300 import dist
    r, w = dist.init("gloo")
    dist.barrier(w)
    step_ms = 10.0 + 5.0 * r          # rank 1 is the slow one
    worst = dist.max_over_ranks(step_ms, w)
    value = dist.weak_scaling_value(1000.0, w, worst)
    dist.barrier(w)
    import torch.distributed as tdist
    tdist.destroy_process_group()
    q.put((r, w, worst, value))


def test_two_gloo_ranks_agree_on_the_slowest_step():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 15.0 for o in out)                      # max over ranks
    assert all(o[3] == pytest.approx(1000.0 * 2 / 0.015) for o in out)


def test_single_rank_is_a_no_op():
    from paper_2109_07073_b300 import dist
    os.environ.pop("WORLD_SIZE", None)
    r, w = dist.init("gloo")
    assert (r, w) == (0, 1)
    assert dist.max_over_ranks(3.0, 1) == 3.0
    assert dist.weak_scaling_value(10.0, 1, 2.0) == 5000.0
