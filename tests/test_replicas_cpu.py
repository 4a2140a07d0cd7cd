"""The multi-GPU path is independent replicas: ranks meet only at a barrier
and a max-reduction of their times (gloo).  World size 2 on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2502_00920_gb300 import replicas as RP
    r, w, loc = RP.ranks()
    RP.init(w)
    RP.barrier(w)
    t = 1.0 + r  # the slower rank took 2 s
    m = RP.max_over_ranks(t, w)
    out.put((r, m, RP.aggregate_rate(100.0, m, w)))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    assert all(m == 2.0 for _, m, _ in res)
    assert all(a == pytest.approx(100.0) for _, _, a in res)  # 2 ranks x 100 units / 2 s


def test_single_rank_needs_no_process_group():
    from paper_2502_00920_gb300 import replicas as RP
    assert RP.max_over_ranks(3.5, 1) == 3.5
    assert RP.aggregate_rate(10.0, 2.0, 1) == 5.0
