"""The multi-rank path on CPU: two gloo processes split a batch of molecules
(disjoint, complete, cost-balanced) and agree on the max of their times."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2404_09452_gb300 import dist as D  # noqa: E402
from paper_2404_09452_gb300 import inputs as I  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    counts = I.batch_atom_counts(n=40)
    mine_rr = D.shard_round_robin(len(counts), rank, world)
    mine_bal = D.shard_balanced([float(c) ** 3 for c in counts], world)[rank]
    t = 1.5 + rank  # stand-in for each rank's elapsed time
    tmax = D.max_over_ranks(t)
    dist.barrier()
    q.put((rank, mine_rr, mine_bal, tmax))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    counts = I.batch_atom_counts(n=40)
    for k in (1, 2):
        parts = [r[k] for r in res]
        assert sorted(sum(parts, [])) == list(range(len(counts)))
        assert not set(parts[0]) & set(parts[1])
    loads = [sum(float(counts[i]) ** 3 for i in r[2]) for r in res]
    assert max(loads) <= 1.2 * min(loads)
    assert all(r[3] == 2.5 for r in res)


def test_single_process_max_is_identity():
    assert D.max_over_ranks(3.25) == 3.25
