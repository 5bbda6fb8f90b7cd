"""The bench's multi-rank plumbing on CPU with gloo, world size 2: the timing is
the max over ranks, the whole-job value counts every rank's work, and the
many-instance ranks take disjoint seeded instances (replicas, no exchange)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import torch.distributed as dist
    r, w = bench.dist_init()
    assert (r, w) == (rank, world) and dist.get_backend() == "gloo"
    t = bench.max_over_ranks(1.0 + rank, w)        # per-rank times 1 s and 2 s
    bench.barrier(w)
    out[rank] = (t, w * 10.0 / t, tuple(bench.batch_instances(r, 3)))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.0                 # max over ranks
    assert res[0][1] == res[1][1] == 10.0                # 2 ranks x 10 units / 2 s
    assert set(res[0][2]).isdisjoint(res[1][2])
    assert sorted(res[0][2] + res[1][2]) == list(range(6))
