"""The multi-GPU path of bench.py runs independent replicas (MAP on one graph does not shard);
its only collective is the final aggregation: the slowest rank's time and the edges of all
ranks.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        # rank r: 10 (r + 1) ms for (r + 1) * 1e9 edges
        v, ms, edges = bench.replica_value(10.0 * (rank + 1), 1e9 * (rank + 1), device="cpu")
        out.put((rank, v, ms, edges))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, v, ms, edges in res:
        assert ms == pytest.approx(20.0)          # the slowest rank
        assert edges == pytest.approx(3e9)        # all ranks' edges
        assert v == pytest.approx(3e9 / 0.020 / 1e9)  # 150 GTEPS


def test_single_process_needs_no_collective():
    import bench

    v, ms, edges = bench.replica_value(10.0, 2e9, device="cpu")
    assert (v, ms, edges) == pytest.approx((200.0, 10.0, 2e9))
