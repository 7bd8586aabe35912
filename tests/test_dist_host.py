"""Host logic of the multi-process runs on CPU (gloo, world size 2): the
slowest rank sets the job's time, and independent units (fields of the PSF
sweep) are split into contiguous shares that cover every unit once."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        mine = [1.0 + rank, 10.0 - rank]
        got = bench.max_over_ranks(mine, None, ws)
        lo, hi = bench.shard_range(977, rank, ws)
        out.put((rank, got, lo, hi))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_shards_with_two_gloo_ranks():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, lo, hi in res:
        assert got == [2.0, 10.0]                 # entry-wise maximum over both ranks
    shares = [(lo, hi) for _, _, lo, hi in res]
    assert shares[0][0] == 0 and shares[-1][1] == 977 and shares[0][1] == shares[1][0]
    assert abs((shares[0][1] - shares[0][0]) - (shares[1][1] - shares[1][0])) <= 1


def test_shard_range_partitions_for_any_world_size():
    import bench
    for n in (0, 1, 7, 977, 1000):
        for ws in (1, 2, 3, 8):
            cover = []
            for r in range(ws):
                lo, hi = bench.shard_range(n, r, ws)
                cover.extend(range(lo, hi))
            assert cover == list(range(n))
