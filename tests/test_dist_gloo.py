"""The replica plumbing of bench.py (barrier, max / sum over ranks) with two gloo ranks on CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    import bench
    d = bench.Dist(world)
    d.barrier()
    # each rank reports its own time and face count; the job takes the slowest time and all faces
    mx = d.allreduce(10.0 * (rank + 1), "max")
    sm = d.allreduce(1000.0 * (rank + 1), "sum")
    d.barrier()
    d.close()
    with open(os.path.join(out, f"r{rank}"), "w") as f:
        f.write(f"{d.rank} {d.world} {mx} {sm}")


def test_replicas_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        rank, world, mx, sm = (tmp_path / f"r{r}").read_text().split()
        assert (int(rank), int(world)) == (r, 2)
        assert float(mx) == 20.0 and float(sm) == 3000.0


def test_single_rank_needs_no_process_group():
    import bench
    d = bench.Dist(1)
    assert d.world == 1 and d.pg is None
    assert d.allreduce(3.5, "max") == 3.5
    d.close()


def test_batch_shards_cover_every_net_once():
    # the 64-net batch split by net over 1..8 ranks: every net on exactly one rank, sizes even
    import bench
    for world in range(1, 9):
        parts = [bench.shard_nets(64, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        assert max(map(len, parts)) - min(map(len, parts)) <= 1
