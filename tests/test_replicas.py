"""The multi-rank path of bench.py (one independent replica per GPU, timing
= max over ranks, value = sum over ranks) on two gloo ranks on the CPU."""
import json
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


def _rank(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    bench.barrier(world)
    ms = [12.5, 20.0][rank]                        # the second rank is slower
    ms_max = bench.reduce_max(ms, world)
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump([ms_max, bench.replica_mlups(1000, 10, ms_max, world)], f)
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank(tmp_path):
    world = 2
    port = _free_port()
    mp.spawn(_rank, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        with open(tmp_path / f"rank{r}.json") as f:
            ms_max, value = json.load(f)
        assert ms_max == 20.0
        # 2 replicas x 1000 sites x 10 steps in 20 ms
        assert value == pytest.approx(2 * 1000 * 10 / 0.020 / 1e6)
