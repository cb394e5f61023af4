"""bench.py's multi-rank logic on CPU: two gloo ranks on 127.0.0.1.

Under torchrun each rank trains an independent replica; the only exchanges
are the barriers around the timed region and the maximum over ranks of the
timed duration, and rank 0 alone prints.  The same helpers run here over gloo
with CPU tensors.
"""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, lr, w = bench.env_rank()
        bench.rank_barrier(world, "cpu")
        ms_local = 10.0 + 5.0 * rank          # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms_local, world, "cpu")
        value = bench.job_throughput(1000.0, world, ms_max)
        bench.rank_barrier(world, "cpu")
        # the reference arm: ranks other than 0 return at once, without work
        printed = None
        if rank != 0:
            import argparse
            printed = bench.run_reference(argparse.Namespace())
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"env": [r, lr, w], "ms_max": ms_max, "value": value, "ref": printed}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_and_throughput(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, x in enumerate(res):
        assert x["env"] == [r, r, world]
        assert x["ms_max"] == pytest.approx(15.0)       # the slowest rank's time
        # whole-job rate: units of both ranks over the slowest rank's time
        assert x["value"] == pytest.approx(world * 1000.0 / 0.015)
    assert res[1]["ref"] is None


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert bench.job_throughput(500.0, 1, 250.0) == pytest.approx(2000.0)
