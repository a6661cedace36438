"""The N > 1 benchmark path on the host: two gloo ranks on 127.0.0.1 (no GPU).

The projections are independent, so bench.py runs one replica per rank with no collective on
the data path; the only cross-rank steps are the barrier around the timed region and the max of
the per-rank times. Checked here: every rank gets the maximum, the whole-job value counts every
rank's units over the slowest rank's time, and the reference arm prints only on rank 0.
"""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    local_ms = 10.0 * (rank + 1)              # rank 1 is the slow one
    total = bench.max_over_ranks(local_ms, world)
    value = bench.job_value(1000, 5, total, world)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"total": total, "value": value}, f)


def test_two_gloo_ranks(tmp_path):
    world = 2
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["total"] == 20.0                             # max over ranks, on every rank
        assert r["value"] == pytest.approx(2 * 1000 * 5 / 0.020)   # all ranks' units / slowest time


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_value(100, 10, 1000.0, 1) == pytest.approx(1000.0)


def test_reference_arm_silent_off_rank_zero(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup, gpus = 1, 1, 2
    bench.run_reference(Args(), rank=1)
    assert capsys.readouterr().out == ""
