"""The N > 1 path of the benchmark on CPU: two gloo ranks on 127.0.0.1.

Several GPUs run independent replicas (one per rank, seeded with the rank);
the only cross-rank steps are the start/stop barriers and the reduction of
the throughput (units summed, time = the slowest rank).  Both are checked
here with world_size 2 over gloo, without a GPU.
"""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    r, w, local = bench.dist_info()
    dist = bench.dist_init(w, local, "gloo")
    units = 1000.0 * (rank + 1)
    secs = 0.5 + rank
    dist.barrier()
    tot, mx = bench.aggregate(dist, units, secs)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"rank": r, "world": w, "units": tot, "secs": mx}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks(tmp_path):
    port = free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, d in enumerate(res):
        assert d["rank"] == r and d["world"] == 2
        assert d["units"] == 3000.0      # whole-job units: summed over ranks
        assert d["secs"] == 1.5          # whole-job time: the slowest rank


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_init(1, 0, "gloo") is None
    assert bench.aggregate(None, 5.0, 2.0) == (5.0, 2.0)


def test_rank_replicas_are_independent_systems():
    sys.path.insert(0, ROOT)
    import bench
    a, b = bench.rank_spec("slab_16m", 0), bench.rank_spec("slab_16m", 1)
    assert a.seed == 0 and b.seed == 1
    assert a.box == b.box and a.rho_l == b.rho_l and a.wave_amp == b.wave_amp


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "0"])) == 0
    assert capsys.readouterr().out == ""
