"""The N>1 path of bench.py on CPU: two ranks over gloo on 127.0.0.1.  The
replicas share no data; the process group carries the barriers around the
timed region and the max over ranks of the per-step times, and the whole-job
value counts every replica's work.  The reference arm runs on rank 0 only."""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    import time
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_env()
    bench.init_ranks(w, "gloo")
    # rank 1 is the slow replica: the barrier holds rank 0 until it arrives
    t0 = time.perf_counter()
    if r == 1:
        time.sleep(0.3)
    bench.rank_barrier(w)
    waited = time.perf_counter() - t0
    ms = [10.0 + 5.0 * r, 40.0 - 3.0 * r]
    mx = bench.max_over_ranks(ms, w)
    val = bench.whole_job_gflops(w, 2.0e9, mx[0])

    class A:
        gpus, steps, warmup = w, 1, 0
    ref = bench.run_reference(A()) if r != 0 else None  # rank 0 would run the 192^3 oracle: not here
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"env": [w, r, local], "waited": waited, "max": mx, "value": val, "ref": ref}, f)


def test_two_gloo_ranks_time_and_aggregate(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, d in enumerate(res):
        assert d["env"] == [world, r, r]
        # the max over ranks of each value, identical on both ranks
        assert d["max"] == [15.0, 40.0]
        # two replicas of 2 GFLOP each in 15 ms
        assert d["value"] == pytest.approx(2 * 2.0e9 / 15e-3 / 1e9)
    assert res[0]["waited"] >= 0.25  # rank 0 left the barrier only after rank 1 entered it
    assert res[1]["ref"] == 0  # the reference arm's other ranks exit 0 without work


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 1.0], 1) == [3.0, 1.0]
    bench.rank_barrier(1)
    bench.init_ranks(1, "gloo")
    import torch.distributed as dist
    assert not dist.is_initialized()
    assert bench.whole_job_gflops(1, 1e9, 1000.0) == pytest.approx(1.0)
