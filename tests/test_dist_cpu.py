"""The benchmark's multi-rank path on CPU: two gloo ranks in spawned
processes (127.0.0.1 rendezvous) run the same helpers bench.py uses under
torchrun -- process-group set-up, barrier, max-over-ranks timing -- and the
sharding of frames across ranks (no data-path collective: each rank forms its
own frames)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    r, w, local = bench._dist()
    backend = dist.get_backend()
    bench._barrier(w)
    ms = 10.0 * (rank + 1)               # the slower rank sets the job's time
    ms_max = bench._max_over_ranks(ms, w)
    q.put({"rank": r, "world": w, "backend": backend, "ms_max": ms_max,
           "seed": bench._workload_seed(r), "rate": bench.whole_job_rate(5, w, ms_max)})
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort(key=lambda d: d["rank"])
    assert [d["rank"] for d in out] == [0, 1]
    assert all(d["world"] == 2 and d["backend"] == "gloo" for d in out)
    assert all(d["ms_max"] == 20.0 for d in out)          # max over ranks
    assert out[0]["seed"] != out[1]["seed"]               # each rank its own frames
    assert out[0]["rate"] == pytest.approx(2 * 5 / 0.020)  # whole job: 10 frames in 20 ms


def test_single_rank_needs_no_process_group():
    import bench
    assert bench._max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(4, 1, 8.0) == pytest.approx(500.0)
