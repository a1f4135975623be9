"""bench.py's multi-rank path on CPU: two ranks over gloo (one process per
GPU on a real node; each renders its own frames, so the only cross-rank steps
are the barrier around the timed region and the max of the ranks' times).
The whole-job rate is the units all ranks processed over the slowest rank's
time."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    os.environ.update({"WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "GS_BENCH_BACKEND": "gloo"})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_init()
    bench.barrier(w)
    # Rank r "took" 10 (r + 1) ms for its 100 frames.
    ms = bench.max_over_ranks(10.0 * (r + 1), w)
    rate = bench.whole_job_rate(100, ms, w)
    bench.barrier(w)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"world": w, "rank": r, "local": local, "backend": dist.get_backend(),
                   "max_ms": ms, "rate": rate}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest_time_and_whole_job_rate(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, d in enumerate(res):
        assert d["world"] == world and d["rank"] == r and d["local"] == r
        assert d["backend"] == "gloo"
        assert d["max_ms"] == 20.0          # the slowest rank's time, on every rank
        assert d["rate"] == pytest.approx(100 * world / 0.020)


def test_single_rank_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_init() == (1, 0, 0)
    bench.barrier(1)
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10, 5.0, 1) == pytest.approx(2000.0)
