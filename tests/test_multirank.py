"""The multi-GPU path's host logic, as two gloo ranks on the CPU (no GPU):
every rank builds its own batch (independent modules of the same size
distribution, so the job scales weakly), the step time is the maximum over
ranks, the job's throughput counts every rank's words, only rank 0 of the
reference arm prints, and a rank that fails raises on the host instead of
leaving the others waiting forever."""
import contextlib
import io
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port, timeout_s=60):
    import datetime
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=timeout_s))


def _rank_main(rank, world, port, out_dir):
    _init(rank, world, port)
    import bench
    w, off, cfg = bench.workload("batch", rank, 40)
    step_ms = 2.0 + rank                       # a slower rank 1
    (m_ms,) = bench.max_over_ranks([step_ms], world)
    e2e, serial = bench.max_over_ranks([10.0 * (rank + 1), 5.0 - rank], world)
    gbs = bench.job_gbs(world, len(w), m_ms)
    # the reference arm: only rank 0 prints its line
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0",
                                         "--modules", "3"]))
    dist.barrier()
    res = {"rank": rank, "words": int(len(w)), "first": [int(x) for x in w[:16]], "n_mod": len(off) - 1,
           "max_ms": m_ms, "e2e": e2e, "serial": serial, "gbs": gbs, "printed": buf.getvalue()}
    json.dump(res, open(os.path.join(out_dir, f"r{rank}.json"), "w"))
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(2)]
    # independent batches of the same shape
    assert r[0]["n_mod"] == r[1]["n_mod"] == 40
    assert r[0]["first"] != r[1]["first"]
    # the slowest rank's time, on every rank
    assert r[0]["max_ms"] == r[1]["max_ms"] == 3.0
    assert r[0]["e2e"] == r[1]["e2e"] == 20.0 and r[0]["serial"] == r[1]["serial"] == 5.0
    # whole-job throughput counts both ranks' words
    assert abs(r[0]["gbs"] - 2 * 4 * r[0]["words"] / 3.0e-3 / 1e9) < 1e-9
    # only rank 0 of the reference arm prints, one JSON line
    lines = r[0]["printed"].strip().splitlines()
    assert len(lines) == 1 and json.loads(lines[0])["impl"] == "reference"
    assert r[1]["printed"] == ""


def _leaving_rank(rank, world, port, out_dir):
    _init(rank, world, port, timeout_s=3)
    import bench
    if rank == 1:
        return                                  # leaves between steps, nothing in flight
    # rank 0 reaches the step-time reduction; the rank that left never does:
    # the process group ends the wait with an error on the host (its
    # timeout, or the lost connection), so rank 0 does not wait forever
    try:
        bench.max_over_ranks([1.0], world)
        outcome = "returned"
    except Exception as e:                      # noqa: BLE001
        outcome = type(e).__name__
    json.dump({"outcome": outcome}, open(os.path.join(out_dir, "r0.json"), "w"))


def test_a_rank_that_leaves_ends_the_others_wait_with_an_error(tmp_path):
    port = _free_port()
    mp.start_processes(_leaving_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = json.load(open(tmp_path / "r0.json"))
    assert r0["outcome"] != "returned"
