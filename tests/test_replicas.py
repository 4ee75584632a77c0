"""The multi-GPU path of the benchmark is replicas only: each rank registers
its own case and the ranks exchange nothing but the timing maximum.  Checked
here with world-size-2 gloo process groups on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import phantom
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        idx = bench.replica_case_index(r)
        case = phantom.make_case("phantom64", index=idx, shape=(8, 16, 16))
        local_ms = 10.0 * (r + 1)                      # rank 1 is the slow one
        mx = bench.reduce_max(local_ms)
        value = bench.whole_job_value(w, 1000, 5, mx)
        out[r] = (w, r, local, idx, float(case.moving.sum()), mx, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_time_by_the_slowest_rank_and_use_their_own_cases():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    a, b = out[0], out[1]
    assert (a[0], a[1], a[2]) == (2, 0, 0) and (b[0], b[1], b[2]) == (2, 1, 1)
    assert a[3] != b[3] and a[4] != b[4]               # different seeded cases
    assert a[5] == b[5] == 20.0                        # max over ranks
    assert a[6] == b[6] == pytest.approx(2 * 1000 * 5 / 0.020)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, gpus = 1, 0, 2
    assert bench.run_reference(Args()) == 0            # returns at once, no oracle work


def test_single_process_reduce_is_identity():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.whole_job_value(1, 206438400, 10, 1000.0) == pytest.approx(2.064384e9)


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on a bounded sample, host
    cores only) prints one JSON line with the contract's keys."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "headneck256",
                        "--steps", "1", "--warmup", "0"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["unit"] == line["unit"]
