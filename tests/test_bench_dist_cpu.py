"""The multi-rank host logic of bench.py on CPU ranks (gloo, world size 2):
day sharding gives every rank its own disjoint days (weak scaling) and the
step time is the maximum over ranks.  No GPU is involved."""
import os
import socket

import pytest


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist = bench.dist_init("gloo")
    days = bench.shard_days(10, rank, world)
    t = bench.dist_max(1.5 + rank)
    bench.dist_barrier()
    out[rank] = (days, t)
    dist.destroy_process_group()


def test_two_rank_sharding_and_max_time():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    d0, t0 = out[0]
    d1, t1 = out[1]
    assert d0 == list(range(0, 10)) and d1 == list(range(10, 20))
    assert set(d0).isdisjoint(d1)
    assert t0 == t1 == 2.5


def test_algorithmic_bytes_of_the_3yr_corridor():
    import bench
    # counts 4*288*400 + mask 288*400/8 + ticks 2*288*438 + q 8*288*150 + G 8*288*150 + 8
    assert bench.algorithmic_bytes(288, 400, 438, 150) == 460800 + 14400 + 252288 + 345600 + 345600 + 8


def test_measured_traffic_only_for_the_profiled_kernel(tmp_path, monkeypatch):
    """The ncu figures are reported only for the form, workload, precision and
    kernel source they were taken of (the source matched by its hash)."""
    import hashlib

    import bench
    src = tmp_path / "paper_1901_09266_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    kernel = b"// a kernel source\n"
    (src / "fused.cu").write_bytes(kernel)
    (tmp_path / "profiles" / "fused_kernel_fp32_corridor-3yr-152d_traffic.txt").write_text(
        "# a capture\n"
        "kernel = k_fused<0,1,1> (FP32 form)\n"
        "form = fused\n"
        "workload = corridor-3yr\n"
        "precision = fp32\n"
        "source = paper_1901_09266_gb300/csrc/fused.cu\n"
        f"source_sha256_16 = {hashlib.sha256(kernel).hexdigest()[:16]}\n"
        "bytes_per_day_iteration = 4398377\n"
        "warp_instructions_per_day_iteration = 3304333\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("fused", "corridor-3yr", "fp32") == 4398377.0
    assert bench.measured_traffic("fused", "corridor-3yr", "fp32", "warp_instructions_per_day_iteration") == 3304333.0
    assert bench.measured_traffic("fused", "corridor-3yr", "bf16") is None
    assert bench.measured_traffic("plain", "corridor-3yr", "fp32") is None
    assert bench.measured_traffic("fused", "corridor-large", "fp32") is None
    (src / "fused.cu").write_bytes(kernel + b"// changed\n")
    assert bench.measured_traffic("fused", "corridor-3yr", "fp32") is None


def test_clock_sampler_reads_clocks_and_throttle_reasons(tmp_path, monkeypatch):
    """The sampler's parsing, against a fake nvidia-smi that prints three samples
    (one with the power cap active) and a malformed line."""
    import time

    import bench
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "echo '2070, 2070, 1400.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo 'not a sample'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ.get('PATH', '')}")
    s = bench.ClockSampler()
    s.start()
    t0 = time.time()
    while len(s.lines) < 4 and time.time() - t0 < 10:
        time.sleep(0.05)
    r = s.stop()
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    empty = tmp_path / "empty"
    empty.mkdir()
    monkeypatch.setenv("PATH", str(empty))
    s = bench.ClockSampler()
    s.start()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]
