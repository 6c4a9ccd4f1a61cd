"""Benchmark of the per-day DODE SPGD solve (Ma & Qian, arXiv 1901.09266, Algorithm 1).

One step = the whole hot path over the full synthetic workload: load the days
(tick table, route times: ``dode_set_days``) and run ``--epochs`` SPGD epochs on
every day (``dode_solve``).  Metric: SPGD day-iterations per second (one
day-iteration = one full-row Adagrad update of one day), whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Default workload: the 3-year corridor (1096 days x 288 five-minute intervals,
150 OD pairs, 300 routes, 400 detectors, 10 % missing), 500 epochs per step,
fused form in FP32 (the paper's precision).  Inputs (~1.3 GB) exceed the
129 MB L2, and every step reloads them.  Beside it, untimed by the step clock:
the plain FP32, fused FP32 and fused BF16 forms at --compare-epochs epochs; the
uneven-day workload over 1 .. 1096 days per launch (autotuned, direct and
graph); the next rows; and the loss-and-gradient form on all 1096 days of the
600-OD corridor in both precisions.

Under torchrun (N > 1) each rank solves its own 1096 days (weak scaling, days
d + 1096 * rank of the same generator); ranks exchange only the timing.
``--impl reference`` times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# algorithmic bytes of one day-iteration (DAR recomputed on chip, never stored):
# counts 4 N O + bit mask N O / 8 + uint16 tick table 2 N A + q read+write
# 8 N K + Adagrad accumulator read+write 8 N K + per-day loss 8
def algorithmic_bytes(N: int, O: int, A: int, K: int) -> int:
    """Bytes one day-iteration must move at least: counts, mask bits, uint16 ticks, q and G read and
    written, and the day's loss."""
    return 4 * N * O + (N * O) // 8 + 2 * N * A + 8 * N * K + 8 * N * K + 8


def shard_days(n_days: int, rank: int, world: int) -> list:
    """Weak scaling: every rank owns a full set of n_days distinct days."""
    return list(range(rank * n_days, (rank + 1) * n_days))


def measured_traffic(form: str, workload: str, precision: str, key: str = "bytes_per_day_iteration"):
    """Per day-iteration figure ``key`` (DRAM bytes, or warp instructions) of one
    form of the solve, from the committed ncu summaries (profiles/*_traffic.txt),
    if one was taken of this form, workload and precision and of the kernel
    source as it is now (matched by hash); else None."""
    import glob
    import hashlib
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*_traffic.txt"))):
        rec = {}
        try:
            for line in open(path):
                if "=" in line and not line.startswith("#"):
                    k, v = line.split("=", 1)
                    rec[k.strip()] = v.strip()
        except OSError:
            continue
        if (rec.get("form"), rec.get("workload"), rec.get("precision")) != (form, workload, precision):
            continue
        try:
            src = open(os.path.join(ROOT, rec.get("source", "")), "rb").read()
        except OSError:
            continue
        if hashlib.sha256(src).hexdigest()[:16] != rec.get("source_sha256_16"):
            continue
        if key in rec:
            return float(rec[key])
    return None


def _peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0):
        self.index = index
        self.proc = None
        self.lines: list = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed plumbing (torchrun); CPU-testable with gloo
# ---------------------------------------------------------------------------

def dist_env():
    """(world size, rank, local rank) from the torchrun environment; (1, 0, 0) without it."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(backend: str):
    """Join the process group of a multi-rank run; the rendezvous address comes from the environment
    (MASTER_ADDR / MASTER_PORT, set by torchrun)."""
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def dist_barrier():
    """Barrier across ranks; a no-op on one rank."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def dist_max(x: float) -> float:
    """The maximum of x over ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_workload(name: str, n_days: int):
    """The seeded synthetic workload called `name` with `n_days` days."""
    from paper_1901_09266_gb300 import synth
    if name == "corridor-3yr":
        return synth.corridor_3yr(n_days=n_days)
    if name == "corridor-uneven":
        return synth.corridor_uneven(n_days=n_days)
    if name == "corridor-large":
        return synth.corridor_large(n_days=n_days)
    if name == "corridor-7d":
        return synth.corridor_7day()
    raise SystemExit(f"unknown workload {name}")


def gpu_inputs(w, days):
    """Speeds, noisy counts (B q_true with the library's own FP32 forward map) and mask."""
    from paper_1901_09266_gb300 import dode
    sp = w.speeds(days)
    mask = w.mask(days)
    qt = w.q_true(days)
    ctx = dode.Context.from_workload(w)
    ctx.set_days(np.zeros((len(days), w.n_intervals, w.net.n_obs), np.float32), sp, mask)
    x = ctx.forward(qt)
    ctx.close()
    counts = w.counts_from(x, days)
    return sp, counts, mask


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

_ORACLE_INPUTS: dict = {}


def oracle_rate(w, days, epochs: int, threads: int):
    """The FP64 oracle's day-iterations per second on these days (inputs built
    once per process and not timed)."""
    from oracle import oracle as orc
    key = (w.name, w.n_days, tuple(days))
    if key not in _ORACLE_INPUTS:
        net = orc.Net.from_workload(w)
        sp = w.speeds(days)
        x = net.forward_days(sp, w.q_true(days).astype(np.float64), n_threads=threads)
        _ORACLE_INPUTS[key] = (net, sp, w.counts_from(x, days), w.mask(days))
    net, sp, counts, mask = _ORACLE_INPUTS[key]
    t0 = time.perf_counter()
    net.solve_days(sp, counts, mask, iters=epochs, eta=5.0, n_threads=threads, day_ids=np.asarray(days))
    dt = time.perf_counter() - t0
    return len(days) * epochs / dt, dt


def run_reference(args):
    """The reference arm: the FP64 oracle, unmodified, timed on the host cores on a bounded sample."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = make_workload(args.workload, args.days)
    threads = os.cpu_count() or 1
    days = list(range(min(args.ref_days, w.n_days)))
    for _ in range(args.warmup):
        oracle_rate(w, days[:threads], 1, threads)
    rates, times = [], []
    for _ in range(args.steps):
        r, dt = oracle_rate(w, days, args.ref_epochs, threads)
        rates.append(r)
        times.append(dt)
    value = float(np.median(rates))
    sample = f"{len(days)} days x {args.ref_epochs} epochs of {w.name} per step, FP64, OpenMP over days"
    line = {
        "impl": "reference", "metric": "SPGD day-iterations/sec", "value": value, "unit": "day-iter/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.median(times)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "days": w.n_days, "epochs_per_step": args.ref_epochs},
        "cpu_baseline": {"value": value, "unit": "day-iter/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "day-iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    """This library's arm: the timed solve, end-to-end and comparison runs, one JSON line on rank 0."""
    import torch
    from paper_1901_09266_gb300 import build, dode, synth

    world, rank, local = dist_env()
    if world > 1:
        dist_init("nccl")
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    w = make_workload(args.workload, args.days)
    days = shard_days(w.n_days, rank, world)
    prec = dode.PREC_BF16 if args.precision == "bf16" else dode.PREC_FP32
    form = dode.FORM_PLAIN if args.form == "plain" else dode.FORM_FUSED
    ctx = dode.Context.from_workload(w, form=form, precision=prec, use_graph=1 if args.graph else 0,
                                     row_chunk=args.row_chunk, day_base=days[0])
    ctx.use_torch_stream()
    sp, counts, mask = gpu_inputs(w, days)
    tuned = None
    if args.autotune:
        from paper_1901_09266_gb300 import autotune
        ctx.set_days(counts, sp, mask)
        tuned = autotune.tune(ctx, iters=3, step=args.step)
        tuned = {k: tuned[k] for k in ("block", "ctas_per_sm", "max_ctas", "ms", "cached")}
    elif args.block or args.ctas:
        ctx.set_launch(args.block, args.ctas)
    D, N, K, O, A = len(days), w.n_intervals, w.routes.n_od, w.net.n_obs, w.net.n_links
    # device-resident inputs and outputs
    sp_d = torch.from_numpy(sp).to(dev)
    ct_d = torch.from_numpy(counts).to(dev)
    mk_d = torch.from_numpy(mask).to(dev)
    q_d = torch.empty((D, N, K), dtype=torch.float32, device=dev)
    l_d = torch.empty(D, dtype=torch.float64, device=dev)
    E = args.epochs

    def step_device():
        ctx.set_days(ct_d, sp_d, mk_d)
        ctx.solve(E, args.step, args.batch, q_out=q_d, loss_out=l_d)

    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()
    dist_barrier()
    launches0 = ctx.total_launches()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    dist_barrier()
    e0.record()
    kern_ms = []
    for _ in range(args.steps):
        step_device()
        kern_ms.append(ctx.last_kernel_ms())
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    dist_barrier()
    ms = e0.elapsed_time(e1)
    ms = dist_max(ms)
    launches = (ctx.total_launches() - launches0) // max(1, args.steps)
    units = D * E * args.steps * world
    value = units / (ms / 1e3)
    final_loss = float(l_d.double().sum().item())

    # end to end: pinned host buffers through the same calls
    sp_h = torch.from_numpy(sp).pin_memory()
    ct_h = torch.from_numpy(counts).pin_memory()
    mk_h = torch.from_numpy(mask).pin_memory()
    q_h = torch.empty((D, N, K), dtype=torch.float32).pin_memory()
    l_h = torch.empty(D, dtype=torch.float64).pin_memory()
    sp_n, ct_n, mk_n, q_n, l_n = sp_h.numpy(), ct_h.numpy(), mk_h.numpy(), q_h.numpy(), l_h.numpy()

    def step_host():
        # this step's inputs were copied during the previous step's solve
        # (dode_prefetch_days); the next step's are copied during this one
        ctx.set_days(ct_n, sp_n, mk_n)
        ctx.prefetch_days(ct_n, sp_n, mk_n)
        ctx.solve(E, args.step, args.batch, q_out=q_n, loss_out=l_n)

    e2e_value = None
    e2e_clk = None
    if args.e2e_steps > 0:
        step_host()
        torch.cuda.synchronize()
        dist_barrier()
        clocks_e2e = ClockSampler(local)
        clocks_e2e.start()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            step_host()
        torch.cuda.synchronize()
        e2e_s = dist_max(time.perf_counter() - t0)
        e2e_clk = clocks_e2e.stop()
        e2e_value = D * E * args.e2e_steps * world / e2e_s
    h2d = sp.nbytes + counts.nbytes + mask.nbytes
    d2h = q_n.nbytes + l_n.nbytes

    # roofline of the fused kernel (algorithmic bytes / CUDA-event duration)
    peaks = _peaks()
    peak = peaks.get("hbm_gbs")
    per_unit = algorithmic_bytes(N, O, A, K)
    kms = float(np.mean(kern_ms))
    achieved = per_unit * D * E / (kms / 1e3) / 1e9
    form_name = "plain" if form == dode.FORM_PLAIN else "fused"
    traffic, traffic_src = args.traffic, "command line" if args.traffic is not None else None
    if traffic is None:
        per = measured_traffic(form_name, w.name, args.precision)
        if per is not None:
            traffic = per * D * E
            traffic_src = (f"ncu dram__bytes_read+write of a 152-day capture of this {form_name} {args.precision} "
                           "kernel source, scaled by day-iterations (profiles/*_traffic.txt)")
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak if peak else 6800.0, "unit": "GB/s",
            "frac": achieved / (peak if peak else 6800.0), "traffic": traffic, "traffic_source": traffic_src,
            "peak_source": "measured" if peak else "fallback", "bytes_per_unit": per_unit,
            "kernel_ms": kms}

    # instruction-issue roofline: measured warp instructions per day-iteration x
    # day-iterations/s of the kernel against 4 issue slots per SM per cycle at the
    # sampled clock
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz") or 2070.0

    def issue_roof(form_key, precision, di_per_s):
        ipu = measured_traffic(form_key, w.name, precision, "warp_instructions_per_day_iteration")
        if ipu is None:
            return None
        peak_issue = n_sm * 4 * mhz * 1e6
        return {"bound": "issue", "achieved": ipu * di_per_s, "peak": peak_issue, "unit": "warp-instr/s",
                "frac": ipu * di_per_s / peak_issue, "instr_per_unit": ipu,
                "source": "ncu smsp__inst_executed.sum of a 152-day capture of this kernel source"}

    issue = issue_roof(form_name, args.precision, D * E / (kms / 1e3))

    # comparison forms at equal epochs from q = 0: plain FP32, fused FP32 and
    # fused BF16, each with its measured DRAM bytes per day-iteration (ncu
    # summary of the same kernel source) and the DRAM rate they imply
    forms = {}
    if args.compare_epochs > 0 and rank == 0:
        for name, fm, pr, fk, pk in [("plain_fp32", dode.FORM_PLAIN, dode.PREC_FP32, "plain", "fp32"),
                                     ("fused_fp32", dode.FORM_FUSED, dode.PREC_FP32, "fused", "fp32"),
                                     ("fused_bf16", dode.FORM_FUSED, dode.PREC_BF16, "fused", "bf16")]:
            c2 = dode.Context.from_workload(w, form=fm, precision=pr)
            c2.use_torch_stream()
            c2.set_days(ct_d, sp_d, mk_d)
            c2.solve(1, args.step, args.batch, q_out=q_d, loss_out=l_d)          # warm-up (and plain DAR build)
            c2.set_days(ct_d, sp_d, mk_d)
            if fm == dode.FORM_PLAIN:
                c2.solve(0, args.step, args.batch, q_out=q_d, loss_out=l_d)      # rebuild DAR outside the timing
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            c2.solve(args.compare_epochs, args.step, args.batch, q_out=q_d, loss_out=l_d)
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 1e3
            rate = D * args.compare_epochs / t
            mb = measured_traffic(fk, w.name, pk)
            pk_gbs = peak if peak else 6800.0
            forms[name] = {"day_iter_per_s": rate, "final_loss": float(l_d.double().sum().item()),
                           "kernel_ms": c2.last_kernel_ms(), "launches": c2.last_launches(),
                           "roofline": {"bound": "hbm", "achieved": per_unit * rate / 1e9, "peak": pk_gbs,
                                        "unit": "GB/s", "frac": per_unit * rate / 1e9 / pk_gbs,
                                        "bytes_per_unit": per_unit},
                           "measured_bytes_per_day_iter": mb,
                           "measured_dram_gbs": (mb * rate / 1e9) if mb is not None else None,
                           "issue_roofline": issue_roof(fk, pk, rate)}
            c2.close()
        base = forms["plain_fp32"]
        for v in forms.values():
            v["speedup_vs_plain_fp32"] = v["day_iter_per_s"] / base["day_iter_per_s"]
            v["final_loss_rel_diff_vs_plain"] = abs(v["final_loss"] - base["final_loss"]) / base["final_loss"]
        f32, f16 = forms["fused_fp32"], forms["fused_bf16"]
        forms["bf16_vs_fp32"] = {
            "day_iter_per_s_ratio": f16["day_iter_per_s"] / f32["day_iter_per_s"],
            "measured_bytes_ratio": (f16["measured_bytes_per_day_iter"] / f32["measured_bytes_per_day_iter"]
                                     if f16["measured_bytes_per_day_iter"] and f32["measured_bytes_per_day_iter"]
                                     else None),
            "final_loss_rel_diff": abs(f16["final_loss"] - f32["final_loss"]) / f32["final_loss"]}

    # uneven days (per-day observed subsets, missing rates U(0, 30 %)) in one
    # persistent launch, the launch shape picked by the autotuner, direct
    # launches against CUDA-graph replay, for days per launch swept over 1 .. 1096
    uneven_sweep = None
    if args.uneven_sweep and rank == 0:
        from paper_1901_09266_gb300 import autotune
        wu = make_workload("corridor-uneven", max(args.uneven_days))
        du = list(range(max(args.uneven_days)))
        spu, ctu, mku = gpu_inputs(wu, du)
        spu_d, ctu_d, mku_d = (torch.from_numpy(a).to(dev) for a in (spu, ctu, mku))
        points = []
        for n in args.uneven_days:
            pt_ = {"days": n}
            qn = torch.empty((n, N, K), dtype=torch.float32, device=dev)
            ln = torch.empty(n, dtype=torch.float64, device=dev)
            for graph in (0, 1):
                cu = dode.Context.from_workload(wu, precision=prec, use_graph=graph)
                cu.use_torch_stream()
                cu.set_days(ctu_d[:n], spu_d[:n], mku_d[:n])
                tuned_u = autotune.tune(cu, iters=3, step=args.step, n_sm=n_sm, cache_path=None)
                cu.set_days(ctu_d[:n], spu_d[:n], mku_d[:n])
                cu.solve(args.uneven_epochs, args.step, args.batch, q_out=qn, loss_out=ln)     # warm-up / capture
                cu.set_days(ctu_d[:n], spu_d[:n], mku_d[:n])
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                cu.solve(args.uneven_epochs, args.step, args.batch, q_out=qn, loss_out=ln)
                b.record()
                torch.cuda.synchronize()
                t = a.elapsed_time(b) / 1e3
                pt_["graph" if graph else "direct"] = {
                    "day_iter_per_s": n * args.uneven_epochs / t, "call_ms": t * 1e3,
                    "kernel_ms": cu.last_kernel_ms(), "grid": cu.last_grid(),
                    "epoch_slices": cu.last_slices(),
                    "shape": {k: tuned_u[k] for k in ("block", "ctas_per_sm", "max_ctas")},
                    "final_loss": float(ln.double().sum().item())}
                cu.close()
            points.append(pt_)
        uneven_sweep = {"workload": wu.name, "epochs": args.uneven_epochs, "precision": args.precision,
                   "observed_links_per_day": [int(x) for x in (mku.reshape(len(du), N, O).any(axis=1).sum(axis=1)
                                                               [[0, -1]])],
                   "points": points}
        del spu_d, ctu_d, mku_d

    # next rows on the same days: pattern-level route choice (weekday / weekend /
    # holiday labels), the R^2 quality check and the DAR distance to the mean DAR
    nxt = None
    if args.next_rows and rank == 0:
        nxt = {}
        c3 = dode.Context.from_workload(w, precision=prec)
        c3.use_torch_stream()
        c3.set_days(ct_d, sp_d, mk_d)
        labels = np.array([synth.day_type(w, d) for d in days], np.int32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c3.set_patterns(labels)
        torch.cuda.synchronize()
        nxt["set_patterns_ms"] = (time.perf_counter() - t0) * 1e3
        c3.solve(args.compare_epochs, args.step, args.batch, q_out=q_d, loss_out=l_d)
        nxt["pattern_solve"] = {"day_iter_per_s": D * args.compare_epochs / (c3.last_kernel_ms() / 1e3),
                                "epochs": args.compare_epochs, "patterns": int(len(set(labels.tolist())))}
        r2_d = torch.empty(D, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c3.r2(q_d, r2_out=r2_d)
        torch.cuda.synchronize()
        r2 = r2_d.cpu().numpy()
        nxt["r2"] = {"ms": (time.perf_counter() - t0) * 1e3, "mean": float(np.nanmean(r2)),
                     "after_epochs": args.compare_epochs}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dist, msq = c3.dar_distance()
        ms_d = (time.perf_counter() - t0) * 1e3
        nxt["dar_distance"] = {"ms": ms_d, "days": D, "mean_dist": float(dist.mean()),
                               "rel_to_mean_norm": float(dist.mean() / np.sqrt(msq))}
        c3.close()
        # consecutive days solved jointly (trips that cross midnight count on the
        # next day): every epoch adds a halo pass over the first and last phases
        c4 = dode.Context.from_workload(w, precision=prec, couple_days=1)
        c4.use_torch_stream()
        c4.set_days(ct_d, sp_d, mk_d)
        c4.solve(1, args.step, args.batch, q_out=q_d, loss_out=l_d)           # warm-up
        c4.set_days(ct_d, sp_d, mk_d)
        c4.solve(args.compare_epochs, args.step, args.batch, q_out=q_d, loss_out=l_d)
        kms = c4.last_kernel_ms()
        nxt["coupled"] = {"day_iter_per_s": D * args.compare_epochs / (kms / 1e3), "epochs": args.compare_epochs,
                          "launches": c4.last_launches(), "final_loss": float(l_d.double().sum().item())}
        c4.close()
        # the paper's efficiency experiment at its largest size: dense random
        # n x n NNLS by Algorithm 1, one pass over B (4 n^2 bytes) per iteration
        n = args.dense_n
        rng = np.random.default_rng(1901)
        Bh = (rng.standard_normal((n, n), dtype=np.float32) / np.float32(np.sqrt(n)))
        xt = np.abs(rng.standard_normal((n, 1))).astype(np.float32)
        Bd = torch.from_numpy(Bh).to(dev)
        Yd = Bd @ torch.from_numpy(xt).to(dev)
        dode.dense_nnls(Bd, Yd, 3, 0.05)                                   # warm-up
        _, _, ld, ms_dense = dode.dense_nnls(Bd, Yd, args.dense_iters, 0.05)
        per = ms_dense / (args.dense_iters + 1)                           # + the final residual pass (one more pass over B)
        nxt["dense_nnls"] = {"n": n, "m": 1, "iters": args.dense_iters, "ms_per_iter": per,
                             "roofline": {"bound": "hbm", "achieved": 4.0 * n * n / (per / 1e3) / 1e9,
                                          "peak": peaks.get("hbm_gbs") or 6800.0, "unit": "GB/s",
                                          "frac": 4.0 * n * n / (per / 1e3) / 1e9 / (peaks.get("hbm_gbs") or 6800.0),
                                          "bytes_per_iter": 4 * n * n, "method": "one pass over B"},
                             "final_loss": float(ld.sum().item())}
        # many right-hand sides sharing B: the two products as TF32 GEMMs on the
        # tensor cores (method 3); each iteration reads B and its transpose once
        tc = []
        for m_tc in args.dense_tc_m:
            Xs = np.abs(rng.standard_normal((n, m_tc))).astype(np.float32)
            Yt = Bd @ torch.from_numpy(Xs).to(dev)
            dode.dense_nnls(Bd, Yt, 2, 0.05, method=3)                    # warm-up
            _, _, lt, ms_tc = dode.dense_nnls(Bd, Yt, args.dense_iters, 0.05, method=3)
            per_tc = ms_tc / (args.dense_iters + 0.5)                      # + the final residual GEMM
            flops = 4.0 * n * n * m_tc
            pk_tf = (peaks.get("bf16_tflops") or 1900.0) / 2.0          # TF32 = half the BF16 rate (nominal ratio)
            tc.append({"m": m_tc, "ms_per_iter": per_tc, "tflops": flops / (per_tc / 1e3) / 1e12,
                       "roofline": {"bound": "hbm", "achieved": 8.0 * n * n / (per_tc / 1e3) / 1e9,
                                    "peak": peaks.get("hbm_gbs") or 6800.0, "unit": "GB/s",
                                    "frac": 8.0 * n * n / (per_tc / 1e3) / 1e9 / (peaks.get("hbm_gbs") or 6800.0),
                                    "bytes_per_iter": 8 * n * n, "method": "B and B^T once each (TF32 GEMMs)"},
                       "tensor_roofline": {"bound": "tensor", "achieved": flops / (per_tc / 1e3) / 1e12,
                                           "peak": pk_tf, "unit": "TFLOP/s",
                                           "frac": flops / (per_tc / 1e3) / 1e12 / pk_tf,
                                           "peak_source": "measured bf16 burst x nominal tf32/bf16 ratio 1/2"},
                       "right_hand_side_iters_per_s": m_tc / (per_tc / 1e3),
                       "final_loss": float(lt.sum().item())})
        nxt["dense_nnls"]["tensor_cores"] = tc
        del Bd, Yd

    # the differentiable loss and gradients on the 600-OD / 1500-route / 1000-detector corridor:
    # loss and gradients (dL/dq, dL/dtheta) of every day, DAR recomputed in both
    # passes, in FP32 and BF16
    loss_grad_large = None
    if args.loss_grad_days > 0 and rank == 0:
        w5 = make_workload("corridor-large", args.loss_grad_days)
        d5 = list(range(args.loss_grad_days))
        sp5, ct5, mk5 = gpu_inputs(w5, d5)
        sp5_d, ct5_d, mk5_d = (torch.from_numpy(a).to(dev) for a in (sp5, ct5, mk5))
        q5 = torch.from_numpy(w5.q_true(d5) * np.float32(0.9)).to(dev)
        dq5 = torch.empty_like(q5)
        N5, O5, A5, K5 = w5.n_intervals, w5.net.n_obs, w5.net.n_links, w5.routes.n_od
        # bytes one loss+gradient pass of a day must move: counts, mask bits,
        # uint16 ticks, q read, dL/dq written, loss and dL/dtheta
        per5 = 4 * N5 * O5 + (N5 * O5) // 8 + 2 * N5 * A5 + 4 * N5 * K5 + 4 * N5 * K5 + 16
        loss_grad_large = {"workload": w5.name, "days": len(d5), "routes": w5.routes.n_routes, "od_pairs": K5,
                 "detectors": O5, "bytes_per_day_pass": per5}
        res5 = {}
        for pname, pr in (("fp32", dode.PREC_FP32), ("bf16", dode.PREC_BF16)):
            c5 = dode.Context.from_workload(w5, precision=pr)
            c5.use_torch_stream()
            c5.set_days(ct5_d, sp5_d, mk5_d)
            c5.loss_grad(q5, 0.1, dq_out=dq5)                     # warm-up
            ms5 = []
            for _ in range(3):
                loss5, _, dth5 = c5.loss_grad(q5, 0.1, dq_out=dq5)
                ms5.append(c5.last_kernel_ms())
            t5 = min(ms5) / 1e3
            res5[pname] = (np.asarray(loss5, np.float64), dq5.detach().cpu().numpy().astype(np.float64),
                           np.asarray(dth5, np.float64))
            pk_gbs = peak if peak else 6800.0
            loss_grad_large[pname] = {"kernel_ms": t5 * 1e3, "day_loss_grads_per_s": len(d5) / t5,
                            "roofline": {"bound": "hbm", "achieved": per5 * len(d5) / t5 / 1e9, "peak": pk_gbs,
                                         "unit": "GB/s", "frac": per5 * len(d5) / t5 / 1e9 / pk_gbs},
                            "total_loss": float(np.sum(loss5)), "dtheta_total": float(np.sum(dth5))}
            c5.close()
        (l32, g32, t32), (l16, g16, t16) = res5["fp32"], res5["bf16"]
        loss_grad_large["bf16_vs_fp32"] = {
            "loss_max_rel": float(np.max(np.abs(l16 - l32) / np.abs(l32))),
            "dq_max_rel_norm": float(np.max(np.sqrt(((g16 - g32) ** 2).sum(axis=(1, 2)) / (g32 ** 2).sum(axis=(1, 2))))),
            "dtheta_max_rel": float(np.max(np.abs(t16 - t32) / np.abs(t32)))}
        del q5, dq5, sp5_d, ct5_d, mk5_d

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        cd = list(range(min(args.ref_days, w.n_days)))
        r, dt = oracle_rate(w, cd, args.ref_epochs, threads)
        cpu = {"value": r, "unit": "day-iter/s", "cores": threads, "kind": "oracle",
               "sample": f"{len(cd)} days x {args.ref_epochs} epochs of {w.name}, FP64, OpenMP over days ({dt:.1f} s)"}

    if rank == 0:
        line = {
            "metric": "SPGD day-iterations/sec", "value": value, "unit": "day-iter/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if prec == dode.PREC_BF16 else "f32", "data": "synthetic",
            "config": {"workload": w.name, "days_per_gpu": D, "intervals": N, "od_pairs": K,
                       "routes": w.routes.n_routes, "links": A, "detectors": O, "epochs_per_step": E,
                       "form": args.form, "precision": args.precision, "graph": bool(args.graph),
                       "row_chunk": args.row_chunk, "epoch_slices": ctx.last_slices(),
                       "launch": tuned or {"block": args.block, "ctas_per_sm": args.ctas},
                       "l2": "inputs larger than L2 (reloaded every step)"},
            "e2e": {"value": e2e_value, "unit": "day-iter/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "clocks": e2e_clk,
                    "overlap": "each step's host-to-device input copy runs during the previous step's solve "
                               "(dode_prefetch_days)"},
            "gpu_launches": int(launches),
            "roofline": roof,
            "issue_roofline": issue,
            "cpu_baseline": cpu,
            "clocks": clk,
            "forms": forms,
            "next": nxt,
            "uneven_sweep": uneven_sweep,
            "loss_grad_large": loss_grad_large,
            "final_loss_total": final_loss,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    """Parse the arguments and run one arm."""
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="corridor-3yr")
    ap.add_argument("--days", type=int, default=1096)
    ap.add_argument("--epochs", type=int, default=500)
    ap.add_argument("--step", type=float, default=5.0)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--row-chunk", type=int, default=0,
                    help="Algorithm 1's row batch b (0 = all observed rows in each update)")
    ap.add_argument("--form", default="fused", choices=["fused", "plain"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"])
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--ctas", type=int, default=0)
    ap.add_argument("--graph", action="store_true", help="replay the solve as a CUDA graph")
    ap.add_argument("--autotune", action="store_true", help="pick the launch shape with the autotuner")
    ap.add_argument("--compare-epochs", type=int, default=20)
    ap.add_argument("--next-rows", type=int, default=1, help="time the pattern, R^2, DAR-distance and dense rows")
    ap.add_argument("--loss-grad-days", type=int, default=1096,
                    help="days of the corridor-large loss+gradient timing (0 = skip)")
    ap.add_argument("--uneven-sweep", type=int, default=1,
                    help="time the uneven-day workload over --uneven-days days per launch (0 = skip)")
    ap.add_argument("--uneven-days", type=lambda v: [int(x) for x in v.split(",")],
                    default=[1, 2, 8, 64, 256, 1096])
    ap.add_argument("--uneven-epochs", type=int, default=50)
    ap.add_argument("--dense-n", type=int, default=6000)
    ap.add_argument("--dense-iters", type=int, default=50)
    ap.add_argument("--dense-tc-m", type=lambda v: [int(x) for x in v.split(",")] if v else [], default=[64, 256],
                    help="right-hand sides of the tensor-core dense timing (multiples of 16; empty = skip)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--ref-days", type=int, default=1096)
    ap.add_argument("--ref-epochs", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per fused launch from an ncu capture of the same kernel")
    ap.add_argument("--dense-case", default="",
                    help="METHOD,M: run one dense NNLS call (n = --dense-n, --dense-iters iterations) and exit; "
                         "the small case the dense kernels' profiles capture")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.dense_case:
        return run_dense_case(args)
    return run_gpu(args)


def run_dense_case(args):
    """One dode_dense_nnls call on the benchmark's dense input (seeded random n x n B, y = B x with
    x >= 0, m columns), printed as one JSON line: the case an ncu capture of a dense kernel runs."""
    import torch
    from paper_1901_09266_gb300 import build, dode
    build.build()
    method, m = (int(v) for v in args.dense_case.split(","))
    n = args.dense_n
    rng = np.random.default_rng(1901)
    B = torch.from_numpy(rng.standard_normal((n, n), dtype=np.float32) / np.float32(np.sqrt(n))).cuda()
    X0 = torch.from_numpy(np.abs(rng.standard_normal((n, m))).astype(np.float32)).cuda()
    Y = (B @ X0).contiguous()
    _, _, loss, ms = dode.dense_nnls(B, Y, args.dense_iters, 0.05, method=method)
    print(json.dumps({"dense_case": {"method": method, "n": n, "m": m, "iters": args.dense_iters,
                                     "kernel_ms": ms, "loss": float(loss.double().sum().item())}}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
