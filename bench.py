"""Benchmark of the PDMP morph hot path on one GB300 (or N replicas).

One step = one pdmp_morph over the 2-D fitted-occupancy workload:
N = 2^20 base samples uniform in [0,10]^2, M = 16,384 RBF centres (gamma = 8)
with weights fitted on the GPU by pdmp_fit_occupancy to 200k points labelled
by 64 random boxes, T = 50 Euler steps, eta = 0.5 / L with L the certified
bound from pdmp_lipschitz_bound.  Work per step: N * T * M feature
evaluations.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

WORKLOAD = "rbf2d-fitted-M16384-N1048576-T50"
METRIC = "feature-evals/s (N*T*M)"
D, M, N, T = 2, 16384, 1 << 20, 50
# --workload small: the same field and fit on 262,144 samples and 3 steps, for
# ncu captures that must stay small (well under a second of replay per pass)
SMALL = {"N": 1 << 18, "T": 3}
L2_FLUSH_BYTES = 256 << 20
LAUNCHES_PER_MORPH = 9
FP32_LANES_PER_SM = 128           # FP32 pipe width per SM per clock
MUFU_EX2_PER_SM = 32              # measured ex2 throughput per SM per clock on GB300
KERNEL_SOURCES = ["paper_2108_11775_gb300/csrc/morph_rbf_fast.cu", "paper_2108_11775_gb300/csrc/sort.cu",
                  "paper_2108_11775_gb300/csrc/common.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"sm_max_mhz": 2070.0}, "fallback"


def alu_peak(n_sms: int, sm_mhz: float) -> float:
    """Feature evaluations per second the FP32 pipe and the MUFU allow: an RBF
    feature in d dimensions needs at least 2d + 1 FP32 operations (d for the
    exponent's linear form, 1 for s, d for the gradient moments) and one ex2."""
    per_sm_clk = min(FP32_LANES_PER_SM / (2 * D + 1), MUFU_EX2_PER_SM / 1.0)
    return n_sms * sm_mhz * 1e6 * per_sm_clk


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        loaded = [v for v in sm if mx and v > 0.5 * max(mx)] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
def build_workload(pdmp, torch, seed=2):
    wk = wl.config2(seed=seed, N=N, M=M)
    fld = pdmp.DeviceField.from_host(wk.field)
    X = torch.from_numpy(wk.fit_X).cuda()
    y = torch.from_numpy(wk.fit_y).cuda()
    w, b, loss, _ = pdmp.fit_occupancy(fld, X, y, 1e-4, 20, 200)
    fitted = fld.with_weights(w, bias=b)
    L, _ = pdmp.lipschitz_bound(fitted, wk.lo - 0.5, wk.hi + 0.5, cells=128)
    eta = float(np.float32(0.5 / L))
    fitted.lipschitz = L
    return wk, fitted, eta, {"fit_loss": loss, "L": L, "eta": eta}


def run_ours(args, world, rank, local):
    import torch
    import paper_2108_11775_gb300 as pdmp

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wk, fld, eta, info = build_workload(pdmp, torch)
    x0 = torch.from_numpy(wk.x0).cuda()
    xT = torch.empty_like(x0)
    ws = torch.empty(pdmp.morph_workspace(fld, N), dtype=torch.uint8, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        pdmp.morph(fld, x0, T, eta, out=xT, ws=ws)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(i & 0xFF)                      # L2 flush between timed launches (not timed)
            starts[i].record(stream)
            pdmp.morph(fld, x0, T, eta, out=xT, ws=ws)
            ends[i].record(stream)
        torch.cuda.synchronize()
        wall1 = time.perf_counter()
        torch.cuda.nvtx.range_pop()
    barrier(world)
    per = [s.elapsed_time(e) / 1e3 for s, e in zip(starts, ends)]
    total = max_over_ranks(world, sum(per))
    status, detail = pdmp.stream_status()
    if status != 0:
        raise RuntimeError(f"device status {status} ({detail})")

    # end to end through the public API with host buffers (pinned), copies timed
    x_host = torch.from_numpy(wk.x0).pin_memory()
    out_host = torch.empty_like(x_host).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    xd = torch.empty_like(x0)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        xd.copy_(x_host, non_blocking=True)
        pdmp.morph(fld, xd, T, eta, out=xd, ws=ws)
        out_host.copy_(xd, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_total = max_over_ranks(world, e0.elapsed_time(e1) / 1e3)
    assert np.isfinite(out_host.numpy()).all()

    work = float(N) * T * M
    value = world * work * args.steps / total
    achieved = work / (sum(per) / len(per))
    pk, pk_kind = peaks()
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = alu_peak(n_sms, float(pk.get("sm_max_mhz", 2070.0)))
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tj = json.load(f)
        if tj.get("kernel_hash") == kernel_hash():
            traffic = tj.get("bytes_per_launch")
    line = {
        "metric": METRIC, "value": value, "unit": "feature-evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "M": M, "T": T, "d": D, "gamma": 8.0, "eta": eta,
                   "L": info["L"], "fit_loss": info["fit_loss"], "l2_flush": "256 MiB write between timed launches",
                   "parallelism": f"replicas{world}"},
        "e2e": {"value": world * work * args.steps / e2e_total, "unit": "feature-evals/s",
                "h2d_bytes_per_step": int(x_host.numel() * 4), "d2h_bytes_per_step": int(out_host.numel() * 4)},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "feature-evals/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_basis": f"{n_sms} SMs x {pk.get('sm_max_mhz', 2070.0)} MHz ({pk_kind} max clock) x "
                                   f"min(128/(2d+1) FP32, 32 ex2) per SM-clock"},
        "clocks": clk.summary(),
        # per step: centre table, 7 kernels of the spatial sort, the morph kernel
        "gpu_launches": args.steps * LAUNCHES_PER_MORPH,
        "wall_s_timed": wall1 - wall0,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wk, fld, eta, target_s=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_baseline(wk, fld, eta, target_s=12.0):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload."""
    import oracle
    ncores = os.cpu_count() or 1
    oracle.set_threads(ncores)
    f = wk.field.with_weights(fld.w.cpu().numpy(), bias=fld.bias)
    probe = 2 * ncores
    t0 = time.perf_counter()
    oracle.morph(f, wk.x0[:probe], T, eta)
    rate = probe * T * M / (time.perf_counter() - t0)
    n = int(max(probe, min(wk.x0.shape[0], rate * target_s / (T * M))))
    n = (n // ncores) * ncores or ncores
    t0 = time.perf_counter()
    oracle.morph(f, wk.x0[probe:probe + n], T, eta)
    dt = time.perf_counter() - t0
    return {"value": n * T * M / dt, "unit": "feature-evals/s", "cores": ncores, "kind": "oracle",
            "sample": f"{n} of the {N} samples, full M={M} and T={T}, FP64 C oracle, {dt:.1f} s"}


def run_reference(args, world, rank, local):
    if rank != 0:
        return
    import oracle
    ncores = os.cpu_count() or 1
    oracle.set_threads(ncores)
    wk = wl.config2(N=max(4096, ncores * 64), M=M)
    f = wk.field.with_weights(wl.proxy_fitted_weights(2, wk.field.centres, wk.boxes))
    L, _ = oracle.lipschitz(f, wk.lo - 0.5, wk.hi + 0.5, cells=64)
    eta = 0.5 / L
    n = ncores * 4
    for i in range(args.warmup):
        oracle.morph(f, wk.x0[:ncores], T, eta)
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.morph(f, wk.x0[i * n % (wk.x0.shape[0] - n):][:n], T, eta)
    dt = time.perf_counter() - t0
    value = args.steps * n * T * M / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "feature-evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "M": M, "T": T, "d": D, "sample_per_step": n},
            "cpu_baseline": {"value": value, "unit": "feature-evals/s", "cores": ncores, "kind": "oracle",
                             "sample": f"{n} samples per step, full M and T, FP64 C oracle"},
            "e2e": {"value": value, "unit": "feature-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["full", "small"], default="full",
                    help="small: 65,536 samples and 5 steps of the same workload (for ncu captures)")
    args = ap.parse_args()
    if args.workload == "small":
        global N, T, WORKLOAD
        N, T = SMALL["N"], SMALL["T"]
        WORKLOAD = f"rbf2d-fitted-M{M}-N{N}-T{T}"
        args.no_cpu_baseline = True
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
