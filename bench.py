"""Benchmark of the PDMP morph hot path on one GB300 (or N replicas).

One step = one pdmp_morph over the 2-D fitted-occupancy workload:
N = 2^20 base samples uniform in [0,10]^2, M = 16,384 RBF centres (gamma = 8)
with the occupancy weights fitted to 200k points labelled by 64 random boxes
(the stored fit of tests/golden/fit_rbf2d_fitted.txt, made by the oracle
alone, which the parity tests check at this size; pdmp_fit_occupancy fits the
same data on the GPU and its loss is reported beside), T = 50 Euler steps,
eta = 0.5 / L with L the stored certified bound (pdmp_lipschitz_bound's is
reported beside).  Work per step: N * T * M feature evaluations.

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
MUFU_SINCOS_PER_SM = 15.6         # measured sin (or cos) throughput per SM per clock on GB300
MUFU_TANH_PER_SM = 15.2           # measured tanh.approx throughput per SM per clock on GB300
MMA_TF32_PER_SM = 480.0           # measured mma.sync TF32 multiply-adds per SM per clock on GB300
MLP_MACS_PER_SAMPLE = 39 * 128 + 2 * 128 * 128 + 128 * 3   # the surrogate network's multiply-adds per sample
KERNEL_SOURCES = ["paper_2108_11775_gb300/csrc/morph_rbf_fast.cu", "paper_2108_11775_gb300/csrc/fast_tile.cuh",
                  "paper_2108_11775_gb300/csrc/sort.cu", "paper_2108_11775_gb300/csrc/common.cuh"]


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
    """Feature evaluations per second at the FP32/ex2 roofline with the
    algorithmic count of an RBF feature in d dimensions: 2d + 2 FP32
    operations (d for the exponent's linear form, one for the weight, one for
    s, d for the gradient moments) and one ex2.  128 FP32 lanes per SM per
    clock give 128 / (2d + 2) features per SM per clock; the ex2 unit (32 per
    SM per clock) is not the limit."""
    per_sm_clk = min(FP32_LANES_PER_SM / (2 * D + 2), MUFU_EX2_PER_SM / 1.0)
    return n_sms * sm_mhz * 1e6 * per_sm_clk


def kernel_pipe_peak(n_sms: int, sm_mhz: float) -> float:
    """The fast kernel's own FP32-pipe ceiling: it folds the weight into the
    exponent and issues 2d + 1 FP32 operations per feature, as packed f32x2
    FMAs that occupy the FMA pipe for two clocks each (one issue slot), so
    128 / (2d + 1) features per SM per clock."""
    return n_sms * sm_mhz * 1e6 * FP32_LANES_PER_SM / (2 * D + 1)


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
    """The largest value over the ranks (timing only: the morph itself needs
    no collective).  Works on the NCCL (CUDA tensors) and gloo (CPU) backends."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_sample_seed(rank: int) -> int:
    """Each rank morphs its own batch of samples (weak scaling): same field,
    different base samples."""
    return 2 + 1000 * rank


def whole_job_rate(world: int, work_per_rank_step: float, steps: int, max_seconds: float) -> float:
    """Units all ranks processed divided by the slowest rank's time."""
    return world * work_per_rank_step * steps / max_seconds


# ---------------------------------------------------------------------------
def build_workload(pdmp, torch, seed=2):
    """The 2-D fitted workload with the stored fit (the oracle's weights and
    bias for this field, and its certified bound L), the field the parity
    tests check at this size.  The library's own fit of the same data runs
    too, and its loss, step size and certified bound on the stored field are
    reported beside the stored ones."""
    wk, params = wl.config2_fitted(seed=seed, N=N)
    fld = pdmp.DeviceField.from_host(wk.field)
    X = torch.from_numpy(wk.fit_X).cuda()
    y = torch.from_numpy(wk.fit_y).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, loss, alpha = pdmp.fit_occupancy(fld, X, y, params["l2"], params["power_iters"], params["iters"])
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t0
    L_gpu, _ = pdmp.lipschitz_bound(fld, wk.lo - 0.5, wk.hi + 0.5, cells=128)
    L = params["L"]
    eta = float(np.float32(0.5 / L))
    fld.lipschitz = L
    fit = {"weights": "stored oracle fit (tests/golden/fit_rbf2d_fitted.txt)", "oracle_loss": params["loss_f64"],
           "gpu_fit_loss": loss, "gpu_fit_rel_diff": abs(loss - params["loss_f64"]) / params["loss_f64"],
           "gpu_fit_alpha": alpha, "gpu_fit_s": fit_s, "L_stored": L, "L_gpu": L_gpu}
    return wk, fld, eta, {"fit_loss": params["loss_f64"], "L": L, "eta": eta, "fit": fit}


def run_ours(args, world, rank, local):
    import torch
    import paper_2108_11775_gb300 as pdmp

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wk, fld, eta, info = build_workload(pdmp, torch)
    if rank:
        wk.x0 = wl.uniform_box(rank_sample_seed(rank), wl.S_SAMPLES, N, wk.lo, wk.hi)
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
    value = whole_job_rate(world, work, args.steps, total)
    achieved = work / (sum(per) / len(per))
    pk, pk_kind = peaks()
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = alu_peak(n_sms, float(pk.get("sm_max_mhz", 2070.0)))
    pipe_peak = kernel_pipe_peak(n_sms, float(pk.get("sm_max_mhz", 2070.0)))
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
                   "L": info["L"], "fit_loss": info["fit_loss"], "fit": info["fit"],
                   "l2_flush": "256 MiB write between timed launches",
                   "parallelism": f"replicas{world}"},
        "e2e": {"value": whole_job_rate(world, work, args.steps, e2e_total), "unit": "feature-evals/s",
                "h2d_bytes_per_step": int(x_host.numel() * 4), "d2h_bytes_per_step": int(out_host.numel() * 4)},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "feature-evals/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_basis": f"{n_sms} SMs x {pk.get('sm_max_mhz', 2070.0)} MHz ({pk_kind} max clock) x "
                                   f"128 FP32 lanes / (2d+2) FP32 operations per feature",
                     "kernel_pipe_peak": pipe_peak, "kernel_pipe_frac": achieved / pipe_peak},
        "clocks": clk.summary(),
        # per step: centre table, 7 kernels of the spatial sort, the morph kernel
        "gpu_launches": args.steps * LAUNCHES_PER_MORPH,
        "wall_s_timed": wall1 - wall0,
    }
    # the oracle baseline and the extras run at N = 1 only (a multi-GPU run times the headline step)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wk, fld, eta, target_s=args.cpu_seconds)
    if world == 1 and not args.no_extras and args.workload == "full":
        culled = extra_culled(pdmp, torch, fld, x0, xT, eta)
        pdmp.morph(fld, x0, T, eta, out=xT, ws=ws)
        inverse = extra_inverse(pdmp, torch, fld, x0, xT, eta, n_sms, pk)
        vjp2d = extra_vjp_rbf2d(pdmp, torch, fld, x0, eta, n_sms, pk)
        culled["speedup_vs_dense"] = (float(N) * T * M / achieved) / (culled["ms"] / 1e3)
        del x0, xT, ws, flush
        torch.cuda.empty_cache()
        line["extras"] = {
            "culled_morph": culled,
            "inverse_2d": inverse,
            "vjp_rbf2d": vjp2d,
            "tanh_net_cost": extra_tanh_net(pdmp, torch, n_sms, pk),
            "cspace_7link": extra_cspace(pdmp, torch, fld, info),
            "sampler": extra_sampler(pdmp, torch, fld, eta),
            "batched_256_envs": extra_batched(pdmp, torch, n_sms, pk),
            "rff7d_differentiation": extra_rff(pdmp, torch, n_sms, pk),
            "surrogate_3d": extra_surrogate(pdmp, torch, args),
        }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _time(torch, fn, reps=3):
    """Best of reps CUDA-event timings of fn() on the current stream (seconds)."""
    stream = torch.cuda.current_stream()
    best = None
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 1e3
        best = t if best is None else min(best, t)
    return best


def extra_batched(pdmp, torch, n_sms, pk):
    """256 environments (d in {2,3}, M ~ U[256,8192], N ~ U[1k,64k], T = 30)
    in one persistent launch, autotuned, replayed from a CUDA graph."""
    hosts = wl.config4()
    envs = []
    for w in hosts:
        f = pdmp.DeviceField.from_host(w.field)
        L, _ = pdmp.lipschitz_bound(f, w.lo - 0.5, w.hi + 0.5, cells=64 if w.field.d == 2 else 16)
        f.lipschitz = L
        envs.append((f, torch.from_numpy(w.x0).cuda(), float(np.float32(0.5 / L)), w.T))
    b = pdmp.Batch(envs)
    best, times = b.autotune(reps=1, use_cache=False)
    b.capture()
    torch.cuda.current_stream().wait_stream(b.graph_stream)
    b.replay()
    torch.cuda.synchronize()
    t = _time(torch, b.replay, reps=3)
    work = b.work()
    # FP32 roofline (2d + 2 operations per feature) per environment's d, weighted by its work
    mhz = float(pk.get("sm_max_mhz", 2070.0))
    t_peak = sum(w.x0.shape[0] * w.field.M * w.T / (n_sms * mhz * 1e6 * 128.0 / (2 * w.field.d + 2)) for w in hosts)
    return {"value": work / t, "unit": "feature-evals/s", "ms_per_launch": 1e3 * t, "work": work,
            "roofline_frac": (work / t) / (work / t_peak), "variant": best,
            "variant_ms": [round(v, 3) for v in times], "launch": "CUDA graph of one pdmp_morph_batched",
            "gpu_launches_per_run": 11}


def extra_cspace(pdmp, torch, fld, info, n=1 << 16, t_steps=20, links=7, per_link=4):
    """Eq. (3) in joint space: a 7-link planar arm (4 body points a link) at
    the centre of the fitted 2-D workspace; the step is the certified one
    (eta = 0.5 / L_q from the field's bounds and the chain lengths).
    Reports sample-steps/s and the body-point feature evaluations per second."""
    chain = wl.planar_arm(links, 4.5, (5.0, 5.0), per_link)
    _, G = pdmp.lipschitz_bound(fld, np.full(2, -0.5), np.full(2, 10.5), cells=128)
    Lq = pdmp.cspace_lipschitz(chain, info["L"], G)
    eta = float(np.float32(0.5 / Lq))
    lo, hi = wl.joint_box(links)
    q0 = torch.from_numpy(wl.uniform_box(11, wl.S_SAMPLES, n, lo, hi)).cuda()
    out = torch.empty_like(q0)
    ws = torch.empty(pdmp.cspace_workspace(fld, chain, n), dtype=torch.uint8, device="cuda")
    run = lambda: pdmp.cspace_morph(fld, chain, q0, t_steps, eta, out=out, ws=ws)
    run()
    t = _time(torch, run, reps=3)
    b = links * per_link
    return {"value": n * t_steps / t, "unit": "sample-steps/s", "ms": 1e3 * t, "N": n, "T": t_steps,
            "joints": links, "body_points": b, "feature_evals_per_s": n * t_steps * b * M / t, "eta": eta, "L_q": Lq,
            "launches_per_step": 11}


def extra_sampler(pdmp, torch, fld, eta, batch=1 << 16, capacity=1 << 20, t_steps=50):
    """The diffeomorphic sampler (Sec. 3.3) on the fitted 2-D field: time for
    the background producer to fill a bucket of 2^20 morphed samples, the
    delivered rate, and the latency of a 10,000-sample draw from the full bucket."""
    lo, hi = np.zeros(2), np.full(2, 10.0)
    t0 = time.perf_counter()
    s = pdmp.Sampler(fld, lo, hi, t_steps, eta, batch=batch, capacity=capacity, seed=3)
    try:
        while s.stats()["queued"] < capacity and time.perf_counter() - t0 < 60:
            time.sleep(0.002)
        fill = time.perf_counter() - t0
        st = s.stats()
        t1 = time.perf_counter()
        _, m = s.draw(10_000)
        draw_us = 1e6 * (time.perf_counter() - t1)
    finally:
        s.close()
    return {"bucket_fill_s": fill, "bucket_samples": capacity, "delivered_per_s": st["produced"] / fill,
            "batch": batch, "T": t_steps, "draw_10k_us": draw_us, "draw_10k_morphed": m, "error": st["error"]}


def extra_culled(pdmp, torch, fld, x0, xT_dense, eta, eps=1e-6):
    """The spatially culled morph on the same workload: its effective rate
    (dense N T M over its time; not a roofline fraction), the fraction of
    the dense feature evaluations it performs, and its largest deviation
    from the dense kernel's x_T."""
    r, W = pdmp.cull_radius(fld, eps)
    ws = torch.empty(pdmp.morph_culled_workspace(fld, N), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(x0)
    run = lambda: pdmp.morph_culled(fld, x0, T, eta, r, out=out, ws=ws)
    for _ in range(3):
        run()
    t = _time(torch, run, reps=5)
    work = torch.zeros(1, dtype=torch.int64, device="cuda")
    pdmp.morph_culled(fld, x0, T, eta, r, out=out, ws=ws, work=work)
    dense = float(N) * T * M
    dev = float((out - xT_dense).abs().max())
    return {"effective_value": dense / t, "unit": "feature-evals/s (dense-equivalent)", "ms": 1e3 * t,
            "speedup_vs_dense": None, "evaluated_fraction": int(work.item()) / dense,
            "eps": eps, "r_cut": r, "sum_abs_w": W, "max_abs_dev_vs_dense": dev,
            "note": "features farther than r_cut from a tile dropped; s and |grad s| change by at most eps"}


def extra_inverse(pdmp, torch, fld, x0, xT, eta, n_sms, pk, n=1 << 18, n_direct=1 << 16, tol=1e-6):
    """Eq. (2) on the 2-D fitted workload: the first n morphed samples x_T
    (T = 50) taken back to x_0 by per-step fixed points on sorted tiles.  The
    rate counts the feature evaluations performed (the kernel's own counter:
    per block, its iterations summed over the steps times its samples times
    M), against the forward's FP32 roofline; the direct kernel runs on the
    first n_direct samples for comparison.  Also the log-density of the same
    samples (inverse, log-det, uniform base density on the box)."""
    z = xT[:n].contiguous()
    ws = torch.empty(pdmp.morph_workspace(fld, n), dtype=torch.uint8, device="cuda")
    y = torch.empty_like(z)
    work = torch.zeros(1, dtype=torch.int64, device="cuda")
    run = lambda: pdmp.morph_inverse(fld, z, T, eta, tol=tol, out=y, ws=ws)
    run()
    t = _time(torch, run, reps=2)
    pdmp.morph_inverse(fld, z, T, eta, tol=tol, out=y, ws=ws, work=work)
    evals = float(work.item())
    rt = float((y - x0[:n]).abs().max())
    zd = xT[:n_direct].contiguous()
    yd = torch.empty_like(zd)
    wd = torch.zeros(1, dtype=torch.int64, device="cuda")
    rund = lambda: pdmp.morph_inverse(fld, zd, T, eta, tol=tol, out=yd, fast=False)
    rund()
    td = _time(torch, rund, reps=1)
    pdmp.morph_inverse(fld, zd, T, eta, tol=tol, out=yd, fast=False, work=wd)
    peak = alu_peak(n_sms, float(pk.get("sm_max_mhz", 2070.0)))
    lo, hi = np.zeros(D), np.full(D, 10.0)
    tl = _time(torch, lambda: pdmp.log_density(fld, z, T, eta, lo, hi, tol=tol, ws=ws), reps=1)
    return {"value": evals / t, "unit": "feature-evals/s", "ms": 1e3 * t, "N": n, "T": T, "tol": tol,
            "roofline_frac": evals / t / peak, "sample_steps_per_s": n * T / t,
            "mean_iterations_per_step": evals / (n * T * M), "round_trip_max_abs": rt,
            "direct_kernel": {"value": float(wd.item()) / td, "N": n_direct, "ms": 1e3 * td},
            "log_density": {"samples_per_s": n / tl, "ms": 1e3 * tl},
            "launches_per_call": 9}


def extra_tanh_net(pdmp, torch, n_sms, pk, d=2, H=64, n=1 << 20, t_steps=50):
    """The paper's own occupancy model (tanh network, Sec. 3.1) as the morph
    cost: sample-steps per second and the fraction of the FP32 roofline for
    the network's multiply-adds per sample-step (forward and input gradient)."""
    net = wl.tanh_net(7, d, H)
    dn = pdmp.DeviceTanhNet.from_host(net)
    L, _ = pdmp.tanh_net_lipschitz(dn)
    eta = float(np.float32(0.5 / L))
    x0 = torch.from_numpy(wl.uniform_box(7, wl.S_SAMPLES, n, np.zeros(d), np.full(d, 10.0))).cuda()
    out = torch.empty_like(x0)
    run = lambda: pdmp.tanh_net_morph(dn, x0, t_steps, eta, out=out)
    for _ in range(3):
        run()
    t = _time(torch, run, reps=5)
    macs = 2 * H * H + 2 * d * H + 2 * H          # W2 h1 and W2^T v2; W1 x and W1^T g1; w3 h2 and w3 (.) (1 - h2^2)
    rate = n * t_steps / t
    clk = n_sms * float(pk.get("sm_max_mhz", 2070.0)) * 1e6
    # binding bound: the two H x H products on the tensor cores as TF32 MMAs with
    # hi/lo splits (3 products each) at 480 multiply-adds per SM per clock; the rest
    # (2dH + 2H FP32 multiply-adds, 2H tanh) fits beside it
    tc_clk = 3 * 2 * H * H / MMA_TF32_PER_SM
    alu_clk = (2 * d * H + 2 * H) / FP32_LANES_PER_SM + 2 * H / MUFU_EX2_PER_SM
    peak = clk / max(tc_clk, alu_clk)
    return {"value": rate, "unit": "sample-steps/s", "ms": 1e3 * t, "N": n, "T": t_steps, "d": d, "H": H,
            "macs_per_sample_step": macs, "roofline_frac": rate / peak, "roofline_bound": "tensor (mma.sync TF32)",
            "fp32_count_frac": rate / (clk * FP32_LANES_PER_SM / macs), "L": L, "eta": eta,
            "note": "roofline_frac against the tensor pipe (3 TF32 products per H x H multiply-add); "
                    "fp32_count_frac against every multiply-add on the FP32 lanes"}


def extra_vjp_rbf2d(pdmp, torch, fld, x0, eta, n_sms, pk, k=5):
    """The VJP of the T-step map on the 2-D fitted workload (N = 2^20, T = 50,
    M = 16,384): checkpoints every k steps from the forward, then the VJP kernel
    (per segment a recompute pass and a Hessian-vector pass).  The rate counts
    both passes (2 N T M); the roofline per pass is the forward's 2d + 2 FP32
    operations per feature, so the fraction is a lower bound (a Hessian-vector
    feature costs more)."""
    gT = torch.from_numpy(wl.f32(wl.rng(2, wl.S_COTANGENT).standard_normal((x0.shape[0], D)))).cuda()
    ck = torch.empty(T // k, x0.shape[0], D, device="cuda")
    pdmp.morph(fld, x0, T, eta, ckpt=ck, k=k)
    g0 = torch.empty_like(x0)
    t = _time(torch, lambda: pdmp.morph_vjp(fld, x0, T, eta, k, gT, ckpt=ck, g0=g0), reps=2)
    # with d/dw and d/dbias: a third, transposed pass per step on the same tiles
    ws_pg = torch.empty(pdmp.morph_vjp_workspace(fld, x0.shape[0], T, k, 1), dtype=torch.uint8, device="cuda")
    t_pg = _time(torch, lambda: pdmp.morph_vjp(fld, x0, T, eta, k, gT, ckpt=ck, g0=g0, want_param_grad=True,
                                               ws=ws_pg), reps=1)
    work = 2.0 * x0.shape[0] * T * M
    peak = alu_peak(n_sms, float(pk.get("sm_max_mhz", 2070.0)))
    return {"value": work / t, "unit": "feature-evals/s (2 passes)", "ms": 1e3 * t, "k": k,
            "roofline_frac_vs_forward_count": work / t / peak,
            "param_grad": {"ms": 1e3 * t_pg, "value": 1.5 * work / t_pg, "unit": "feature-evals/s (3 passes)"}}


def extra_rff(pdmp, torch, n_sms, pk):
    """7-D random Fourier field (M = 4096, N = 2^20, T = 20, k = 5): forward
    with checkpoints, VJP from them, and the log-det pass."""
    wk = wl.config3()
    f = pdmp.DeviceField.from_host(wk.field)
    L, _ = pdmp.lipschitz_bound(f)
    eta = float(np.float32(0.5 / L))
    x0 = torch.from_numpy(wk.x0).cuda()
    gT = torch.from_numpy(wk.extra["gT"]).cuda()
    N, T, k, M = x0.shape[0], wk.T, wk.extra["k"], wk.field.M
    ck = torch.empty(T // k, N, 7, device="cuda")
    out = torch.empty_like(x0)
    t_fwd = _time(torch, lambda: pdmp.morph(f, x0, T, eta, out=out, ckpt=ck, k=k), reps=2)
    g0 = torch.empty_like(x0)
    t_vjp = _time(torch, lambda: pdmp.morph_vjp(f, x0, T, eta, k, gT, ckpt=ck, g0=g0), reps=2)
    # with d/dw and d/dbias: a third pass per step (the weight terms) on the same tensor-core kernel
    ws_pg = torch.empty(pdmp.morph_vjp_workspace(f, N, T, k, 1), dtype=torch.uint8, device="cuda")
    t_pg = _time(torch, lambda: pdmp.morph_vjp(f, x0, T, eta, k, gT, ckpt=ck, g0=g0, want_param_grad=True,
                                               ws=ws_pg), reps=1)
    t_ld = _time(torch, lambda: pdmp.logdet(f, x0, T, eta), reps=1)
    # the inverse of the forward's output (Eq. 2), on the tensor cores
    y = torch.empty_like(x0)
    wk_inv = torch.zeros(1, dtype=torch.int64, device="cuda")
    t_inv = _time(torch, lambda: pdmp.morph_inverse(f, out, T, eta, out=y), reps=1)
    pdmp.morph_inverse(f, out, T, eta, out=y, work=wk_inv)
    inv_rt = float((y - x0).abs().max())
    work = float(N) * T * M
    d = 7
    clk = n_sms * float(pk.get("sm_max_mhz", 2070.0)) * 1e6
    # Binding bounds per feature and sample, per SM and clock.  MUFU: sin and
    # cos (15.6 each per SM per clock, measured), 2 per feature in every pass.
    # Tensor pipe: mma.sync m16n8k8 TF32 at 480 multiply-adds per SM per clock
    # (measured); a 16 x 8 tile of one MMA is 1024 multiply-adds over 128
    # feature-samples.  Forward / VJP recompute: theta and grad s, 3 + 3 MMAs
    # (48 per feature-sample); VJP Hessian-vector pass: 12 MMAs (96); log-det:
    # 18 MMAs (144).  The pass's bound is the slower of the two.
    mufu_fs = MUFU_SINCOS_PER_SM / 2.0
    tc = lambda n_mma: MMA_TF32_PER_SM / (n_mma * 1024.0 / 128.0)
    bounds = {"forward": min(mufu_fs, tc(6)), "vjp_recompute": min(mufu_fs, tc(6)), "vjp_hvp": min(mufu_fs, tc(12)),
              "logdet": min(mufu_fs, tc(18))}
    names = {k: ("mufu" if bounds[k] == mufu_fs else "tensor") for k in bounds}
    # the VJP's two passes each sweep N T M: its bound is the sum of the passes' times
    t_bound = {"forward": work / (clk * bounds["forward"]),
               "vjp": work / (clk * bounds["vjp_recompute"]) + work / (clk * bounds["vjp_hvp"]),
               "logdet": work / (clk * bounds["logdet"])}
    t_meas = {"forward": t_fwd, "vjp": t_vjp, "logdet": t_ld}
    rates = {"forward": work / t_fwd, "vjp_per_pass": 2 * work / t_vjp, "logdet": work / t_ld,
             "vjp_param_grad_per_pass": 3 * work / t_pg}
    return {**rates, "unit": "feature-evals/s",
            "roofline_frac": {k: t_bound[k] / t_meas[k] for k in t_bound},
            "roofline_bound": {"forward": names["forward"], "vjp": f"{names['vjp_recompute']} + {names['vjp_hvp']}",
                               "logdet": names["logdet"]},
            "roofline_peak_per_sm_clk": bounds,
            "mufu_frac": {k: rates[k] / (clk * mufu_fs) for k in rates}, "mufu_peak": clk * mufu_fs,
            "ms": {"forward": 1e3 * t_fwd, "vjp": 1e3 * t_vjp, "vjp_param_grad": 1e3 * t_pg, "logdet": 1e3 * t_ld,
                   "inverse": 1e3 * t_inv},
            "inverse": {"value": float(wk_inv.item()) / t_inv, "unit": "feature-evals/s performed",
                        "mean_iterations_per_step": float(wk_inv.item()) / work, "round_trip_max_abs": inv_rt},
            "note": "roofline_frac = the bound's time / the measured time, with each pass bound by the slower of "
                    "MUFU sin+cos and the mma.sync TF32 tensor pipe (feature-samples per SM per clock in "
                    "roofline_peak_per_sm_clk); the VJP counts its recompute and Hessian-vector passes "
                    "(2 N T M), with the parameter gradient also its weight pass (3 N T M)"}


def extra_surrogate(pdmp, torch, args):
    """3-D fitted field (M = 8192, gamma = 8, 48 boxes, T = 40): MLP trained on
    2^20 pairs from the plain morph, then inference on N = 2^24 with the plain
    morph as fallback, against the plain morph alone."""
    wk = wl.config5()
    f0 = pdmp.DeviceField.from_host(wk.field)
    w, bias, fit_loss, _ = pdmp.fit_occupancy(f0, torch.from_numpy(wk.fit_X).cuda(), torch.from_numpy(wk.fit_y).cuda(),
                                              1e-4, 20, 200)
    f = f0.with_weights(w, bias=bias)
    L, _ = pdmp.lipschitz_bound(f, wk.lo - 0.5, wk.hi + 0.5, cells=32)
    f.lipschitz = L
    eta = float(np.float32(0.5 / L))
    T = wk.T
    xtr = torch.from_numpy(wk.extra["x_train"]).cuda()
    tau_r, xTtr = pdmp.residual_threshold(f, xtr, T, eta, 0.99)
    scale = pdmp.displacement_rms(xtr, xTtr).cpu().numpy()
    net = pdmp.Surrogate(wk.lo, wk.hi, scale, seed=5)
    B, steps = 4096, args.surrogate_steps
    loss = torch.zeros(1, device="cuda")
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev0.record(stream)
    for s in range(steps):
        lr = 2e-3 * 0.5 * (1.0 + np.cos(np.pi * s / steps)) + 1e-5
        i = (s * B) % (xtr.shape[0] - B)
        net.train_step(xtr[i:i + B], xTtr[i:i + B], lr=lr, loss=loss if s == steps - 1 else None)
    ev1.record(stream)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    train_step_ms = ev0.elapsed_time(ev1) / steps
    x0 = torch.from_numpy(wk.x0).cuda()
    boxes = torch.from_numpy(wk.boxes).cuda()
    plain = torch.empty_like(x0)
    ws = torch.empty(pdmp.morph_workspace(f, x0.shape[0]), dtype=torch.uint8, device="cuda")
    t_plain = _time(torch, lambda: pdmp.morph(f, x0, T, eta, out=plain, ws=ws), reps=2)
    # the residual check on the culled kernel (eps = 1e-6 on s and |grad s|), and on the dense one
    r_cut, _ = pdmp.cull_radius(f, 1e-6)
    sws = torch.empty(pdmp.surrogate_workspace(f, x0.shape[0]), dtype=torch.uint8, device="cuda")
    sur, sur_d = torch.empty_like(x0), torch.empty_like(x0)
    res = {}

    def run_sur():
        res["nf"] = net.infer(f, x0, T, eta, tau_r, out=sur, ws=sws, r_cut=r_cut)[1]

    def run_sur_dense():
        res["nf_dense"] = net.infer(f, x0, T, eta, tau_r, out=sur_d, ws=sws)[1]
    run_sur()
    t_sur = _time(torch, run_sur, reps=2)
    run_sur_dense()
    t_sur_d = _time(torch, run_sur_dense, reps=2)
    # the plain morph culled the same way: the surrogate's check and fallback are culled too
    cws = torch.empty(pdmp.morph_culled_workspace(f, x0.shape[0]), dtype=torch.uint8, device="cuda")
    plain_c = torch.empty_like(x0)
    t_plain_c = _time(torch, lambda: pdmp.morph_culled(f, x0, T, eta, r_cut, out=plain_c, ws=cws), reps=1)
    col = lambda x: float(pdmp.box_labels(boxes, x).float().mean().item())
    c_prior, c_plain, c_sur, c_sur_d = col(x0), col(plain), col(sur), col(sur_d)
    del sws, cws
    # the network alone (inference kernel) on the N samples
    pred = torch.empty_like(x0)
    t_net = _time(torch, lambda: net.forward(x0, out=pred), reps=3)
    n_inf = float(x0.shape[0])
    macs = MLP_MACS_PER_SAMPLE
    clk = torch.cuda.get_device_properties(0).multi_processor_count * float(
        peaks()[0].get("sm_max_mhz", 2070.0)) * 1e6
    bf16_peak = float(peaks()[0].get("bf16_tflops", 1908.7)) * 1e12
    # the network's special-function work per sample: 384 SiLU (one tanh each) and
    # 36 sin / cos of the encoding
    mufu_peak_samples = clk / (384 / MUFU_TANH_PER_SM + 36 / MUFU_SINCOS_PER_SM)
    mlp = {"samples_per_s": n_inf / t_net, "ms": 1e3 * t_net, "macs_per_sample": macs,
           "tflops": 2.0 * macs * n_inf / t_net / 1e12,
           "frac_of_bf16_peak": 2.0 * macs * n_inf / t_net / bf16_peak,
           "frac_of_mufu_bound": n_inf / t_net / mufu_peak_samples,
           "train_step_ms": train_step_ms, "train_batch": B,
           "note": "bf16 peak: MEASURED_PEAKS.json bf16_tflops (cuBLAS, burst); MUFU bound: 384 tanh (SiLU) at "
                   "15.2 and 36 sin/cos (encoding) at 15.6 per SM per clock, measured"}
    return {"speedup_vs_plain_morph": t_plain / t_sur, "ms_plain": 1e3 * t_plain, "ms_surrogate": 1e3 * t_sur,
            "speedup_vs_culled_plain_morph": t_plain_c / t_sur,
            "check": "culled check and fallback (r_cut = %.4g from eps = 1e-6)" % r_cut,
            "dense_check": {"ms_surrogate": 1e3 * t_sur_d, "speedup_vs_plain_morph": t_plain / t_sur_d,
                            "fallback_fraction": res["nf_dense"] / x0.shape[0], "collision_rate": c_sur_d},
            "context_culled_plain_morph": {"ms": 1e3 * t_plain_c, "speedup_of_surrogate": t_plain_c / t_sur},
            "mlp": mlp,
            "fallback_fraction": res["nf"] / x0.shape[0], "collision_rate": {"prior": c_prior, "plain_morph": c_plain,
                                                                             "surrogate": c_sur},
            "equal_collision_rate": c_sur <= c_plain + 1e-3, "tau_r": tau_r, "train_steps": steps,
            "train_s": train_s, "final_train_loss": float(loss.item()), "N": int(x0.shape[0]), "T": T}


def cpu_baseline(wk, fld, eta, target_s=12.0):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload."""
    import oracle
    ncores = os.cpu_count() or 1
    oracle.set_threads(ncores)
    f = wk.field                       # the stored fit, the field the GPU step morphs
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
            "sample": f"{n} of the {N} samples, full M={M} and T={T}, FP64 C oracle, {dt:.1f} s",
            "per_core": n * T * M / dt / ncores, "cpu": host_cpu()}


def host_cpu() -> str:
    """The host CPU's model line from /proc/cpuinfo (or the platform's name)."""
    import platform
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware"):
                    return f"{platform.machine()} {line.split(':', 1)[1].strip()}"
    except OSError:
        pass
    return platform.machine() or "unknown"


def run_reference(args, world, rank, local):
    if rank != 0:
        return
    import oracle
    ncores = os.cpu_count() or 1
    oracle.set_threads(ncores)
    wk, params = wl.config2_fitted(N=max(4096, ncores * 64))
    f = wk.field
    eta = float(np.float32(0.5 / params["L"]))
    n = ncores * 16            # samples per step: about 0.15 s of the oracle on 16 cores
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


def profile_case(case: str, reps: int = 1):
    """One small launch of one kernel family (for ncu captures of kernels other
    than the headline one): inputs a few tens of MB, a handful of launches."""
    import torch
    import paper_2108_11775_gb300 as pdmp
    torch.cuda.set_device(0)
    out = {"case": case}
    if case in ("rff7d", "vjp", "logdet"):
        wk = wl.config3(N=1 << 17)
        f = pdmp.DeviceField.from_host(wk.field)
        L, _ = pdmp.lipschitz_bound(f)
        eta = float(np.float32(0.5 / L))
        x0 = torch.from_numpy(wk.x0).cuda()
        T, k = 4, 2
        ck = torch.empty(T // k, x0.shape[0], 7, device="cuda")
        if case == "rff7d":
            out["ms"] = 1e3 * _time(torch, lambda: pdmp.morph(f, x0, T, eta, ckpt=ck, k=k), reps=reps)
        elif case == "vjp":
            pdmp.morph(f, x0, T, eta, ckpt=ck, k=k)
            gT = torch.from_numpy(wk.extra["gT"][:x0.shape[0]]).cuda()
            out["ms"] = 1e3 * _time(torch, lambda: pdmp.morph_vjp(f, x0, T, eta, k, gT, ckpt=ck), reps=reps)
        else:
            out["ms"] = 1e3 * _time(torch, lambda: pdmp.logdet(f, x0, T, eta), reps=reps)
    elif case == "culled":
        lo, hi = np.zeros(2), np.full(2, 10.0)
        centres = wl.uniform_box(2, wl.S_CENTRES, M, lo, hi)
        boxes = wl.random_boxes(2, 64, lo, hi, 0.3, 1.5)
        f = pdmp.DeviceField.from_host(wl.Field(wl.RBF, centres, wl.proxy_fitted_weights(2, centres, boxes), gamma=8.0))
        x0 = torch.from_numpy(wl.uniform_box(2, wl.S_SAMPLES, 1 << 18, lo, hi)).cuda()
        r, _ = pdmp.cull_radius(f, 1e-6)
        out["ms"] = 1e3 * _time(torch, lambda: pdmp.morph_culled(f, x0, 3, 4.5e-4, r), reps=reps)
    elif case in ("vjp_rbf", "logdet_rbf"):
        lo, hi = np.zeros(2), np.full(2, 10.0)
        centres = wl.uniform_box(2, wl.S_CENTRES, M, lo, hi)
        boxes = wl.random_boxes(2, 64, lo, hi, 0.3, 1.5)
        f = pdmp.DeviceField.from_host(wl.Field(wl.RBF, centres, wl.proxy_fitted_weights(2, centres, boxes), gamma=8.0))
        x0 = torch.from_numpy(wl.uniform_box(2, wl.S_SAMPLES, 1 << 18, lo, hi)).cuda()
        if case == "vjp_rbf":
            ck = torch.empty(2, x0.shape[0], 2, device="cuda")
            pdmp.morph(f, x0, 4, 4.5e-4, ckpt=ck, k=2)
            gT = torch.ones_like(x0)
            out["ms"] = 1e3 * _time(torch, lambda: pdmp.morph_vjp(f, x0, 4, 4.5e-4, 2, gT, ckpt=ck), reps=reps)
        else:
            out["ms"] = 1e3 * _time(torch, lambda: pdmp.logdet(f, x0, 3, 4.5e-4), reps=reps)
    elif case == "inverse":
        lo, hi = np.zeros(2), np.full(2, 10.0)
        centres = wl.uniform_box(2, wl.S_CENTRES, M, lo, hi)
        boxes = wl.random_boxes(2, 64, lo, hi, 0.3, 1.5)
        f = pdmp.DeviceField.from_host(wl.Field(wl.RBF, centres, wl.proxy_fitted_weights(2, centres, boxes), gamma=8.0))
        x0 = torch.from_numpy(wl.uniform_box(2, wl.S_SAMPLES, 1 << 18, lo, hi)).cuda()
        z = pdmp.morph(f, x0, 2, 4.5e-4)
        out["ms"] = 1e3 * _time(torch, lambda: pdmp.morph_inverse(f, z, 2, 4.5e-4), reps=reps)
    elif case == "inverse_rff":
        wk = wl.config3(N=1 << 17)
        f = pdmp.DeviceField.from_host(wk.field)
        L, _ = pdmp.lipschitz_bound(f)
        eta = float(np.float32(0.5 / L))
        z = pdmp.morph(f, torch.from_numpy(wk.x0).cuda(), 4, eta)
        out["ms"] = 1e3 * _time(torch, lambda: pdmp.morph_inverse(f, z, 4, eta), reps=reps)
    elif case == "tanh":
        net = pdmp.DeviceTanhNet.from_host(wl.tanh_net(7, 2, 64))
        L, _ = pdmp.tanh_net_lipschitz(net)
        x0 = torch.from_numpy(wl.uniform_box(7, wl.S_SAMPLES, 1 << 18, np.zeros(2), np.full(2, 10.0))).cuda()
        out["ms"] = 1e3 * _time(torch, lambda: pdmp.tanh_net_morph(net, x0, 3, float(np.float32(0.5 / L))), reps=reps)
    elif case == "surrogate":
        # the 3-D surrogate end to end, as the extra runs it (training, plain morph, inference)
        import types
        out.update(extra_surrogate(pdmp, torch, types.SimpleNamespace(surrogate_steps=1500)))
    elif case == "mlp":
        # the surrogate network's inference kernel (random initial weights: the
        # kernel's work does not depend on their values) on 2^20 samples
        lo, hi = np.zeros(3), np.full(3, 5.0)
        net = pdmp.Surrogate(lo, hi, np.ones(3), seed=5)
        x0 = torch.from_numpy(wl.uniform_box(5, wl.S_SAMPLES, 1 << 20, lo, hi)).cuda()
        pred = torch.empty_like(x0)
        out["ms"] = 1e3 * _time(torch, lambda: net.forward(x0, out=pred), reps=reps)
    else:
        raise SystemExit(f"unknown case {case}")
    status, detail = pdmp.stream_status()
    if status != 0:
        raise RuntimeError(f"device status {status} ({detail})")
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched / RFF / surrogate measurements")
    ap.add_argument("--surrogate-steps", type=int, default=1500)
    ap.add_argument("--workload", choices=["full", "small"], default="full",
                    help="small: 262,144 samples and 3 steps of the same workload (for ncu captures)")
    ap.add_argument("--case", choices=["rff7d", "vjp", "logdet", "culled", "inverse", "inverse_rff", "vjp_rbf", "logdet_rbf",
                                       "tanh", "mlp", "surrogate"],
                    default=None,
                    help="run one small launch of that kernel family and exit (for ncu captures)")
    ap.add_argument("--case-reps", type=int, default=1, help="timed repetitions of --case (best of)")
    args = ap.parse_args()
    if args.case:
        profile_case(args.case, reps=args.case_reps)
        return
    if args.workload == "small":
        global N, T, WORKLOAD
        N, T = SMALL["N"], SMALL["T"]
        WORKLOAD = f"rbf2d-fitted-M{M}-N{N}-T{T}"
        args.no_cpu_baseline = True
        args.no_extras = True
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
