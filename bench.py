"""Benchmark of the THIIM E/H sweeps on one GB300 (or N independent replicas).

Workload (default): the 512^3 textured thin-film stack in complex128 — 12
split fields + 28 coefficient arrays, 86 GB resident in HBM — with the
plane-wave source; one step = thiim_iterate(200) followed by thiim_residual
(the FP64 relative update of the last iteration).  MLUP/s = cells x
iterations / time.  Every input array is larger than L2, so no flush is
needed between steps.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead
(the same metric on a bounded slab of the same workload, on the host cores).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "THIIM E+H MLUP/s at 512^3 and % of HBM roofline; complex64 vs FP64 at ≤1e-6"
BYTES_PER_LUP = {"c128": 52 * 16, "pair": 52 * 16, "c64": 52 * 8}   # 40 arrays read + 12 written per cell
DTYPE = {"c128": "f64", "pair": "f32x2", "c64": "f32"}
PRECISION_CODE = {"c128": 0, "c64": 1, "pair": 2}
KERNEL = {"c128": "sweep_kernel<Native<double>>", "pair": "sweep_kernel<PairArith<1,1>>",
          "c64": "sweep_kernel<Native<float>>"}
FLOPS_PER_LUP = 248                                  # the paper's count (Sec. III-A)
SWEEP_SRC = os.path.join(ROOT, "paper_1510_05218_gb300", "csrc", "thiim_sweep.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sweep_traffic.json")


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _sweep_sha():
    with open(SWEEP_SRC, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def _traffic(kernel_key, cells):
    """DRAM bytes per launch from the committed ncu summary, if it matches the source."""
    try:
        with open(TRAFFIC_FILE) as fh:
            d = json.load(fh)
        e = d[kernel_key]
        if e.get("src_sha") != _sweep_sha():
            return None
        return float(e["bytes_per_cell"]) * cells
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def cpu_oracle_rate(stack, planes, target_s, threads):
    """Oracle MLUP/s on a slab of `planes` z-planes (full x, y) of the stack."""
    import numpy as np

    import oracle
    from oracle.coeffs import build_coeffs
    k0 = max(0, min(stack.nz - planes, stack.k_s - planes // 2))
    k1 = k0 + planes
    eps = stack.eps_planes(k0, k1)
    tf = (stack.k_s - k0, 1.0) if k0 <= stack.k_s < k1 else None
    co = build_coeffs(eps, stack.sigma_pml_e()[k0:k1], stack.sigma_pml_h()[k0:k1], stack.omega, stack.tau, tfsf=tf)
    f = [np.zeros(eps.shape, np.complex128) for _ in range(12)]
    oracle.iterate(f, co, 1, bc=3, nthreads=threads)          # warm-up
    cells = eps.size
    done, t0 = 0, time.perf_counter()
    while True:
        oracle.iterate(f, co, 1, bc=3, nthreads=threads)
        done += 1
        el = time.perf_counter() - t0
        if el >= target_s or done >= 10000:
            break
    return cells * done / el / 1e6, dict(planes=[k0, k1], cells=cells, iters=done, seconds=el)


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    from workloads import stack_config
    st = stack_config(args.workload)
    threads = os.cpu_count() or 1
    planes = args.ref_planes
    rates = []
    for _ in range(args.warmup):
        cpu_oracle_rate(st, planes, 2.0, threads)
    for _ in range(args.steps):
        r, info = cpu_oracle_rate(st, planes, args.ref_seconds, threads)
        rates.append(r)
    value = statistics.median(rates)
    sample = ("oracle (plain C, OpenMP over z) on a %dx%dx%d slab (planes %d-%d) of the %s workload, "
              "%d iterations in %.1f s per step" % (st.nx, st.ny, planes, info["planes"][0], info["planes"][1],
                                                    args.workload, info["iters"], info["seconds"]))
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": args.ref_seconds * 1000.0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "%s: %dx%dx%d textured thin-film stack, complex128" % (args.workload, st.nx, st.ny, st.nz),
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": "MLUP/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "MLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    import paper_1510_05218_gb300 as p
    from workloads import stack_config

    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p.load_library()

    st = stack_config(args.workload)
    prec = PRECISION_CODE[args.precision]
    dt = torch.complex64 if prec == p.THIIM_C64 else torch.complex128
    shape = (st.nz, st.ny, st.nx)
    cells = st.nx * st.ny * st.nz
    iters = args.iters
    stream = torch.cuda.Stream(device=dev)

    eps_host = torch.from_numpy(st.eps())
    eps_pinned = eps_host.pin_memory()
    del eps_host
    eps = eps_pinned.to(dev)
    ctx = p.thiim_create(st.nx, st.ny, st.nz, prec, 3, stream)
    co = [torch.empty(shape, dtype=dt, device=dev) for _ in range(28)]
    fields = [torch.zeros(shape, dtype=dt, device=dev) for _ in range(12)]
    sig_e, sig_h = st.sigma_pml_e(), st.sigma_pml_h()
    with torch.cuda.stream(stream):
        p.thiim_build_coeffs(ctx, eps, sig_e, sig_h, st.omega, st.tau, st.k_s, 1.0, co)
    p.thiim_set_coeffs(ctx, co)
    p.thiim_set_fields(ctx, fields)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # --- device-resident timing -------------------------------------------
    for _ in range(args.warmup):
        p.thiim_iterate(ctx, iters)
        p.thiim_residual(ctx)
    torch.cuda.synchronize()
    sampler = ClockSampler(local if os.environ.get("CUDA_VISIBLE_DEVICES") is None else 0)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_stop = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    residuals = []
    for s in range(args.steps):
        ev[s][0].record(stream)
        p.thiim_iterate(ctx, iters)
        ev[s][1].record(stream)
        residuals.append(p.thiim_residual(ctx))
    t_stop.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms_total = t_start.elapsed_time(t_stop)
    ms_iter_calls = sum(a.elapsed_time(b) for a, b in ev)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms_total], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    value = world * cells * iters * args.steps / (ms_total / 1e3) / 1e6

    # roofline of the dominant kernel (the fused sweep): one launch per iteration
    launch_s = ms_iter_calls / 1e3 / (args.steps * iters)
    alg_bytes = BYTES_PER_LUP[args.precision] * cells
    peak, peak_kind = _peaks()
    achieved = alg_bytes / launch_s / 1e9
    kernel_key = KERNEL[args.precision]
    traffic = _traffic(kernel_key, cells)

    # --- end to end through the public API with host buffers --------------
    e2e = None
    if not args.no_e2e:
        host_fields = [torch.empty(shape, dtype=dt).pin_memory() for _ in range(12)]
        h2d = eps_pinned.numel() * 16 + 2 * st.nz * 8
        d2h = sum(t.numel() * t.element_size() for t in host_fields)
        e2e_times = []
        for s in range(args.e2e_warmup + args.e2e_steps):
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                eps.copy_(eps_pinned, non_blocking=True)
                p.thiim_build_coeffs(ctx, eps, sig_e, sig_h, st.omega, st.tau, st.k_s, 1.0, co)
                for f in fields:
                    f.zero_()
            p.thiim_set_fields(ctx, fields)
            p.thiim_iterate(ctx, iters)
            p.thiim_residual(ctx)
            with torch.cuda.stream(stream):
                for hf, f in zip(host_fields, fields):
                    hf.copy_(f, non_blocking=True)
            stream.synchronize()
            el = time.perf_counter() - t0
            if world > 1:
                import torch.distributed as dist
                t = torch.tensor([el], device=dev, dtype=torch.float64)
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                el = float(t.item())
            if s >= args.e2e_warmup:
                e2e_times.append(el)
        e2e = {"value": world * cells * iters / statistics.median(e2e_times) / 1e6, "unit": "MLUP/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "steps": args.e2e_steps,
               "what": "H2D permittivity map, thiim_build_coeffs, zero fields, thiim_iterate(%d), "
                       "thiim_residual, D2H of the 12 fields" % iters}
        del host_fields

    p.thiim_destroy(ctx)
    if rank != 0:
        return

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        threads = os.cpu_count() or 1
        rate, info = cpu_oracle_rate(st, args.ref_planes, args.ref_seconds, threads)
        cpu = {"value": rate, "unit": "MLUP/s", "cores": threads, "kind": "oracle",
               "sample": "plain C FP64 oracle, OpenMP over z, on a %dx%dx%d slab (planes %d-%d) of the same "
                         "stack, %d iterations in %.1f s" % (st.nx, st.ny, args.ref_planes, info["planes"][0],
                                                             info["planes"][1], info["iters"], info["seconds"])}

    out = {
        "metric": METRIC, "value": value, "unit": "MLUP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": "%s: %dx%dx%d textured thin-film stack (seeded sinusoid texture), %s, "
                               "%d THIIM iterations + FP64 residual per step" % (
                                   args.workload, st.nx, st.ny, st.nz, args.precision, iters),
                   "grid": [st.nx, st.ny, st.nz], "iters_per_step": iters, "precision": args.precision,
                   "kernel": "fused out-of-place z-streaming sweep, one launch per iteration",
                   "l2": "inputs larger than L2 (no flush needed)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": kernel_key, "alg_bytes_per_lup": BYTES_PER_LUP[args.precision],
                     "launch_ms": launch_s * 1e3},
        "gflops_paper_count": value * FLOPS_PER_LUP / 1e3,
        "residual_last": residuals[-1] if residuals else None,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": args.steps * (iters + 1),
        "cpu_baseline": cpu,
    }
    print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="stack512")
    ap.add_argument("--precision", default="c128", choices=["c128", "pair", "c64"])
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--e2e-warmup", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-planes", type=int, default=16)
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
