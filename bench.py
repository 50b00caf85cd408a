"""Benchmark of the THIIM E/H sweeps on one GB300 (or N independent replicas).

Workload (default): the 512^3 textured thin-film stack in complex128 — 12
split fields + 28 coefficient arrays, 86 GB resident in HBM — with the
plane-wave source; one step = thiim_iterate(200) followed by thiim_residual
(the FP64 relative update of the last iteration).  The headline computes in
FP64 (dtype f64), the paper's arithmetic.  GB300 executes FP64 at a small
fraction of its FP32 rate, so the line carries two rooflines for the sweep:
the FP64 pipe (instructions per cell against the pipe rate measured in the
same run) and HBM (832 algorithmic bytes per cell against the measured copy
bandwidth).  "variants" (the last key, numbers only) reports the other
arithmetic of the same data and the other configurations: FP32-pair
arithmetic on complex128 data, complex64, temporal blocking, the material
table, mixed precision with FP64 defect correction, the 32-solve batch, the
spectrum and the adjoint, each measured after one warm-up.  MLUP/s = cells x
iterations / time.  Every input array is larger than L2, so no flush is
needed between steps.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead
(the same metric on a bounded slab of the same workload, on the host cores).
"""
from __future__ import annotations

import argparse
import hashlib
import json
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
# material-table variant: 12 splits read + 12 written, one material-id byte
TABLE_BYTES_PER_LUP = {"c128": 24 * 16 + 1, "pair": 24 * 16 + 1, "c64": 24 * 8 + 1}
DTYPE = {"c128": "f64", "pair": "f32x2", "c64": "f32"}
PRECISION_CODE = {"c128": 0, "c64": 1, "pair": 2}
KERNEL = {"c128": "sweep_kernel<Native<double>>", "pair": "sweep_kernel<PairArith<1,1>>",
          "c64": "sweep_kernel<Native<float>>"}
# FP64 pipe instructions (DFMA, DADD, DMUL) per cell and iteration of the
# sweep's arithmetic without halo recomputation: per split 8 multiply-adds for
# t x + c D (+ Src) and 2 adds for the difference, plus 2 adds per full
# component sum (12 splits, 6 components): 12 * 10 + 6 * 2 = 132.
FP64_INSTR_PER_LUP = 132
PRECISION_NOTE = {"c128": "with native FP64 arithmetic",
                  "pair": "with FP32-pair arithmetic (parity with the FP64 oracle <= 1e-12)",
                  "c64": "stored as complex64 with FP32 arithmetic"}
FLOPS_PER_LUP = 248                                  # the paper's count (Sec. III-A)
SWEEP_SRC = [os.path.join(ROOT, "paper_1510_05218_gb300", "csrc", f) for f in ("thiim_sweep.cuh", "thiim_internal.h", "thiim_arith.cuh")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sweep_traffic.json")


def _sig(x, n=4):
    """x rounded to n significant digits (keeps the JSON line short)."""
    if x is None or x == 0 or x != x:
        return x
    return float("%.*g" % (n, x))


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
    """Hash of the sweep's source and of its tile configuration."""
    h = hashlib.sha256()
    for path in SWEEP_SRC:
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


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


def _cpu_model():
    """The host CPU as lscpu names it (for the CPU-baseline record)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    from workloads import stack_config
    st = stack_config(args.workload)
    threads = os.cpu_count() or 1
    planes = args.ref_planes
    rates, step_ms = [], []
    for _ in range(args.warmup):
        cpu_oracle_rate(st, planes, 2.0, threads)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r, info = cpu_oracle_rate(st, planes, args.ref_seconds, threads)
        step_ms.append((time.perf_counter() - t0) * 1e3)
        rates.append(r)
    value = statistics.median(rates)
    sample = ("oracle (plain C, OpenMP over z) on a %dx%dx%d slab (planes %d-%d) of the %s workload, "
              "%d iterations in %.1f s per step" % (st.nx, st.ny, planes, info["planes"][0], info["planes"][1],
                                                    args.workload, info["iters"], info["seconds"]))
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(step_ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "%s: %dx%dx%d textured thin-film stack, complex128" % (args.workload, st.nx, st.ny, st.nz),
                   "parallelism": "host cores",
                   "sample": "each step times a %d-plane slab of the full grid (the oracle at the full size "
                             "would take minutes per iteration); MLUP/s counts the slab's cells" % planes},
        "cpu_baseline": {"value": value, "unit": "MLUP/s", "cores": threads, "kind": "oracle", "sample": sample,
                         "cpu_model": _cpu_model()},
        "e2e": {"value": value, "unit": "MLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def _max_over_ranks(value, dev):
    """Max of a float over all ranks (NCCL on the GPU, or gloo on the CPU); the value itself at N = 1."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_mlups(world, cells, iters, steps, ms_total):
    """Whole-job throughput: every rank runs its own replica of the workload."""
    return world * cells * iters * steps / (ms_total / 1e3) / 1e6


def _clock_index(local):
    return local if os.environ.get("CUDA_VISIBLE_DEVICES") is None else 0


def _stack_problem(p, torch, st, precision, stream, dev, table=False):
    """Context + device arrays of a layered stack, coefficients built on the GPU
    (28 arrays, or with table=True a material map and (material, plane) table)."""
    prec = PRECISION_CODE[precision]
    dt = torch.complex64 if prec == p.THIIM_C64 else torch.complex128
    shape = (st.nz, st.ny, st.nx)
    ctx = p.thiim_create(st.nx, st.ny, st.nz, prec, 3, stream)
    fields = [torch.zeros(shape, dtype=dt, device=dev) for _ in range(12)]
    if table:
        em = st.material_eps()
        eps = torch.from_numpy(st.material_ids()).to(dev)     # the material map stands in for eps
        co = [torch.empty(len(em) * st.nz * 28, dtype=dt, device=dev)]
        with torch.cuda.stream(stream):
            p.thiim_build_material_table(ctx, em, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s,
                                         1.0, co[0])
        p.thiim_set_material_coeffs(ctx, eps, len(em), co[0])
    else:
        eps = torch.from_numpy(st.eps()).to(dev)
        co = [torch.empty(shape, dtype=dt, device=dev) for _ in range(28)]
        with torch.cuda.stream(stream):
            p.thiim_build_coeffs(ctx, eps, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s, 1.0, co)
        p.thiim_set_coeffs(ctx, co)
    p.thiim_set_fields(ctx, fields)
    torch.cuda.synchronize()
    return ctx, co, fields, eps


def _time_iterate(p, torch, ctx, stream, iters, warmup, steps):
    """CUDA-event time of thiim_iterate(iters) + thiim_residual, per step."""
    for _ in range(warmup):
        p.thiim_iterate(ctx, iters)
        p.thiim_residual(ctx)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = []
    t0.record(stream)
    for s in range(steps):
        ev[s][0].record(stream)
        p.thiim_iterate(ctx, iters)
        ev[s][1].record(stream)
        res.append(p.thiim_residual(ctx))
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1), sum(a.elapsed_time(b) for a, b in ev), res


def _variant_sweep(p, torch, st, precision, stream, dev, iters, warmup, steps, peak, temporal=1, autotune=True,
                   table=False):
    ctx, co, fields, eps = _stack_problem(p, torch, st, precision, stream, dev, table=table)
    choice = None
    if temporal != 1:
        p.thiim_set_tuning(ctx, temporal, 0)
        choice = (temporal, 0)
    elif autotune:
        from paper_1510_05218_gb300 import tuning
        choice, _ = tuning.autotune(ctx, fields, st.nx, st.ny, st.nz, PRECISION_CODE[precision], iters=20,
                                    repeats=1, stream=stream)
        if choice[0] != 1:          # keep this variant single-iteration; temporal blocking is its own line
            p.thiim_set_tuning(ctx, 1, choice[1])
    try:
        ms_total, ms_iter, res = _time_iterate(p, torch, ctx, stream, iters, warmup, steps)
    finally:
        p.thiim_destroy(ctx)
    cells = st.nx * st.ny * st.nz
    launch_s = ms_iter / 1e3 / (steps * iters)
    alg = (TABLE_BYTES_PER_LUP if table else BYTES_PER_LUP)[precision]
    achieved = alg * cells / launch_s / 1e9
    del co, fields, eps
    torch.cuda.empty_cache()
    return {"value": _sig(cells * iters * steps / (ms_total / 1e3) / 1e6), "dtype": DTYPE[precision],
            "frac_hbm": _sig(achieved / peak, 3), "launch_ms": _sig(launch_s * 1e3 * temporal),
            "tuning": list(choice) if choice else None}


def _variant_mixed(p, torch, st, stream, dev, inner, outer, warmup):
    """complex64 corrections with FP64 defect correction at this grid."""
    shape = (st.nz, st.ny, st.nx)
    eps = torch.from_numpy(st.eps()).to(dev)
    ctx64 = p.thiim_create(st.nx, st.ny, st.nz, p.THIIM_C128, 3, stream)
    co64 = [torch.empty(shape, dtype=torch.complex128, device=dev) for _ in range(28)]
    with torch.cuda.stream(stream):
        p.thiim_build_coeffs(ctx64, eps, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s, 1.0, co64)
    p.thiim_destroy(ctx64)
    ctx = p.thiim_create(st.nx, st.ny, st.nz, p.THIIM_C64, 3, stream)
    co32 = [torch.empty(shape, dtype=torch.complex64, device=dev) for _ in range(28)]
    work = [torch.zeros(shape, dtype=torch.complex64, device=dev) for _ in range(12)]
    x64 = [torch.zeros(shape, dtype=torch.complex128, device=dev) for _ in range(12)]
    try:
        with torch.cuda.stream(stream):
            p.thiim_build_coeffs(ctx, eps, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s, 1.0, co32)
        del eps
        p.thiim_set_coeffs(ctx, co32)
        p.thiim_set_fields(ctx, work)
        for _ in range(warmup):
            p.thiim_mixed_solve(ctx, co64, x64, inner, 1, 0.0)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        done, r = p.thiim_mixed_solve(ctx, co64, x64, inner, outer, 0.0)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
    finally:
        p.thiim_destroy(ctx)
    cells = st.nx * st.ny * st.nz
    del co64, co32, work, x64
    torch.cuda.empty_cache()
    return {"value": _sig(cells * inner * done / (ms / 1e3) / 1e6), "dtype": "f32+f64", "inner": inner,
            "residual": _sig(r, 3)}


def _variant_mixed_accuracy(p, torch, stream, dev):
    """complex64 against FP64, the accuracy half of the metric: the 32^3 stack
    solved by native FP64 (to residual 1e-11 or 300k iterations; ~1e-10
    reached) and by the mixed solver (complex64 corrections, FP64 defect every
    50, run to its residual floor), both on the GPU; the error is the relative
    L2 difference of each full component.  Stopping the mixed solve earlier,
    at residual 1e-7, measured 3.2e-6: the slow tail of the iteration."""
    from workloads import stack_config
    st = stack_config("stack32")
    shape = (st.nz, st.ny, st.nx)
    eps = torch.from_numpy(st.eps()).to(dev)
    args = (st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s, 1.0)
    t0 = time.perf_counter()
    ctx = p.thiim_create(st.nx, st.ny, st.nz, p.THIIM_C128, 3, stream)
    try:
        co64 = [torch.empty(shape, dtype=torch.complex128, device=dev) for _ in range(28)]
        f64 = [torch.zeros(shape, dtype=torch.complex128, device=dev) for _ in range(12)]
        with torch.cuda.stream(stream):
            p.thiim_build_coeffs(ctx, eps, *args, co64)
        p.thiim_set_tuning(ctx, 1, 4)
        p.thiim_set_coeffs(ctx, co64)
        p.thiim_set_fields(ctx, f64)
        it64, r64 = 0, 1.0
        while it64 < 300000 and r64 > 1e-11:
            p.thiim_iterate(ctx, 2500)
            it64 += 2500
            r64 = p.thiim_residual(ctx)
    finally:
        p.thiim_destroy(ctx)
    ctx = p.thiim_create(st.nx, st.ny, st.nz, p.THIIM_C64, 3, stream)
    try:
        co32 = [torch.empty(shape, dtype=torch.complex64, device=dev) for _ in range(28)]
        work = [torch.zeros(shape, dtype=torch.complex64, device=dev) for _ in range(12)]
        x64 = [torch.zeros(shape, dtype=torch.complex128, device=dev) for _ in range(12)]
        with torch.cuda.stream(stream):
            p.thiim_build_coeffs(ctx, eps, *args, co32)
        p.thiim_set_tuning(ctx, 1, 4)
        p.thiim_set_coeffs(ctx, co32)
        p.thiim_set_fields(ctx, work)
        # to the mixed solver's FP64-residual floor (about 5e-8 here): 2000 outer steps
        outer, rm = p.thiim_mixed_solve(ctx, co64, x64, 50, 2000, 1e-9)
    finally:
        p.thiim_destroy(ctx)
    torch.cuda.synchronize()
    errs = []
    for c in range(6):
        ref = f64[2 * c] + f64[2 * c + 1]
        mix = x64[2 * c] + x64[2 * c + 1]
        errs.append(float(torch.linalg.vector_norm(mix - ref) / torch.linalg.vector_norm(ref)))
    return {"max_rel_err": _sig(max(errs), 3), "bound": 1e-6, "grid": 32, "fp64_residual": _sig(r64, 2),
            "mixed_residual": _sig(rm, 2)}


def _variant_batch(p, torch, precision, stream, dev, iters, check, warmup):
    """The 32-solve spectrum sweep (uneven grids) in one persistent launch per iteration."""
    from workloads import batch_configs
    stacks = batch_configs(32, seed=1)
    probs = [_stack_problem(p, torch, st, precision, stream, dev) for st in stacks]
    ctxs = [pr[0] for pr in probs]
    cells = sum(st.nx * st.ny * st.nz for st in stacks)
    try:
        for _ in range(warmup):
            p.thiim_batch_iterate(ctxs, check, check, 0.0)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        its, res = p.thiim_batch_iterate(ctxs, iters, check, 0.0)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
    finally:
        for c in ctxs:
            p.thiim_destroy(c)
    del probs
    torch.cuda.empty_cache()
    return {"value": _sig(cells * iters / (ms / 1e3) / 1e6), "dtype": DTYPE[precision], "iters": iters,
            "residual_max": _sig(max(res), 3)}


def _variant_spectrum(p, torch, precision, n_lambda, iters):
    """Absorption spectrum of the 128^3 stack: n_lambda wavelengths x 2 polarisations
    in one batch, a fixed number of iterations each (wall clock of the whole call:
    coefficient builds, batched iterations, absorbed-power reductions)."""
    from paper_1510_05218_gb300.spectrum import absorption_spectrum
    from workloads import stack_config
    st = stack_config("stack128")
    eps = st.eps()
    lams = [st.lam * (0.8 + 0.8 * b / max(1, n_lambda - 1)) for b in range(n_lambda)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = absorption_spectrum(eps, lams, st.sigma_pml_e(), st.sigma_pml_h(), st.k_s, st.tau, st.absorber_mask(),
                            precision=PRECISION_CODE[precision], max_iters=iters, check_every=50, tol=0.0)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    torch.cuda.empty_cache()
    cells = st.nx * st.ny * st.nz
    solves = 2 * n_lambda
    return {"value": _sig(solves * cells * iters / dt / 1e6), "dtype": DTYPE[precision], "solves": solves,
            "A_first_last": [_sig(r["A_unpolarised"][0]), _sig(r["A_unpolarised"][-1])]}


def _variant_adjoint_steady(p, torch, stream, dev, terms, peak):
    """Steady-state adjoint on the 128^3 stack: `terms` propagation steps of
    thiim_adjoint_steady plus its one gradient evaluation (CUDA events)."""
    from workloads import stack_config
    st = stack_config("stack128")
    ctx, co, fields, eps = _stack_problem(p, torch, st, "c128", stream, dev)
    shape = (st.nz, st.ny, st.nx)
    try:
        lam = [torch.zeros(shape, dtype=torch.complex128, device=dev) for _ in range(6)] + \
              [torch.full(shape, 1e-3, dtype=torch.complex128, device=dev) for _ in range(6)]
        gco = [torch.zeros(shape, dtype=torch.complex128, device=dev) for _ in range(28)]
        p.thiim_adjoint_steady(ctx, lam, gco, fields, 2, 2, 0.0)      # warm-up (scratch allocation)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        p.thiim_adjoint_steady(ctx, lam, gco, fields, terms, terms, 0.0)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
    finally:
        p.thiim_destroy(ctx)
    del co, fields, eps, lam, gco
    torch.cuda.empty_cache()
    cells = st.nx * st.ny * st.nz
    # per term and cell: lam, lh, the running sum and the t, c arrays read; lam, lh, the sum written
    alg = (12 + 6 + 12 + 24) * 16 + (12 + 6 + 12) * 16
    return {"value": _sig(cells * terms / (ms / 1e3) / 1e6), "dtype": "f64",
            "frac_hbm": _sig(cells * terms * alg / (ms / 1e3) / 1e9 / peak, 3)}


def _variant_adjoint_checkpointed(p, torch, stream, dev, reps=2):
    """The inverse-design gradient of the adjoint workload (128^3, texture box,
    300 iterations, checkpoint every 20): coefficients from Re eps, the
    checkpointed solve, the absorbed power J and J.backward() (segment
    recomputation + reverse sweeps + the permittivity chain rule), timed with
    CUDA events after one warm-up gradient."""
    from paper_1510_05218_gb300.autograd import Differentiable
    from workloads import stack_config
    st = stack_config("adjoint128")
    eps = st.eps()
    sig_d = torch.from_numpy(st.omega * eps.imag * st.absorber_mask()).to(dev)
    args = (st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s, 1.0)
    n_it, every = 300, 20
    with torch.cuda.stream(stream):
        dmod = Differentiable(st.nx, st.ny, st.nz, stream=stream)
        eps_im = torch.from_numpy(eps.imag.copy()).to(dev)
        base = torch.from_numpy(eps.real.copy()).to(dev)

        def grad_once(evs=None):
            er = base.clone().requires_grad_(True)
            co = dmod.build_coeffs(er, eps_im, *args)
            x = dmod.solve(co, n_it, every)
            ex, ey, ez = x[6] + x[7], x[8] + x[9], x[10] + x[11]
            J = 0.5 * torch.sum(sig_d * (ex.abs() ** 2 + ey.abs() ** 2 + ez.abs() ** 2))
            if evs:
                evs[1].record(stream)
            J.backward()
            return er.grad

        try:
            grad_once()
            torch.cuda.synchronize()
            fwd, tot = [], []
            for _ in range(reps):
                evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                evs[0].record(stream)
                grad_once(evs)
                evs[2].record(stream)
                torch.cuda.synchronize()
                fwd.append(evs[0].elapsed_time(evs[1]))
                tot.append(evs[0].elapsed_time(evs[2]))
        finally:
            dmod.close()
    torch.cuda.empty_cache()
    cells = st.nx * st.ny * st.nz
    ms_f, ms_t = min(fwd), min(tot)
    return {"ms_forward": _sig(ms_f), "ms_backward": _sig(ms_t - ms_f), "gradients_per_s": _sig(1e3 / ms_t, 3),
            "value": _sig(cells * n_it / (ms_t / 1e3) / 1e6), "dtype": "f64"}


def run_grid_sweep(args):
    """MLUP/s against the cubic grid size (64^3 .. 512^3 in steps of 64), one
    JSON line per size and path — the GPU counterpart of the paper's grid-size
    experiment (Sec. IV-C, Fig. 7).  Not the benchmark's headline."""
    import torch

    import paper_1510_05218_gb300 as p
    from workloads import stack_config
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    p.load_library()
    stream = torch.cuda.Stream(device=dev)
    peak, _ = _peaks()
    modes = [("pair", 1), ("c64", 1), ("c64", 2), ("c128", 1)]
    for n in range(64, 513, 64):
        st = stack_config("stack%d" % n)
        cells = n ** 3
        for prec, temporal in modes:
            ctx, co, fields, eps = _stack_problem(p, torch, st, prec, stream, dev)
            del eps
            try:
                p.thiim_set_tuning(ctx, temporal, min(32, n))
                iters = max(20, min(200, int(2e10 / cells)))
                ms, _, res = _time_iterate(p, torch, ctx, stream, iters, 1, 2)
            finally:
                p.thiim_destroy(ctx)
            del co, fields
            torch.cuda.empty_cache()
            mlups = cells * iters * 2 / (ms / 1e3) / 1e6
            print(json.dumps({"grid": n, "precision": prec, "iterations_per_launch": temporal, "mlups": mlups,
                              "frac_hbm_alg": mlups * 1e6 * BYTES_PER_LUP[prec] / 1e9 / peak,
                              "iters": iters, "zchunk": min(32, n)}), flush=True)


def run_extended(args):
    """Configurations too long for the default run, one JSON line each:
    C2 — the 128^3 stack converged by native FP64 and by the mixed solver
    (complex64 corrections, FP64 defect every 50), relative L2 error of each
    full component of the mixed solution against the FP64 one; C3 — the
    32-solve batch (FP32-pair arithmetic on complex128 data, 1e-12 oracle
    parity) run toward relative residual 1e-8 with a bounded iteration count,
    each solve's residual recorded per chunk so that the iterations a solve
    still needs can be extrapolated from its asymptotic rate."""
    import math

    import torch

    import paper_1510_05218_gb300 as p
    from workloads import batch_configs, stack_config
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    p.load_library()
    stream = torch.cuda.Stream(device=dev)
    which = args.extended_configs.split(",")

    if "c2" in which:
        st = stack_config(args.c2_workload)
        shape = (st.nz, st.ny, st.nx)
        cells = st.nx * st.ny * st.nz
        eps = torch.from_numpy(st.eps()).to(dev)
        bargs = (st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s, 1.0)
        ctx = p.thiim_create(st.nx, st.ny, st.nz, p.THIIM_C128, 3, stream)
        co64 = [torch.empty(shape, dtype=torch.complex128, device=dev) for _ in range(28)]
        f64 = [torch.zeros(shape, dtype=torch.complex128, device=dev) for _ in range(12)]
        traj64 = []
        try:
            with torch.cuda.stream(stream):
                p.thiim_build_coeffs(ctx, eps, *bargs, co64)
            p.thiim_set_coeffs(ctx, co64)
            p.thiim_set_fields(ctx, f64)
            it64, r64, t0 = 0, 1.0, time.perf_counter()
            while it64 < args.c2_max_fp64 and r64 > args.c2_tol_fp64:
                p.thiim_iterate(ctx, 5000)
                it64 += 5000
                r64 = p.thiim_residual(ctx)
                traj64.append([it64, _sig(r64, 3)])
            sec64 = time.perf_counter() - t0
        finally:
            p.thiim_destroy(ctx)
        ctx = p.thiim_create(st.nx, st.ny, st.nz, p.THIIM_C64, 3, stream)
        co32 = [torch.empty(shape, dtype=torch.complex64, device=dev) for _ in range(28)]
        work = [torch.zeros(shape, dtype=torch.complex64, device=dev) for _ in range(12)]
        x64 = [torch.zeros(shape, dtype=torch.complex128, device=dev) for _ in range(12)]
        trajm = []
        try:
            with torch.cuda.stream(stream):
                p.thiim_build_coeffs(ctx, eps, *bargs, co32)
            p.thiim_set_coeffs(ctx, co32)
            p.thiim_set_fields(ctx, work)
            outer, rm, t0, best, stall = 0, 1.0, time.perf_counter(), 1.0, 0
            while outer < args.c2_max_outer and rm > args.c2_tol_fp64:
                done, rm = p.thiim_mixed_solve(ctx, co64, x64, args.c2_inner, 500, args.c2_tol_fp64)
                outer += done
                trajm.append([outer, _sig(rm, 3)])
                stall = stall + 1 if rm > 0.9 * best else 0     # floor reached: 2500 outer steps without 10 %
                best = min(best, rm)
                if done < 500 or stall >= 5:
                    break
            secm = time.perf_counter() - t0
        finally:
            p.thiim_destroy(ctx)
        torch.cuda.synchronize()
        names = ["Hx", "Hy", "Hz", "Ex", "Ey", "Ez"]
        errs = {}
        for c in range(6):
            ref = f64[2 * c] + f64[2 * c + 1]
            mix = x64[2 * c] + x64[2 * c + 1]
            errs[names[c]] = _sig(float(torch.linalg.vector_norm(mix - ref) / torch.linalg.vector_norm(ref)), 3)
        print(json.dumps({"config": "C2", "workload": "%s (%dx%dx%d)" % (args.c2_workload, st.nx, st.ny, st.nz),
                          "fp64": {"iterations": it64, "residual": _sig(r64, 3), "seconds": _sig(sec64, 3),
                                   "mlups": _sig(cells * it64 / sec64 / 1e6), "trajectory": traj64[::4]},
                          "mixed": {"outer_steps": outer, "inner_per_outer": args.c2_inner, "fp64_residual": _sig(rm, 3),
                                    "seconds": _sig(secm, 3), "trajectory": trajm},
                          "rel_l2_err_mixed_vs_fp64": errs, "max_err": max(errs.values()), "bound": 1e-6}),
              flush=True)
        del co64, f64, co32, work, x64, eps
        torch.cuda.empty_cache()

    if "diverge" in which:
        # where the last update of a non-converging stack lives: per z plane, per
        # material and per full component, after --diverge-iters FP64 iterations
        st = stack_config(args.c2_workload)
        shape = (st.nz, st.ny, st.nx)
        eps = torch.from_numpy(st.eps()).to(dev)
        ctx = p.thiim_create(st.nx, st.ny, st.nz, p.THIIM_C128, 3, stream)
        co = [torch.empty(shape, dtype=torch.complex128, device=dev) for _ in range(28)]
        f = [torch.zeros(shape, dtype=torch.complex128, device=dev) for _ in range(12)]
        try:
            with torch.cuda.stream(stream):
                p.thiim_build_coeffs(ctx, eps, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s, 1.0, co)
            p.thiim_set_coeffs(ctx, co)
            p.thiim_set_fields(ctx, f)
            done = 0
            while done < args.diverge_iters:
                n = min(10000, args.diverge_iters - done)
                p.thiim_iterate(ctx, n)
                done += n
            r0 = p.thiim_residual(ctx)
            torch.cuda.synchronize()
            prev = [t.clone() for t in f]
            p.thiim_iterate(ctx, 1)
            r1 = p.thiim_residual(ctx)
            torch.cuda.synchronize()
        finally:
            p.thiim_destroy(ctx)
        names = ["Hx", "Hy", "Hz", "Ex", "Ey", "Ez"]
        d2 = [((f[2 * c] + f[2 * c + 1]) - (prev[2 * c] + prev[2 * c + 1])).abs() ** 2 for c in range(6)]
        x2 = [(f[2 * c] + f[2 * c + 1]).abs() ** 2 for c in range(6)]
        dtot = sum(float(t.sum()) for t in d2)
        xtot = sum(float(t.sum()) for t in x2)
        dplane = sum(t.sum(dim=(1, 2)) for t in d2).cpu().numpy() / dtot
        xplane = sum(t.sum(dim=(1, 2)) for t in x2).cpu().numpy() / xtot
        ids = torch.from_numpy(st.material_ids()).to(dev)
        dsum = sum(d2)
        mat = {st.MATERIAL_ORDER[m]: _sig(float(dsum[ids == m].sum()) / dtot, 3) for m in range(4)}
        # split differences (Hxy - Hxz, ...): the undamped modes where sigma* = 0
        sd = sum(float(((f[2 * c] - f[2 * c + 1]) - (prev[2 * c] - prev[2 * c + 1])).abs().pow(2).sum())
                 for c in range(6))
        top = [int(k) for k in dplane.argsort()[::-1][:8]]
        print(json.dumps({"config": "diverge", "workload": "%s (%dx%dx%d)" % (args.c2_workload, st.nx, st.ny, st.nz),
                          "iterations": done, "residual": _sig(r0, 3), "residual_next": _sig(r1, 3),
                          "layers": {"pml_top": [0, st.L], "source_plane": st.k_s, "texture": [
                              _sig(float(st.z_top().min()), 3), _sig(float(st.z_top().max()), 3)],
                              "asi_end": st.z_asi_end, "glass_end": st.z_glass_end, "pml_bottom": [st.nz - st.L, st.nz]},
                          "update_share_by_material": mat,
                          "update_share_by_component": {names[c]: _sig(float(d2[c].sum()) / dtot, 3) for c in range(6)},
                          "split_difference_update_vs_full": _sig(sd / dtot, 3),
                          "top_update_planes": [[k, _sig(float(dplane[k]), 3), _sig(float(xplane[k]), 3)] for k in top],
                          "update_share_per_8_planes": [_sig(float(dplane[i:i + 8].sum()), 2)
                                                        for i in range(0, st.nz, 8)]}), flush=True)
        del co, f, prev, d2, x2, eps
        torch.cuda.empty_cache()

    if "pml" in which:
        # the same stack with other absorbing layers: cells x conductivity scale,
        # native FP64, residual every 10k iterations
        import dataclasses
        base = stack_config(args.c2_workload)
        for spec in args.pml_variants.split(","):
            cells, scale = spec.split(":")
            st = dataclasses.replace(base, pml_cells=int(cells))
            st.sigma_max *= float(scale)
            shape = (st.nz, st.ny, st.nx)
            eps = torch.from_numpy(st.eps()).to(dev)
            ctx = p.thiim_create(st.nx, st.ny, st.nz, p.THIIM_C128, 3, stream)
            co = [torch.empty(shape, dtype=torch.complex128, device=dev) for _ in range(28)]
            f = [torch.zeros(shape, dtype=torch.complex128, device=dev) for _ in range(12)]
            traj = []
            try:
                with torch.cuda.stream(stream):
                    p.thiim_build_coeffs(ctx, eps, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s,
                                         1.0, co)
                p.thiim_set_coeffs(ctx, co)
                p.thiim_set_fields(ctx, f)
                done = 0
                while done < args.diverge_iters:
                    p.thiim_iterate(ctx, 10000)
                    done += 10000
                    traj.append([done, _sig(p.thiim_residual(ctx), 3)])
            finally:
                p.thiim_destroy(ctx)
            print(json.dumps({"config": "pml", "workload": args.c2_workload, "pml_cells": st.L,
                              "sigma_max": _sig(st.sigma_max, 3), "trajectory": traj}), flush=True)
            del co, f, eps
            torch.cuda.empty_cache()

    if "c3" in which:
        stacks = batch_configs(32, seed=1)
        probs = [_stack_problem(p, torch, st, "pair", stream, dev) for st in stacks]
        ctxs = [pr[0] for pr in probs]
        active = list(range(len(ctxs)))
        its = [0] * len(ctxs)
        res = [1.0] * len(ctxs)
        traj = [[] for _ in ctxs]
        t0 = time.perf_counter()
        try:
            done_total = 0
            while active and done_total < args.c3_max_iters and time.perf_counter() - t0 < args.c3_max_seconds:
                chunk = min(args.c3_chunk, args.c3_max_iters - done_total)
                n, r = p.thiim_batch_iterate([ctxs[b] for b in active], chunk, 100, args.c3_tol)
                for b, nb, rb in zip(active, n, r):
                    its[b] += nb
                    res[b] = rb
                    traj[b].append([its[b], _sig(rb, 3)])
                active = [b for b in active if res[b] > args.c3_tol]
                done_total += chunk
        finally:
            for c in ctxs:
                p.thiim_destroy(c)
        sec = time.perf_counter() - t0
        rows = []
        for b, st in enumerate(stacks):
            row = {"grid": [st.nx, st.ny, st.nz], "lam": _sig(st.lam, 3), "iters": its[b],
                   "residual": _sig(res[b], 3), "converged": res[b] <= args.c3_tol}
            tr = traj[b]
            if not row["converged"] and len(tr) >= 2 and tr[-1][1] > 0 and tr[-2][1] > 0:
                rate = (math.log10(tr[-2][1]) - math.log10(tr[-1][1])) / (tr[-1][0] - tr[-2][0])
                row["decades_per_1e4_iters"] = _sig(rate * 1e4, 3)
                if rate > 0:
                    row["iters_to_tol_extrapolated"] = int(its[b] + (math.log10(res[b]) - math.log10(args.c3_tol))
                                                           / rate)
            rows.append(row)
        print(json.dumps({"config": "C3", "solves": len(stacks), "tol": args.c3_tol, "dtype": "f32x2",
                          "max_iters": args.c3_max_iters, "max_seconds": args.c3_max_seconds, "seconds": _sig(sec, 3),
                          "converged": sum(r["converged"] for r in rows), "per_solve": rows}), flush=True)
        del probs
        torch.cuda.empty_cache()


def run_one_variant(args):
    """One variant of the default run alone (for profiling), one JSON line."""
    import torch

    import paper_1510_05218_gb300 as p
    from workloads import stack_config
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    p.load_library()
    stream = torch.cuda.Stream(device=dev)
    peak, _ = _peaks()
    st = stack_config(args.workload)
    v = args.variant
    if v in ("pair", "c128", "c64"):
        r = _variant_sweep(p, torch, st, v, stream, dev, args.iters, 1, 1, peak)
    elif v == "c64_temporal2":
        r = _variant_sweep(p, torch, st, "c64", stream, dev, args.iters, 1, 1, peak, temporal=2)
    elif v in ("pair_table", "c64_table"):
        r = _variant_sweep(p, torch, st, v.split("_")[0], stream, dev, args.iters, 1, 1, peak, table=True)
    elif v == "mixed":
        r = _variant_mixed(p, torch, st, stream, dev, 50, 4, 1)
    elif v == "batch32":
        r = _variant_batch(p, torch, "pair", stream, dev, args.iters, 50, 1)
    elif v == "adjoint_steady_128":
        r = _variant_adjoint_steady(p, torch, stream, dev, args.iters, peak)
    elif v == "adjoint_ckpt_128":
        r = _variant_adjoint_checkpointed(p, torch, stream, dev)
    else:
        raise SystemExit("unknown variant %s" % v)
    print(json.dumps({"variant": v, **r}), flush=True)


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
    peak, peak_kind = _peaks()

    table = args.coeffs == "table"
    ctx, co, fields, eps = _stack_problem(p, torch, st, args.precision, stream, dev, table=table)
    tuning_info = None
    if args.fp64_int_ops:
        p.thiim_set_fp64_int_ops(ctx, args.fp64_int_ops)
    if args.temporal != 1 or args.zchunk:
        p.thiim_set_tuning(ctx, args.temporal, args.zchunk)
        tuning_info = {"choice": [args.temporal, args.zchunk], "source": "command line"}
    elif not args.no_autotune:
        from paper_1510_05218_gb300 import tuning
        choice, times = tuning.autotune(ctx, fields, st.nx, st.ny, st.nz, PRECISION_CODE[args.precision],
                                        iters=20, repeats=2, stream=stream)
        tuning_info = {"choice": list(choice), "source": "autotune (footprint-model candidates, timed)",
                       "seconds_per_20_iterations": {"%d/%d" % k: round(v, 5) for k, v in times.items()}}
    eps_pinned = eps.cpu().pin_memory()
    sig_e, sig_h = st.sigma_pml_e(), st.sigma_pml_h()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # --- device-resident timing -------------------------------------------
    for _ in range(args.warmup):
        p.thiim_iterate(ctx, iters)
        p.thiim_residual(ctx)
    torch.cuda.synchronize()
    # the FP64 pipe's measured rate, right after the warm-up (same clocks)
    fp64_rate = p.thiim_fp64_pipe_rate(stream) if args.precision == "c128" else None
    sampler = ClockSampler(_clock_index(local))
    sampler.start()
    time.sleep(0.3)
    barrier()
    ms_total, ms_iter_calls, residuals = _time_iterate(p, torch, ctx, stream, iters, 0, args.steps)
    barrier()
    clocks = sampler.stop()
    ms_total = _max_over_ranks(ms_total, dev)
    ms_step = ms_total / args.steps
    value = _job_mlups(world, cells, iters, args.steps, ms_total)

    # roofline of the dominant kernel (the fused sweep): one launch per iteration
    launch_s = ms_iter_calls / 1e3 / (args.steps * iters)
    alg_per_lup = (TABLE_BYTES_PER_LUP if table else BYTES_PER_LUP)[args.precision]
    achieved = alg_per_lup * cells / launch_s / 1e9
    kernel_key = KERNEL[args.precision][:-1] + ", table>" if table else KERNEL[args.precision]
    traffic = _traffic(kernel_key, cells)
    hbm = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": traffic, "peak_kind": peak_kind, "kernel": kernel_key, "alg_bytes_per_lup": alg_per_lup,
           "launch_ms": launch_s * 1e3}
    if fp64_rate:
        # FP64 arithmetic: the sweep is bound by the FP64 pipe, not by HBM
        achieved_fp64 = FP64_INSTR_PER_LUP * cells / launch_s / 1e9
        roofline = {"bound": "fp64_pipe", "achieved": achieved_fp64, "peak": fp64_rate / 1e9,
                    "unit": "G FP64 instr/s", "frac": achieved_fp64 * 1e9 / fp64_rate, "traffic": traffic,
                    "peak_kind": "measured in this run (thiim_fp64_pipe_rate: DFMA throughput, all SMs)",
                    "kernel": kernel_key, "alg_fp64_instr_per_lup": FP64_INSTR_PER_LUP,
                    "launch_ms": launch_s * 1e3,
                    "hbm": {k: hbm[k] for k in ("achieved", "peak", "unit", "frac", "peak_kind",
                                                "alg_bytes_per_lup")}}
    else:
        roofline = hbm

    # --- end to end through the public API with host buffers --------------
    e2e = None
    if not args.no_e2e:
        host_fields = [torch.empty(shape, dtype=dt).pin_memory() for _ in range(12)]
        h2d = eps_pinned.numel() * eps_pinned.element_size() + 2 * st.nz * 8
        d2h = sum(t.numel() * t.element_size() for t in host_fields)
        e2e_times = []
        for s in range(args.e2e_warmup + args.e2e_steps):
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                eps.copy_(eps_pinned, non_blocking=True)       # permittivity map, or material ids
                if table:
                    p.thiim_build_material_table(ctx, st.material_eps(), sig_e, sig_h, st.omega, st.tau, st.k_s,
                                                 1.0, co[0])
                    p.thiim_set_material_coeffs(ctx, eps, len(st.material_eps()), co[0])
                else:
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
            el = _max_over_ranks(time.perf_counter() - t0, dev)
            if s >= args.e2e_warmup:
                e2e_times.append(el)
        e2e = {"value": world * cells * iters / statistics.median(e2e_times) / 1e6, "unit": "MLUP/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "steps": args.e2e_steps,
               "what": ("H2D material-id map, thiim_build_material_table" if table else
                        "H2D permittivity map, thiim_build_coeffs") +
                       ", zero fields, thiim_iterate(%d), thiim_residual, D2H of the 12 fields" % iters}
        del host_fields

    p.thiim_destroy(ctx)
    del co, fields, eps
    torch.cuda.empty_cache()

    variants = {}
    if not args.no_variants:
        # FP32-pair arithmetic on the same complex128 data first: FP64-accurate
        # (1e-12 parity with the oracle), narrower exponent range than FP64
        for mode in ("pair", "c128", "c64"):
            if mode != args.precision:
                variants[mode] = _variant_sweep(p, torch, st, mode, stream, dev, iters, 1, 1, peak)
        variants["c64_temporal2"] = _variant_sweep(p, torch, st, "c64", stream, dev, iters, 1, 1, peak, temporal=2)
        for mode in ("pair", "c64"):
            variants[mode + "_table"] = _variant_sweep(p, torch, st, mode, stream, dev, iters, 1, 1, peak,
                                                       table=True)
        variants["mixed"] = _variant_mixed(p, torch, st, stream, dev, 50, 4, 1)
        variants["mixed"]["accuracy"] = _variant_mixed_accuracy(p, torch, stream, dev)
        bprec = "pair" if args.precision == "c128" else args.precision
        variants["batch32"] = _variant_batch(p, torch, bprec, stream, dev, 200, 50, 1)
        variants["spectrum16x2"] = _variant_spectrum(p, torch, bprec, 16, 200)
        variants["adjoint_steady_128"] = _variant_adjoint_steady(p, torch, stream, dev, 200, peak)
        variants["adjoint_ckpt_128"] = _variant_adjoint_checkpointed(p, torch, stream, dev)

    if rank != 0:
        return

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        threads = os.cpu_count() or 1
        rate, info = cpu_oracle_rate(st, args.ref_planes, args.ref_seconds, threads)
        rate1, info1 = cpu_oracle_rate(st, 2, 3.0, 1)
        cpu = {"value": rate, "unit": "MLUP/s", "cores": threads, "kind": "oracle", "cpu_model": _cpu_model(),
               "single_thread": {"value": rate1, "sample": "%d iterations of a %dx%dx2 slab in %.1f s"
                                 % (info1["iters"], st.nx, st.ny, info1["seconds"])},
               "sample": "plain C FP64 oracle, OpenMP over z, on a %dx%dx%d slab (planes %d-%d) of the same "
                         "stack, %d iterations in %.1f s" % (st.nx, st.ny, args.ref_planes, info["planes"][0],
                                                             info["planes"][1], info["iters"], info["seconds"])}

    out = {
        "metric": METRIC, "value": value, "unit": "MLUP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": "%s: %dx%dx%d textured thin-film stack (seeded sinusoid texture), complex128 data "
                               "%s, %d THIIM iterations + FP64 residual per step" % (
                                   args.workload, st.nx, st.ny, st.nz, PRECISION_NOTE[args.precision], iters),
                   "grid": [st.nx, st.ny, st.nz], "iters_per_step": iters, "precision": args.precision,
                   "kernel": "fused out-of-place z-streaming sweep, one launch per iteration",
                   "coefficients": ("material-id map (1 B/cell) + (material, plane) table: a variant, not the "
                                    "paper's 28-array layout" if table else "28 arrays (the paper's layout)"),
                   "tuning": tuning_info,
                   "l2": "inputs larger than L2 (no flush needed)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline,
        "gflops_paper_count": value * FLOPS_PER_LUP / 1e3,
        "residual_last": residuals[-1] if residuals else None,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": args.steps * (iters + 1),
        "cpu_baseline": cpu,
        "variants_legend": ("MLUP/s of the same 512^3 stack in other arithmetic (pair: FP32 pairs on complex128 "
                            "data, 1e-12 oracle parity; c64: complex64), with 2 iterations per launch, with "
                            "material-table coefficients, mixed c64 + FP64 defect (accuracy: 32^3 converged, vs "
                            "FP64), 32 uneven batched solves, a 16x2 spectrum, the steady adjoint at 128^3 and "
                            "the checkpointed inverse-design gradient (128^3, 300 iterations, checkpoint every "
                            "20; value = forward LUP / gradient time); frac_hbm uses the single-iteration "
                            "algorithmic bytes"),
        "variants": variants,
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
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--coeffs", default="arrays", choices=["arrays", "table"],
                    help="table: material-id map + (material, plane) table (a variant, not the headline layout)")
    ap.add_argument("--temporal", type=int, default=1, help="iterations per launch (2: complex64 only)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--grid-sweep", action="store_true", help="MLUP/s vs grid size 64^3..512^3 (not the headline)")
    ap.add_argument("--zchunk", type=int, default=0, help="z planes per CTA (0: library default)")
    ap.add_argument("--fp64-int-ops", type=int, default=0,
                    help="complex128: binary64 adds (1) or adds and products (3) on the integer pipe "
                         "(bit-identical; thiim_set_fp64_int_ops)")
    ap.add_argument("--variant", default="", help="run one entry of the variants alone (profiling)")
    ap.add_argument("--extended-configs", default="",
                    help="c2,c3,diverge,pml: convergence runs, the growing-mode diagnosis and absorbing-layer variants "
                         "(minutes; not the headline)")
    ap.add_argument("--c2-workload", default="stack128")
    ap.add_argument("--c2-tol-fp64", type=float, default=1e-11)
    ap.add_argument("--c2-max-fp64", type=int, default=700000)
    ap.add_argument("--c2-max-outer", type=int, default=20000)
    ap.add_argument("--c2-inner", type=int, default=50, help="complex64 iterations per FP64 defect")
    ap.add_argument("--c3-tol", type=float, default=1e-8)
    ap.add_argument("--diverge-iters", type=int, default=200000)
    ap.add_argument("--pml-variants", default="24:1,24:4,6:1", help="absorbing-layer cells:conductivity scale")
    ap.add_argument("--c3-max-iters", type=int, default=24000)
    ap.add_argument("--c3-chunk", type=int, default=4000)
    ap.add_argument("--c3-max-seconds", type=float, default=1e9, help="stop C3 after this wall time")
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
    elif args.grid_sweep:
        run_grid_sweep(args)
    elif args.extended_configs:
        run_extended(args)
    elif args.variant:
        run_one_variant(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
