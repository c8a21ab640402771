"""Throughput benchmark of the two-fluid D3Q19 colour-gradient step.

One bench "step" is one lattice time step (all of: pull streaming, moments,
gradients, collision, perturbation, recolouring, store) over the whole
lattice.  Workload (default): moving droplet in uniform flow, 128^3 periodic,
radius 20, background velocity (0.05, 0, 0), density ratio 10, viscosity
ratio 1, sigma = 0.005, beta = 0.7, FP32 storage and arithmetic.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--storage f32|f16|bf16] [--kernel fused|two_pass] [--n 128]

Prints one JSON line.  `value` is whole-job MLUPS with the populations
resident in HBM (inputs of 637 MB, larger than the 129 MB L2, so no flush is
needed between steps); `e2e` is the same metric through the C ABI with host
buffers (initial fields uploaded from pinned host memory, every step's FP64
diagnostics copied back into pinned host memory in stream order through
lbm_step_diagnostics_async, final moments downloaded, all inside the timed
region).  Multi-GPU runs are independent replicas (one lattice per rank):
the step has no cross-lattice exchange.
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("MLUPS (two-fluid D3Q19) and % of HBM roofline; FP16-store vs FP32 "
          "at stated error")
BYTES_PER_VALUE = {"f32": 4, "f16": 2, "bf16": 2}


def workload(n):
    """Moving droplet in uniform flow (density ratio 10, sigma = 0.005)."""
    return dict(nx=n, ny=n, nz=n, wall=(0, 0, 0), improved=True,
                rho_in_R=10.0, rho_in_B=1.0, alpha_R=0.97, alpha_B=0.7,
                tau_R=1.0, tau_B=1.0, tau_e=1.0, tau_q=1.0, tau_pi=1.0,
                A_R=0.01125, A_B=0.01125, beta=0.7, delta=0.98,
                force=(0.0, 0.0, 0.0), gravity=(0.0, 0.0, 0.0))


def storage_references(storage, rho_in_R, rho_in_B, rho_R, rho_B):
    """Deviation references for FP16/BF16 storage: the colour with more mass
    (the background phase) is stored as f - rho_in phi, the other as is, so
    that the absent colour stays exactly zero."""
    if storage == "f32":
        return 0.0, 0.0
    return (rho_in_R, 0.0) if rho_R.sum() >= rho_B.sum() else (0.0, rho_in_B)


def workload_fields(n):
    from paper_1904_03618_gb300 import workloads
    return workloads.droplet(n, n, n, 20.0 * n / 128.0, 10.0, 1.0,
                             velocity=(0.05, 0.0, 0.0))


# ---------------------------------------------------------------------------
class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        if not shutil.which("nvidia-smi"):
            return
        self.proc = subprocess.Popen(
            ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
             "--format=csv,noheader,nounits", "-lms", "100"],
            stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profiled_traffic(kernel, storage, n):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel (source hash recorded beside it)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "fused_step_traffic.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    h = hashlib.sha256()
    for f in ("lbm_fused.cuh", "lbm_fused_tma.cuh", "lbm_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1904_03618_gb300", "csrc", f), "rb").read())
    key = "%s_%s" % (kernel, storage)
    if vals.get("source_sha256") != h.hexdigest()[:16] or key + "_bytes_per_cell" not in vals:
        return None
    return float(vals[key + "_bytes_per_cell"]) * n ** 3


# ---------------------------------------------------------------------------
def cpu_oracle_sample(n_sample, seconds):
    """Time the FP64 oracle, as it stands, on the host cores on a bounded
    sample of the workload (a smaller cube of the same case)."""
    import oracle
    from paper_1904_03618_gb300 import workloads
    pd = workload(n_sample)
    p = oracle.params_from(pd)
    rR, rB, u = workloads.droplet(n_sample, n_sample, n_sample, 20.0 * n_sample / 128.0,
                                  10.0, 1.0, velocity=(0.05, 0.0, 0.0))
    f = oracle.init(p, rR, rB, u)
    t0 = time.perf_counter()
    f = oracle.step(p, f, 1)
    one = time.perf_counter() - t0
    steps = max(1, int(seconds / max(one, 1e-6)))
    t0 = time.perf_counter()
    f = oracle.step(p, f, steps)
    dt = time.perf_counter() - t0
    cells = n_sample ** 3 * steps
    return {"value": cells / dt / 1e6, "unit": "MLUPS", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "%d^3 lattice of the same case, %d steps, %.1f s" % (
                n_sample, steps, dt)}, steps, dt


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle, as it stands, on the host cores.  Each
    bench step is one oracle time step on a cube of the same case whose size
    is chosen so that warm-up plus timed steps take about two minutes."""
    if rank != 0:
        return
    import oracle
    from paper_1904_03618_gb300 import workloads
    probe = 24
    pp = oracle.params_from(workload(probe))
    fr, fb, fu = workloads.droplet(probe, probe, probe, 20.0 * probe / 128.0, 10.0, 1.0,
                                   velocity=(0.05, 0.0, 0.0))
    fp = oracle.init(pp, fr, fb, fu)
    t0 = time.perf_counter()
    oracle.step(pp, fp, 2)
    rate = 2 * probe ** 3 / (time.perf_counter() - t0)
    budget = 120.0 / (args.steps + args.warmup)
    ns = int(max(8, min(args.n, (rate * budget) ** (1.0 / 3.0))))
    pd = workload(ns)
    p = oracle.params_from(pd)
    rR, rB, u = workloads.droplet(ns, ns, ns, 20.0 * ns / 128.0, 10.0, 1.0,
                                  velocity=(0.05, 0.0, 0.0))
    f = oracle.init(p, rR, rB, u)
    for _ in range(args.warmup):
        f = oracle.step(p, f, 1)
    per_step = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        f = oracle.step(p, f, 1)
        per_step.append(time.perf_counter() - t0)
    mean = statistics.mean(per_step)
    mlups = ns ** 3 / mean / 1e6
    cb = {"value": mlups, "unit": "MLUPS", "cores": oracle.num_threads(),
          "kind": "oracle",
          "sample": "each step: one FP64 oracle step on a %d^3 cube of the same case "
                    "(%d steps timed)" % (ns, args.steps)}
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * mean, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_block(args, world), "cpu_baseline": cb,
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_block(args, world):
    return {"workload": "moving droplet in uniform flow, %d^3 periodic D3Q19 two-fluid, "
                        "R=%g, u=(0.05,0,0), density ratio 10, viscosity ratio 1, "
                        "sigma=0.005, beta=0.7" % (args.n, 20.0 * args.n / 128.0),
            "lattice": [args.n, args.n, args.n], "storage": args.storage,
            "kernel": args.kernel, "fused_config": args.fused_config or "library default",
            "model": "improved (Eq. 18 + Eq. 45 correction)",
            "parallelism": "replicas x%d" % world if world > 1 else "single GPU",
            "l2_policy": "inputs larger than L2 (%.0f MB populations)" % (
                args.n ** 3 * 38 * BYTES_PER_VALUE[args.storage] / 1e6)}


# ---------------------------------------------------------------------------
# Replica bookkeeping of N > 1 runs (no data-path collective: each rank
# advances its own lattice; only the timings meet).
def max_over_ranks(value, dist, device=None):
    """The largest of the ranks' values (every rank gets it)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world, cells_per_rank, seconds):
    """Cell updates of all ranks over the slowest rank's time, in MLUPS."""
    return world * cells_per_rank / seconds / 1e6


# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1904_03618_gb300 import lbm

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    n = args.n
    N = n ** 3
    pd = workload(n)
    rR, rB, u = (np.ascontiguousarray(a, dtype=np.float32) for a in workload_fields(n))
    params = lbm.make_params(storage=args.storage, kernel=args.kernel, **pd)
    params.ref_R, params.ref_B = storage_references(args.storage, pd["rho_in_R"],
                                                    pd["rho_in_B"], rR, rB)
    stream = torch.cuda.Stream(dev)
    lat = lbm.Lattice(params, device=dev, stream=stream)
    if args.kernel == "fused" and args.fused_config:
        ty, zc, hold = (int(v) for v in args.fused_config.split(","))
        lbm.lbm_set_fused_config(lat.ctx, ty, zc, hold)
    lat.init_fields(rR, rB, u)
    launches = lbm.lbm_launches_per_step(lat.ctx)

    # --- device-resident throughput -------------------------------------
    for _ in range(args.warmup):
        lbm.lbm_step(lat.ctx, 1)
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sampler = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ
                           else int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local_rank]))
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize(dev)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        lbm.lbm_step(lat.ctx, 1)
        ev[k][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    total_ms = t_start.elapsed_time(t_end)
    launch_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    diag = lat.diagnostics(raise_unstable=False)
    total_ms = max_over_ranks(total_ms, dist, dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_mlups(world, N, ms_per_step * 1e-3)

    # --- end to end through the C ABI with host buffers -------------------
    pin = lambda a: torch.from_numpy(a).pin_memory()  # noqa: E731
    hR, hB, hu = pin(rR), pin(rB), pin(u)
    oR = torch.empty(rR.shape, dtype=torch.float32).pin_memory()
    oB = torch.empty(rB.shape, dtype=torch.float32).pin_memory()
    ou = torch.empty(u.shape, dtype=torch.float32).pin_memory()
    e2e_steps = max(args.steps // 4, 10)
    monitor = torch.zeros((e2e_steps, 16), dtype=torch.float64).pin_memory()
    lbm.lbm_init_fields(lat.ctx, hR, hB, hu)  # warm the staging buffers
    lbm.lbm_moments(lat.ctx, oR, oB, ou)
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    lbm.lbm_init_fields(lat.ctx, hR, hB, hu)
    for k in range(e2e_steps):
        # one step, its diagnostics and their copy into pinned host memory,
        # queued without a host wait
        lbm.lbm_step_diagnostics_async(lat.ctx, 1, monitor[k])
    lbm.lbm_moments(lat.ctx, oR, oB, ou)
    lbm.lbm_sync(lat.ctx)  # every step's diagnostics are in host memory
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    e2e_value = whole_job_mlups(world, N * e2e_steps, e2e_s)
    h2d = 5 * 4 * N / e2e_steps
    d2h = (5 * 4 * N + e2e_steps * 16 * 8) / e2e_steps
    mon = monitor.numpy()
    e2e_check = {"steps_reported": int((mon[:, 12] > 0).sum()),
                 "nonfinite_cells_max": float(mon[:, 5].max()),
                 "error_words": int((mon[:, 14] != 0).sum())}

    # --- roofline of the dominant kernel --------------------------------
    peak, peak_kind = measured_peaks()
    alg_bytes = 2 * 38 * BYTES_PER_VALUE[args.storage] * N  # read + write per launch
    # launch_ms brackets one lbm_step call: the fused kernel's launch, or both
    # launches of the two-pass form (charged together to the step's bytes)
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
    traffic = profiled_traffic(args.kernel, args.storage, n)

    variants = None
    if rank == 0 and world == 1 and args.storage == "f32" and not args.no_variants:
        variants = storage_variants(lbm, dev, pd, rR, rB, u, n, args)
    lat.close()
    batch = batch_measure(args, dev) if (rank == 0 and args.batch > 0) else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, _, _ = cpu_oracle_sample(args.cpu_n, args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic", "config": config_block(args, world),
                "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                        "check": e2e_check},
                "gpu_launches": args.steps * launches,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                             "unit": "GB/s", "frac": achieved / peak,
                             "traffic": traffic,
                             "peak_source": "%s hbm_gbs (MEASURED_PEAKS.json)" % peak_kind
                             if peak_kind == "measured" else "fallback 6.8 TB/s",
                             "algorithmic_bytes_per_cell": 2 * 38 * BYTES_PER_VALUE[args.storage],
                             "kernel_ms": launch_ms},
                "clocks": clocks,
                "storage_variants": variants,
                "batch": batch,
                "cpu_baseline": cpu,
                "check": {"nonfinite_cells": diag[5], "negative_density_cells": diag[6],
                          "mass_R": diag[0], "mass_B": diag[1]}}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def storage_variants(lbm, dev, pd, rR, rB, u, n, args):
    """FP16 / BF16 deviation storage and the FP32 in-place step (one
    population array) on the same workload: device-resident MLUPS (same
    timing as the FP32 line, fewer steps) and the error after
    `variant_steps` steps against the FP32 two-buffer run from the same
    initial state: relative L2 of the total density and of the velocity
    (velocity normalised by its FP32 L2 norm)."""
    import torch
    out = {}
    steps = args.variant_steps

    def run(storage, nsteps, timed):
        p = lbm.make_params(storage=storage, kernel=args.kernel, **pd)
        p.ref_R, p.ref_B = storage_references(storage, pd["rho_in_R"], pd["rho_in_B"], rR, rB)
        s = torch.cuda.Stream(dev)
        lat = lbm.Lattice(p, device=dev, stream=s)
        lat.init_fields(rR, rB, u)
        ms = None
        if timed:
            for _ in range(args.warmup):
                lbm.lbm_step(lat.ctx, 1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(timed):
                lbm.lbm_step(lat.ctx, 1)
            e1.record(s)
            s.synchronize()
            ms = e0.elapsed_time(e1) / timed
            lat.init_fields(rR, rB, u)
        lat.step(nsteps)
        mom = lat.moments()
        lat.close()
        return ms, mom

    _, ref = run("f32", steps, 0)
    rho_ref = (ref[0] + ref[1]).double()
    u_ref = ref[2].double()
    peak, _ = measured_peaks()
    for storage in ("f16", "bf16"):
        ms, got = run(storage, steps, max(args.steps // 4, 50))
        rho = (got[0] + got[1]).double()
        uu = got[2].double()
        mlups = n ** 3 / (ms * 1e-3) / 1e6
        out[storage] = {
            "value": mlups, "unit": "MLUPS", "ms_per_step": ms,
            "roofline_frac": mlups * 1e6 * 152 / (peak * 1e9),
            "algorithmic_bytes_per_cell": 152,
            "err_vs_f32_after_steps": steps,
            "rho_rel_l2": float((rho - rho_ref).norm() / rho_ref.norm()),
            "u_rel_l2": float((uu - u_ref).norm() / u_ref.norm()),
        }
    # the in-place step: one FP32 population array (AA access pattern), a
    # phase-field pass and the in-place collision per step
    p = lbm.make_params(storage="f32", kernel=args.kernel, **pd)
    s = torch.cuda.Stream(dev)
    ip = lbm.InPlaceLattice(p, device=dev, stream=s)
    ip.init_fields(rR, rB, u)
    timed = max(args.steps // 4, 50)
    ip.step(args.warmup)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(timed):
        ip.step(1)
    e1.record(s)
    s.synchronize()
    ms = e0.elapsed_time(e1) / timed
    ip.init_fields(rR, rB, u)
    ip.step(steps)
    got = ip.moments()
    rho = (got[0] + got[1]).double()
    uu = got[2].double()
    mlups = n ** 3 / (ms * 1e-3) / 1e6
    out["inplace_f32"] = {
        "value": mlups, "unit": "MLUPS", "ms_per_step": ms,
        "roofline_frac": mlups * 1e6 * 488 / (peak * 1e9),
        "algorithmic_bytes_per_cell": 488, "memory_bytes_per_cell": 168,
        "gpu_launches_per_step": 2,
        "err_vs_f32_after_steps": steps,
        "rho_rel_l2": float((rho - rho_ref).norm() / rho_ref.norm()),
        "u_rel_l2": float((uu - u_ref).norm() / u_ref.norm()),
    }
    del ip
    return out


def batch_measure(args, dev):
    """Batched sweep: `args.batch` independent droplet cases of uneven cubic
    sizes advanced together (one persistent launch per step, CUDA-graph
    replay).  MLUPS over all cases, FP32 and FP16 storage."""
    import numpy as np
    import torch

    from paper_1904_03618_gb300 import autotune, lbm, params as P, workloads
    samples = workloads.droplet_sweep(args.batch, seed=1234)
    cases = [P.droplet_case(s) for s in samples]
    cells = sum(c["nx"] ** 3 for c in cases)
    out = {"cases": len(cases), "cells": cells,
           "edges": sorted({c["nx"] for c in cases}),
           "workload": "droplet sweep: cubic boxes of edge 32/48/64/96, radius edge/4, "
                       "density ratio U[1,20], sigma U[0.001,0.02], speed U[0,0.05] "
                       "(half static), seed 1234"}
    peak, _ = measured_peaks()
    for storage in ("f32", "f16"):
        plist = []
        fields = []
        for c, s in zip(cases, samples):
            n = c["nx"]
            f = workloads.droplet(n, n, n, 0.25 * n, c["rho_in_R"], 1.0,
                                  velocity=(s["speed"], 0.0, 0.0))
            p = lbm.make_params(storage=storage, **c)
            p.ref_R, p.ref_B = storage_references(storage, c["rho_in_R"], 1.0, f[0], f[1])
            plist.append(p)
            fields.append(f)
        stream = torch.cuda.Stream(dev)
        b = lbm.Batch(plist, device=dev, stream=stream)
        for k, f in enumerate(fields):
            rR, rB, u = (np.ascontiguousarray(a, dtype=np.float32) for a in f)
            lbm.lbm_batch_init_fields(b.ctx, k, rR, rB, u)
        stream.synchronize()
        del fields
        tuned = autotune.tune(b.ctx, plist, stream, steps=6, cache_path=None)
        b.step(max(args.warmup, 4))
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(args.batch_steps)
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1) / args.batch_steps
        bad = sum(b.diagnostics(k, raise_unstable=False)[5] for k in range(0, len(cases), 64))
        b.close()
        mlups = cells / (ms * 1e-3) / 1e6
        bpc = 304 if storage == "f32" else 152
        out[storage] = {"value": mlups, "unit": "MLUPS", "ms_per_step": ms,
                        "roofline_frac": mlups * 1e6 * bpc / (peak * 1e9),
                        "steps": args.batch_steps, "gpu_launches_per_step": 1,
                        "autotuned_config": {"tile_y": tuned[0], "zchunk": tuned[1],
                                             "hold": tuned[2]},
                        "nonfinite_cells_sampled": bad}
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--kernel", default="fused", choices=["fused", "two_pass"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--fused-config", default="",
                    help="tile_y,zchunk,hold of the fused kernel (default: library choice)")
    ap.add_argument("--cpu-n", type=int, default=48)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--variant-steps", type=int, default=200)
    ap.add_argument("--batch", type=int, default=512,
                    help="number of cases of the batched droplet sweep (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=30)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
