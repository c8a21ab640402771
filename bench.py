"""Throughput benchmark of the two-fluid D3Q19 colour-gradient step.

One bench "step" is one lattice time step (all of: pull streaming, moments,
gradients, collision, perturbation, recolouring, store) over the whole
lattice.  Headline workload (default): the three-dimensional Rayleigh-Taylor
instability of Sec. IV.C on 256 x 256 x 1024 cells, periodic in x and y,
halfway bounce-back walls in z, heavy red fluid (3) over light blue fluid (1)
(Atwood number 0.5), gravity 1e-5, Re = 256, single-mode cosine interface of
amplitude 0.05 L (Eq. 56), FP32 storage and arithmetic.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload rt|droplet] [--storage f32|f16|bf16]
                  [--kernel fused|two_pass] [--L 256] [--n 128] [--gemm]

Prints one JSON line.  `value` is whole-job MLUPS with the populations
resident in HBM (20 GB of FP32 populations, far larger than the 129 MB L2,
so no flush is needed between steps); `e2e` is the same metric through the
C ABI with host buffers (initial fields uploaded from pinned host memory,
every step's diagnostics -- summed inside the step kernel by
lbm_step_monitored -- copied back into pinned host memory in stream order,
final moments downloaded, all inside the timed region; the field transfers
are paid once per e2e run, so e2e grows with the number of steps).  Extra keys: `droplet_128` (the 128^3
moving droplet in FP32, FP16, BF16 and the in-place step), `storage_variants`
(the headline workload in FP16 and BF16), `batch` (512 independent droplet
cases in one launch per step), `oracle_error` (FP32 / FP16 / BF16 runs
against the FP64 oracle on the CPU-baseline sample).  Multi-GPU runs are
independent replicas (one lattice per rank, weak scaling); `--slabs` cuts
one lattice into z-slabs over the ranks instead (NCCL halo exchange after
every step, strong scaling), or with `--emulate-slabs S` into S slabs on
one GPU.
"""
from __future__ import annotations

import argparse
import json
import math
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
# algorithmic bytes of one cell update: 38 populations read + 38 written
ALG_BYTES = {"f32": 304, "f16": 152, "bf16": 152}


# ---------------------------------------------------------------------------
# Workloads
def droplet_params(n):
    """Moving droplet in uniform flow (density ratio 10, sigma = 0.005)."""
    return dict(nx=n, ny=n, nz=n, wall=(0, 0, 0), improved=True,
                rho_in_R=10.0, rho_in_B=1.0, alpha_R=0.97, alpha_B=0.7,
                tau_R=1.0, tau_B=1.0, tau_e=1.0, tau_q=1.0, tau_pi=1.0,
                A_R=0.01125, A_B=0.01125, beta=0.7, delta=0.98,
                force=(0.0, 0.0, 0.0), gravity=(0.0, 0.0, 0.0))


def droplet_fields(n):
    from paper_1904_03618_gb300 import workloads
    return workloads.droplet(n, n, n, 20.0 * n / 128.0, 10.0, 1.0,
                             velocity=(0.05, 0.0, 0.0))


def rt_params(L):
    from paper_1904_03618_gb300 import rt
    return rt.rt_params(L=L)


def rt_fields(L, dtype=None):
    import numpy as np

    from paper_1904_03618_gb300 import workloads
    return workloads.rayleigh_taylor(L, L, 4 * L, L, 0.05, 2 * L, 3.0, 1.0,
                                     dtype=dtype or np.float64)


def workload(kind, size):
    """(lbm params dict, fields function of the size, description)."""
    if kind == "rt":
        pd = rt_params(size)
        desc = ("Rayleigh-Taylor instability, %dx%dx%d D3Q19 two-fluid, periodic x/y, "
                "bounce-back walls in z, density 3/1 (Atwood 0.5), gravity 1e-5, Re 256, "
                "Eq. 56 single-mode perturbation amplitude 0.05 L, A_R = A_B = 1e-3, "
                "beta 0.7" % (size, size, 4 * size))
        return pd, rt_fields, desc
    pd = droplet_params(size)
    desc = ("moving droplet in uniform flow, %d^3 periodic D3Q19 two-fluid, R=%g, "
            "u=(0.05,0,0), density ratio 10, viscosity ratio 1, sigma=0.005, beta=0.7"
            % (size, 20.0 * size / 128.0))
    return pd, droplet_fields, desc


def storage_references(storage, pd, rho_R, rho_B, both=False):
    """Deviation references for FP16/BF16 storage.  Droplets: the colour
    with more mass (the background phase) is stored as f - rho_in phi, the
    other as is, so that the absent colour stays exactly zero.  Rayleigh-
    Taylor (`both`): each colour fills half the box, so both store their
    deviation from their own pure rest state."""
    if storage == "f32":
        return 0.0, 0.0
    if both:
        return pd["rho_in_R"], pd["rho_in_B"]
    return ((pd["rho_in_R"], 0.0) if rho_R.sum() >= rho_B.sum()
            else (0.0, pd["rho_in_B"]))


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


def kernel_source_hash():
    """The step kernels' sources and the launch rules that pick their tile
    and z chunk (the DRAM bytes per cell depend on both)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("lbm_fused.cuh", "lbm_fused_tma.cuh", "lbm_device.cuh", "lbm_dispatch.cu"):
        h.update(open(os.path.join(ROOT, "paper_1904_03618_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(key, cells):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel (source hash recorded beside it)."""
    path = os.path.join(ROOT, "profiles", "fused_step_traffic.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha256") != kernel_source_hash() or key + "_bytes_per_cell" not in vals:
        return None
    return float(vals[key + "_bytes_per_cell"]) * cells


# ---------------------------------------------------------------------------
# CPU oracle legs (the only parts of the benchmark that run oracle/)
def cpu_oracle_sample(args):
    """Time the FP64 oracle, as it stands, on the host cores on a bounded
    sample of the headline workload: the same case on a smaller lattice
    (Rayleigh-Taylor L = args.cpu_L: L x L x 4L cells, same gravity and
    Reynolds number), as many steps as fit in about args.cpu_seconds.
    Returns the baseline record and the oracle's final state."""
    import oracle
    size = args.cpu_L if args.workload == "rt" else args.cpu_n
    pd, fields, _ = workload(args.workload, size)
    p = oracle.params_from(pd)
    rR, rB, u = fields(size)
    f = oracle.init(p, rR, rB, u)
    cells = pd["nx"] * pd["ny"] * pd["nz"]
    t0 = time.perf_counter()
    f = oracle.step(p, f, 2)
    one = (time.perf_counter() - t0) / 2
    steps = max(2, int(args.cpu_seconds / max(one, 1e-6)))
    f0 = oracle.init(p, rR, rB, u)
    t0 = time.perf_counter()
    f = oracle.step(p, f0, steps)
    dt = time.perf_counter() - t0
    rec = {"value": cells * steps / dt / 1e6, "unit": "MLUPS",
           "cores": oracle.num_threads(), "kind": "oracle",
           "sample": "%dx%dx%d lattice of the same case, %d steps, %.1f s" % (
               pd["nx"], pd["ny"], pd["nz"], steps, dt)}
    mR, mB, mu = oracle.moments(p, f)
    return rec, (pd, size, steps, mR, mB, mu)


def oracle_error(lbm, dev, sample, args):
    """FP32 / FP16 / BF16 runs of the CPU-baseline sample on the GPU, from
    the same initial fields and for the same number of steps as the oracle:
    relative L2 of the total density and of the velocity against the FP64
    oracle, and each colour's relative mass change."""
    import numpy as np
    import torch
    pd, size, steps, mR, mB, mu = sample
    _, fields, _ = workload(args.workload, size)
    rR, rB, u = (np.ascontiguousarray(a, dtype=np.float32) for a in fields(size))
    rho_o = mR + mB
    out = {"steps": steps, "lattice": [pd["nx"], pd["ny"], pd["nz"]]}
    for storage in ("f32", "f16", "bf16"):
        p = lbm.make_params(storage=storage, **pd)
        p.ref_R, p.ref_B = storage_references(storage, pd, rR, rB,
                                              both=args.workload == "rt")
        s = torch.cuda.Stream(dev)
        lat = lbm.Lattice(p, device=dev, stream=s)
        lat.init_fields(rR, rB, u)
        lat.step(steps)
        gR, gB, gu = (t.double().cpu().numpy() for t in lat.moments())
        lat.close()
        rho = gR + gB
        un = max(float(np.linalg.norm(mu)), 1e-3 * math.sqrt(mu.size))
        out[storage] = {
            "rho_rel_l2": float(np.linalg.norm(rho - rho_o) / np.linalg.norm(rho_o)),
            "u_rel_l2": float(np.linalg.norm(gu - mu) / un),
            "mass_R_rel_change": float(gR.sum() / rR.astype(np.float64).sum() - 1.0),
            "mass_B_rel_change": float(gB.sum() / rB.astype(np.float64).sum() - 1.0),
            "oracle_mass_R_rel_change": float(mR.sum() / rR.astype(np.float64).sum() - 1.0),
        }
    return out


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle, as it stands, on the host cores.  Each
    bench step is one oracle time step on a lattice of the same case whose
    size is chosen so that warm-up plus timed steps take about two minutes."""
    if rank != 0:
        return
    import oracle
    probe = 8 if args.workload == "rt" else 24
    pd, fields, _ = workload(args.workload, probe)
    pp = oracle.params_from(pd)
    fp = oracle.init(pp, *fields(probe))
    t0 = time.perf_counter()
    oracle.step(pp, fp, 2)
    cells_probe = pd["nx"] * pd["ny"] * pd["nz"]
    rate = 2 * cells_probe / (time.perf_counter() - t0)
    budget = 120.0 / (args.steps + args.warmup)
    full = args.L if args.workload == "rt" else args.n
    shape_cells = 4.0 if args.workload == "rt" else 1.0  # cells = shape * size^3
    size = int(max(8, min(full, (rate * budget / shape_cells) ** (1.0 / 3.0))))
    if args.workload == "rt":
        size -= size % 2
    pd, fields, _ = workload(args.workload, size)
    p = oracle.params_from(pd)
    f = oracle.init(p, *fields(size))
    cells = pd["nx"] * pd["ny"] * pd["nz"]
    for _ in range(args.warmup):
        f = oracle.step(p, f, 1)
    per_step = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        f = oracle.step(p, f, 1)
        per_step.append(time.perf_counter() - t0)
    mean = statistics.mean(per_step)
    mlups = cells / mean / 1e6
    cb = {"value": mlups, "unit": "MLUPS", "cores": oracle.num_threads(),
          "kind": "oracle",
          "sample": "each step: one FP64 oracle step on a %dx%dx%d lattice of the same "
                    "case (%d steps timed)" % (pd["nx"], pd["ny"], pd["nz"], args.steps)}
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * mean, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_block(args, world), "cpu_baseline": cb,
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_block(args, world):
    size = args.L if args.workload == "rt" else args.n
    pd, _, desc = workload(args.workload, size)
    cells = pd["nx"] * pd["ny"] * pd["nz"]
    return {"workload": desc,
            "lattice": [pd["nx"], pd["ny"], pd["nz"]], "storage": args.storage,
            "kernel": args.kernel, "fused_config": args.fused_config or "library default",
            "model": "improved (Eq. 18 + Eq. 45 correction)",
            "parallelism": "replicas x%d" % world if world > 1 else "single GPU",
            "l2_policy": "inputs larger than L2 (%.0f MB populations per buffer)" % (
                cells * 38 * BYTES_PER_VALUE[args.storage] / 1e6)}


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
def time_steps(lbm, torch, ctx, stream, steps, warmup):
    """(mean per-launch ms, total ms) of `steps` single-step calls on the
    context's stream, CUDA events on that stream."""
    for _ in range(warmup):
        lbm.lbm_step(ctx, 1)
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(steps):
        ev[k][0].record(stream)
        lbm.lbm_step(ctx, 1)
        ev[k][1].record(stream)
    t1.record(stream)
    stream.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in ev), t0.elapsed_time(t1)


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

    size = args.L if args.workload == "rt" else args.n
    pd, fields, _ = workload(args.workload, size)
    N = pd["nx"] * pd["ny"] * pd["nz"]
    rR, rB, u = (np.ascontiguousarray(a, dtype=np.float32) for a in fields(size))
    params = lbm.make_params(storage=args.storage, kernel=args.kernel, **pd)
    params.ref_R, params.ref_B = storage_references(args.storage, pd, rR, rB,
                                                    both=args.workload == "rt")
    stream = torch.cuda.Stream(dev)
    lat = lbm.Lattice(params, device=dev, stream=stream)
    if args.kernel == "fused" and args.fused_config:
        ty, zc, hold = (int(v) for v in args.fused_config.split(","))
        lbm.lbm_set_fused_config(lat.ctx, ty, zc, hold)
    lat.init_fields(rR, rB, u)
    launches = lbm.lbm_launches_per_step(lat.ctx)
    fused_cfg = lbm.lbm_get_fused_config(lat.ctx) if args.kernel == "fused" else None

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
    e2e_steps = max(args.steps, 20)
    monitor = torch.zeros((e2e_steps, 16), dtype=torch.float64).pin_memory()
    # warm the staging buffers, the monitor record and the monitored
    # kernel (its first launch loads it)
    lbm.lbm_init_fields(lat.ctx, hR, hB, hu)
    lbm.lbm_step_monitored(lat.ctx, 1, monitor[0])
    lbm.lbm_moments(lat.ctx, oR, oB, ou)
    lbm.lbm_sync(lat.ctx)
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    lbm.lbm_init_fields(lat.ctx, hR, hB, hu)
    for k in range(e2e_steps):
        # one step, the diagnostics of the state it reads (summed inside the
        # step kernel) and their copy into pinned host memory, queued
        # without a host wait
        lbm.lbm_step_monitored(lat.ctx, 1, monitor[k])
    lbm.lbm_moments(lat.ctx, oR, oB, ou)
    lbm.lbm_sync(lat.ctx)  # every step's diagnostics are in host memory
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    e2e_value = whole_job_mlups(world, N * e2e_steps, e2e_s)
    h2d = 5 * 4 * N / e2e_steps
    d2h = (5 * 4 * N + e2e_steps * 16 * 8) / e2e_steps
    mon = monitor.numpy()
    e2e_check = {"steps_reported": int((mon[:, 12] == np.arange(e2e_steps)).sum()),
                 "nonfinite_cells_max": float(mon[:, 5].max()),
                 "error_words": int((mon[:, 14] != 0).sum())}
    del hR, hB, hu, oR, oB, ou

    # --- roofline of the dominant kernel --------------------------------
    peak, peak_kind = measured_peaks()
    alg_bytes = ALG_BYTES[args.storage] * N  # read + write per launch
    # launch_ms brackets one lbm_step call: the fused kernel's launch, or both
    # launches of the two-pass form (charged together to the step's bytes)
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
    traffic = profiled_traffic("%s_%s_%s" % (args.workload, args.kernel, args.storage), N)
    lat.close()
    del lat
    torch.cuda.empty_cache()

    extras = {}
    if rank == 0 and world == 1 and not args.no_variants:
        if args.workload == "rt" and args.storage == "f32":
            extras["storage_variants"] = storage_variants_rt(lbm, dev, pd, rR, rB, u, args)
        del rR, rB, u
        torch.cuda.empty_cache()
        extras["droplet_128"] = droplet_variants(lbm, dev, args)
        torch.cuda.empty_cache()
    if rank == 0 and args.batch > 0:
        extras["batch"] = batch_measure(args, dev)
    if rank == 0 and args.gemm:
        extras["gemm"] = gemm_measure(lbm, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, sample = cpu_oracle_sample(args)
        extras["oracle_error"] = oracle_error(lbm, dev, sample, args)

    if rank == 0:
        cfg = config_block(args, world)
        if fused_cfg is not None:
            cfg["fused_config_used"] = {"tile_y": fused_cfg[0], "zchunk": fused_cfg[1],
                                        "hold": fused_cfg[2]}
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": args.storage, "data": "synthetic", "config": cfg,
                "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                        "check": e2e_check},
                "gpu_launches": args.steps * launches,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                             "unit": "GB/s", "frac": achieved / peak,
                             "traffic": traffic,
                             "peak_source": "%s hbm_gbs (MEASURED_PEAKS.json)" % peak_kind
                             if peak_kind == "measured" else "fallback 6.8 TB/s",
                             "algorithmic_bytes_per_cell": ALG_BYTES[args.storage],
                             "kernel_ms": launch_ms},
                "clocks": clocks,
                "cpu_baseline": cpu,
                "check": {"nonfinite_cells": diag[5], "negative_density_cells": diag[6],
                          "mass_R": diag[0], "mass_B": diag[1]}}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _drift(got, ref):
    rho = (got[0] + got[1]).double()
    rho_ref = (ref[0] + ref[1]).double()
    uu, u_ref = got[2].double(), ref[2].double()
    return {"rho_rel_l2": float((rho - rho_ref).norm() / rho_ref.norm()),
            "u_rel_l2": float((uu - u_ref).norm() / u_ref.norm())}


def _run_lattice(lbm, dev, p, fields, nsteps, timed, warmup):
    """(mean ms per step over `timed` steps or None, moments after `nsteps`
    steps from the initial fields)."""
    import torch
    s = torch.cuda.Stream(dev)
    lat = lbm.Lattice(p, device=dev, stream=s)
    lat.init_fields(*fields)
    ms = None
    if timed:
        ms, _ = time_steps(lbm, torch, lat.ctx, s, timed, warmup)
        lat.init_fields(*fields)
    lat.step(nsteps)
    mom = lat.moments()
    lat.close()
    return ms, mom


def storage_variants_rt(lbm, dev, pd, rR, rB, u, args):
    """The headline workload with FP16 / BF16 deviation storage: MLUPS
    (CUDA events, per launch) and the drift of the density and velocity
    against the FP32 run after `variant_steps` steps from the same state."""
    peak, _ = measured_peaks()
    N = pd["nx"] * pd["ny"] * pd["nz"]
    steps = args.variant_steps
    p = lbm.make_params(storage="f32", kernel=args.kernel, **pd)
    _, ref = _run_lattice(lbm, dev, p, (rR, rB, u), steps, 0, args.warmup)
    out = {}
    for storage in ("f16", "bf16"):
        p = lbm.make_params(storage=storage, kernel=args.kernel, **pd)
        p.ref_R, p.ref_B = storage_references(storage, pd, rR, rB, both=True)
        ms, got = _run_lattice(lbm, dev, p, (rR, rB, u), steps, max(args.steps, 20),
                               args.warmup)
        mlups = N / (ms * 1e-3) / 1e6
        out[storage] = {"value": mlups, "unit": "MLUPS", "kernel_ms": ms,
                        "roofline_frac": mlups * 1e6 * ALG_BYTES[storage] / (peak * 1e9),
                        "algorithmic_bytes_per_cell": ALG_BYTES[storage],
                        "err_vs_f32_after_steps": steps, **_drift(got, ref)}
        del got
    return out


def droplet_variants(lbm, dev, args):
    """The 128^3 moving droplet (density ratio 10): FP32, FP16 and BF16
    deviation storage and the FP32 and FP16 in-place step (one population
    array),
    device-resident MLUPS and the fraction of the HBM roofline at the
    algorithmic 304 / 152 bytes per cell update; 16-bit and in-place drift
    against the FP32 run after `variant_steps` steps."""
    import numpy as np
    import torch
    n = args.n
    pd = droplet_params(n)
    rR, rB, u = (np.ascontiguousarray(a, dtype=np.float32) for a in droplet_fields(n))
    peak, _ = measured_peaks()
    N = n ** 3
    steps = args.variant_steps
    timed = max(args.steps * 5, 100)
    out = {"workload": workload("droplet", n)[2]}
    ref = None
    for storage in ("f32", "f16", "bf16"):
        p = lbm.make_params(storage=storage, kernel=args.kernel, **pd)
        p.ref_R, p.ref_B = storage_references(storage, pd, rR, rB)
        ms, got = _run_lattice(lbm, dev, p, (rR, rB, u), steps, timed, args.warmup)
        mlups = N / (ms * 1e-3) / 1e6
        rec = {"value": mlups, "unit": "MLUPS", "kernel_ms": ms,
               "roofline_frac": mlups * 1e6 * ALG_BYTES[storage] / (peak * 1e9),
               "algorithmic_bytes_per_cell": ALG_BYTES[storage]}
        if storage == "f32":
            ref = got
            rec["traffic"] = profiled_traffic("droplet_fused_f32", N)
        else:
            rec.update(err_vs_f32_after_steps=steps, **_drift(got, ref))
        out[storage] = rec
    # the in-place step: one population array (AA access pattern), FP32 and
    # FP16 deviation storage, a phase-field pass and the in-place collision
    # per step; its fraction is taken at the method's 304 / 152 B/cell, not
    # at the 488 / 260 B/cell the two passes move
    for storage in ("f32", "f16"):
        p = lbm.make_params(storage=storage, kernel=args.kernel, **pd)
        p.ref_R, p.ref_B = storage_references(storage, pd, rR, rB)
        s = torch.cuda.Stream(dev)
        ip = lbm.InPlaceLattice(p, device=dev, stream=s)
        ip.init_fields(rR, rB, u)
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
        ip.close()
        mlups = N / (ms * 1e-3) / 1e6
        vb = ALG_BYTES[storage] // 2  # bytes of one cell's 38 values
        out["inplace_" + storage] = {
            "value": mlups, "unit": "MLUPS", "ms_per_step": ms,
            "roofline_frac": mlups * 1e6 * ALG_BYTES[storage] / (peak * 1e9),
            "algorithmic_bytes_per_cell": ALG_BYTES[storage],
            "moved_bytes_per_cell": 3 * vb + 32, "memory_bytes_per_cell": vb + 16,
            "gpu_launches_per_step": 2, "err_vs_f32_after_steps": steps, **_drift(got, ref)}
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
            p.ref_R, p.ref_B = storage_references(storage, c, f[0], f[1])
            plist.append(p)
            fields.append(f)
        stream = torch.cuda.Stream(dev)
        b = lbm.Batch(plist, device=dev, stream=stream)
        for k, f in enumerate(fields):
            rR, rB, u = (np.ascontiguousarray(a, dtype=np.float32) for a in f)
            lbm.lbm_batch_init_fields(b.ctx, k, rR, rB, u)
        stream.synchronize()
        del fields
        if args.batch_tune:
            tuned = autotune.tune(b.ctx, plist, stream, steps=6, cache_path=None)
        else:
            tuned = lbm.lbm_get_fused_config(b.ctx)
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
        out[storage] = {"value": mlups, "unit": "MLUPS", "ms_per_step": ms,
                        "roofline_frac": mlups * 1e6 * ALG_BYTES[storage] / (peak * 1e9),
                        "steps": args.batch_steps, "gpu_launches_per_step": 1,
                        "autotuned_config": {"tile_y": tuned[0], "zchunk": tuned[1],
                                             "hold": tuned[2]},
                        "nonfinite_cells_sampled": bad}
        torch.cuda.empty_cache()
    return out


def gemm_measure(lbm, dev):
    """The surrogate network's tensor-core GEMM (lbm_gemm_bf16) on the
    shapes of its use: forward H W (65,536 x 256 x 256), the input layer
    (65,536 x 256 x 5), the backward dZ W^T, the weight gradient H^T dZ
    (256 x 256 x 65,536), and one layer of a batch-256 training step (256 x
    256 x 256); time by CUDA events over 20 launches, against cuBLAS on the
    same BF16-rounded operands (torch.matmul) for context.  The FP32
    operands are read once and C written once, 4 (MK + KN + MN) bytes: at
    these shapes the product is bound by HBM (about 86 flop per byte against
    a ridge near 280), so the line reports both fractions."""
    import torch
    torch.manual_seed(0)
    peak = hbm = None
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        mp = json.load(open(path))
        peak = float(mp["bf16_tflops"])
        hbm = float(mp["hbm_gbs"])
    shapes = [("forward H W", 65536, 256, 256, False, False),
              ("input layer X W", 65536, 256, 5, False, False),
              ("backward dZ W^T", 65536, 256, 256, False, True),
              ("weight gradient H^T dZ", 256, 256, 65536, True, False),
              ("training layer, batch 256", 256, 256, 256, False, False)]
    out = {"peak_tflops": peak, "hbm_gbs": hbm}
    err = torch.zeros(4, dtype=torch.int32, device=dev)
    s = torch.cuda.Stream(dev)
    for name, M, N, K, trans_a, trans_b in shapes:
        if trans_a:  # A stored K x M: A(m, k) = A[k * M + m]
            A = torch.randn(K, M, device=dev)
            sa_m, sa_k = 1, M
        else:
            A = torch.randn(M, K, device=dev)
            sa_m, sa_k = K, 1
        if trans_b:  # B stored N x K: B(k, n) = B[n * K + k]
            B = torch.randn(N, K, device=dev)
            sb_k, sb_n = 1, K
        else:
            B = torch.randn(K, N, device=dev)
            sb_k, sb_n = N, 1
        C = torch.empty(M, N, device=dev)
        torch.cuda.synchronize(dev)

        def gemm():
            lbm.lbm_gemm_bf16(A, sa_m, sa_k, B, sb_k, sb_n, C, N, M, N, K, err,
                              s.cuda_stream)
        for _ in range(3):
            gemm()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(20):
            gemm()
        e1.record(s)
        s.synchronize()
        ms = e0.elapsed_time(e1) / 20
        Ab = (A.t() if trans_a else A).to(torch.bfloat16).contiguous()
        Bb = (B.t() if trans_b else B).to(torch.bfloat16).contiguous()
        with torch.cuda.stream(s):
            for _ in range(3):
                torch.matmul(Ab, Bb)
            e0.record(s)
            for _ in range(20):
                torch.matmul(Ab, Bb)
            e1.record(s)
        s.synchronize()
        ms_cublas = e0.elapsed_time(e1) / 20
        flops = 2.0 * M * N * K
        nbytes = 4.0 * (M * K + K * N + M * N)
        out[name] = {"M": M, "N": N, "K": K, "ms": ms, "tflops": flops / ms / 1e9,
                     "cublas_bf16_tflops": flops / ms_cublas / 1e9,
                     "frac_of_peak": (flops / ms / 1e9 / peak) if peak else None,
                     "operand_gbs": nbytes / ms / 1e6,
                     "frac_of_hbm": (nbytes / ms / 1e6 / hbm) if hbm else None}
    out["error_word"] = int(err.max().item())
    return out


def run_slabs(args, rank, world, local_rank):
    """One lattice cut into z-slabs, one per rank (NCCL halo exchange after
    every step, paper_1904_03618_gb300/slabs.py), or --emulate-slabs S slabs
    on one GPU in one process (device copies).  value = cells of the whole
    lattice per second over the slowest rank (strong scaling)."""
    import numpy as np
    import torch

    from paper_1904_03618_gb300 import lbm, slabs
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    size = args.L if args.workload == "rt" else args.n
    pd, fields_fn, desc = workload(args.workload, size)
    N = pd["nx"] * pd["ny"] * pd["nz"]
    fields = tuple(np.ascontiguousarray(a, dtype=np.float32) for a in fields_fn(size))
    refs = storage_references(args.storage, pd, fields[0], fields[1],
                              both=args.workload == "rt")
    if world > 1:
        plan = slabs.SlabPlan(pd["nz"], world, rank, bool(pd["wall"][2]))
        obj = slabs.SlabLattice(pd, plan, dist, dev, args.storage, refs)
        obj.init_fields(fields)
        nslabs = world
        ctxs = [obj.lat.ctx]
    else:
        nslabs = max(1, args.emulate_slabs)
        obj = slabs.SlabsOnOneDevice(pd, nslabs, device=dev, storage=args.storage, refs=refs)
        obj.init_fields(fields)
        ctxs = [lat.ctx for lat in obj.lats]
    del fields
    stream = torch.cuda.current_stream(dev)
    obj.step(args.warmup)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    obj.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    # the step kernels alone (no exchange), for the roofline of this rank
    k_ms, _ = time_steps(lbm, torch, ctxs[0], stream, args.steps, 1)
    plan0 = obj.plan if world > 1 else obj.plans[0]
    local_cells = pd["nx"] * pd["ny"] * plan0.nz_local
    peak, peak_kind = measured_peaks()
    achieved = ALG_BYTES[args.storage] * local_cells / (k_ms * 1e-3) / 1e9
    if rank == 0:
        line = {"metric": METRIC, "value": N / (ms * 1e-3) / 1e6, "unit": "MLUPS",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
                "config": dict(config_block(args, world),
                               parallelism="z-slabs x%d (%s)" % (
                                   nslabs, "NCCL point-to-point halo exchange" if world > 1
                                   else "one device, device-copy halo exchange")),
                "e2e": None,
                "gpu_launches": args.steps * nslabs,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                             "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                             "peak_source": "%s hbm_gbs" % peak_kind,
                             "algorithmic_bytes_per_cell": ALG_BYTES[args.storage],
                             "kernel_ms": k_ms, "kernel": "step of slab 0 (own planes "
                             "plus ghosts), exchange excluded"},
                "cpu_baseline": None}
        print(json.dumps(line), flush=True)
    obj.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rt", choices=["rt", "droplet"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--kernel", default="fused", choices=["fused", "two_pass"])
    ap.add_argument("--L", type=int, default=256, help="Rayleigh-Taylor edge (L x L x 4L)")
    ap.add_argument("--n", type=int, default=128, help="droplet cube edge")
    ap.add_argument("--fused-config", default="",
                    help="tile_y,zchunk,hold of the fused kernel (default: library choice)")
    ap.add_argument("--cpu-L", type=int, default=32,
                    help="Rayleigh-Taylor edge of the CPU-baseline sample")
    ap.add_argument("--cpu-n", type=int, default=48, help="droplet edge of the CPU sample")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--variant-steps", type=int, default=200)
    ap.add_argument("--batch", type=int, default=512,
                    help="number of cases of the batched droplet sweep (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--no-batch-tune", dest="batch_tune", action="store_false",
                    help="run the batch in the library's default configuration")
    ap.add_argument("--gemm", action="store_true",
                    help="also time the surrogate's tensor-core GEMM")
    ap.add_argument("--slabs", action="store_true",
                    help="one lattice cut into z-slabs over the ranks (strong scaling)")
    ap.add_argument("--emulate-slabs", type=int, default=1,
                    help="with --slabs on one GPU: that many slabs in one process")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.slabs:
        run_slabs(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
