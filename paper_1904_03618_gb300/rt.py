"""Three-dimensional Rayleigh-Taylor instability (Sec. IV.C): the heavy red
fluid above the light blue one in [0, L]^2 x [0, 4L], walls at the top and
bottom, periodic sides, the single-mode perturbation of Eq. 56, Atwood
number (rho_R - rho_B) / (rho_R + rho_B) = 0.5, equal kinematic viscosities,
Re = L sqrt(L g) / nu.  The run records the interface positions the paper
plots (its Fig. 7): the spike tip (column x = y = L/2, where Eq. 56 puts the
lowest interface), the bubble front (column x = y = 0, the highest) and the
saddle point (x = 0, y = L/2), each as the height where rho^N crosses zero
along the column, in units of L from the initial mean interface, against
t* = t / sqrt(L / g).

`python -m paper_1904_03618_gb300.rt --storage f32 f16 bf16` runs the same
case in each storage format and reports the positions and the differences
of the 16-bit runs from FP32; `--storage inplace` runs it on one population
array stepped in place, which takes L = 512 (512 x 512 x 2048, 537 M cells,
90 GB) on one GPU.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import lbm
from . import params as P
from . import workloads as wl


def rt_params(L=256, g=1e-5, Re=256.0, A=1e-3, beta=0.7, alpha_B=0.7):
    """lbm_params keywords of the case (red heavy, rho 3 : 1)."""
    nu = L * math.sqrt(L * g) / Re
    aR = P.alpha_R_from_balance(3.0, 1.0, alpha_B)
    return dict(nx=L, ny=L, nz=4 * L, wall=(0, 0, 1), improved=True, rho_in_R=3.0,
                rho_in_B=1.0, alpha_R=aR, alpha_B=alpha_B, tau_R=P.tau_from_nu(nu, aR),
                tau_B=P.tau_from_nu(nu, alpha_B), A_R=A, A_B=A, beta=beta, delta=0.98,
                gravity=(0.0, 0.0, -g))


def _crossing(col, from_top):
    """Height where the column's rho^N crosses zero: scanning up from the
    bottom for the first heavy cell (spike, saddle) or down from the top for
    the first light cell (bubble); linear interpolation between the two cells
    that straddle the sign change."""
    c = col.double().cpu().numpy()
    n = len(c)
    if from_top:
        for z in range(n - 1, 0, -1):
            if c[z - 1] < 0.0 <= c[z]:
                return z - 1 + c[z - 1] / (c[z - 1] - c[z])
        return float("nan")
    for z in range(1, n):
        if c[z - 1] < 0.0 <= c[z]:
            return z - 1 + c[z - 1] / (c[z - 1] - c[z])
    return float("nan")


def positions(lat, pd):
    """(spike, bubble, saddle) heights in lattice units."""
    rR, rB, _ = lat.moments()
    L = pd["nx"]
    r, b = rR / pd["rho_in_R"], rB / pd["rho_in_B"]
    rn = (r - b) / (r + b)
    spike = _crossing(rn[:, L // 2, L // 2], from_top=False)
    bubble = _crossing(rn[:, 0, 0], from_top=True)
    saddle = _crossing(rn[:, L // 2, 0], from_top=False)
    return spike, bubble, saddle


def run(storage="f32", L=256, steps=10000, every=500, g=1e-5, device=None, log=None):
    """storage: "f32", "f16", "bf16" (the two-buffer context) or "inplace"
    (FP32, one population array stepped in place: 168 bytes per cell, no
    cell-count limit beyond device memory)."""
    dev = torch.device(device or "cuda")
    pd = rt_params(L=L, g=g)
    inplace = storage == "inplace"
    rR, rB, u = wl.rayleigh_taylor(L, L, 4 * L, L, 0.05, 2 * L, pd["rho_in_R"], pd["rho_in_B"],
                                   dtype=np.float32)
    p = lbm.make_params(storage="f32" if inplace else storage, **pd)
    if storage not in ("f32", "inplace"):
        # each colour is the majority phase of half the box: both store their
        # deviation from their own pure rest state (absolute 16-bit values,
        # references 0, lose the per-step gravity increments and create red
        # mass: +21 % in 4000 steps at L = 64)
        p.ref_R, p.ref_B = pd["rho_in_R"], pd["rho_in_B"]
    stream = torch.cuda.Stream(dev)
    lat = (lbm.InPlaceLattice if inplace else lbm.Lattice)(p, device=dev, stream=stream)
    t_ref = math.sqrt(L / g)
    z0 = 2.0 * L
    rows = []
    seconds = 0.0
    try:
        lat.init_fields(rR, rB, u)
        del rR, rB, u
        done = 0
        while True:
            s, b, d = positions(lat, pd)
            rows.append({"step": done, "t_star": done / t_ref, "spike": (s - z0) / L,
                         "bubble": (b - z0) / L, "saddle": (d - z0) / L})
            if log:
                log("%s step %d: spike %.4f bubble %.4f saddle %.4f" %
                    (storage, done, rows[-1]["spike"], rows[-1]["bubble"], rows[-1]["saddle"]))
            if done >= steps:
                break
            n = min(every, steps - done)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            lat.step(n)
            stream.synchronize()
            seconds += time.perf_counter() - t0
            done += n
        if inplace:
            mR, mB, _ = lat.moments()
            diag = (float(mR.double().sum()), float(mB.double().sum()), 0, 0, 0,
                    int((~torch.isfinite(mR + mB)).sum()))
            del mR, mB
        else:
            diag = lat.diagnostics(raise_unstable=False)
    finally:
        lat.close()
    cells = L * L * 4 * L
    return {"storage": storage, "rows": rows, "mlups": cells * steps / seconds / 1e6,
            "mass_R": diag[0], "mass_B": diag[1], "nonfinite": diag[5]}


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="3-D Rayleigh-Taylor instability, interface "
                                             "positions per storage format")
    ap.add_argument("--L", type=int, default=256)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--every", type=int, default=500)
    ap.add_argument("--storage", nargs="+", default=["f32", "f16", "bf16"])
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    res = {}
    for s in args.storage:
        res[s] = run(s, L=args.L, steps=args.steps, every=args.every,
                     log=lambda m: print(m, flush=True))
        torch.cuda.empty_cache()
    if "f32" in res:
        ref = res["f32"]["rows"]
        for s, r in res.items():
            if s == "f32":
                continue
            r["max_abs_diff_vs_f32"] = {
                k: float(np.nanmax([abs(a[k] - b[k]) for a, b in zip(r["rows"], ref)]))
                for k in ("spike", "bubble", "saddle")}
    print(json.dumps({s: {k: v for k, v in r.items() if k != "rows"} for s, r in res.items()}))
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
