"""Moving droplet between moving plates (Sec. IV.A), the paper's own test of
Galilean invariance: a 140 x 140 x 4 lattice, periodic in x and z, the two
plates of the y axis moving with U = 0.02 along x from t = 0 (Zou-He
velocity nodes), a circular drop of radius 30 (a red column along z) at the
centre, brought to equilibrium at rest; rho_in 3 / 1, alpha 0.9 / 0.7
(pressure balance), A_R = A_B = 0.01, beta = 0.5, mu_R = mu_B = 0.075 (tau_v
= 1 for both fluids), other relaxation times 1.  The plates drag the fluid
and the drop until the flow is uniform; the improved model keeps the drop
circular and the original model turns it elliptic (the paper's Fig. 1).

`python -m paper_1904_03618_gb300.moving_droplet --steps 120000 --every 20000`
reports the drop's principal-axis ratio and position for both models.

The three-dimensional form (`--sphere`): a sphere of radius 20 centred in a
periodic 128^3 box, the whole fluid moving at (0.05, 0, 0) from t = 0,
density ratios 1 (alpha 1/3 for both) and 10 (alpha 0.97 / 0.7), viscosity
ratio 1 (tau_v = 1 for both), sigma = 0.005 (A_R = A_B = 0.01125), beta =
0.7, 20,000 steps.  Galilean invariance: the drop translates with the flow
(its centroid advances by U t) and keeps the shape of the initial sphere;
the record is the ratio of the largest to the smallest principal axis of the
red region (rho^N > 0), the centroid lag behind x0 + U t, and the red mass.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import lbm
from . import params as P
from . import workloads as wl


def case_params(improved=True, n=140, nz=4, U=0.02):
    """lbm_params keywords of the case."""
    nu_R = 0.075 / 3.0
    nu_B = 0.075 / 1.0
    aR = P.alpha_R_from_balance(3.0, 1.0, 0.7)
    return dict(nx=n, ny=n, nz=nz, wall=(0, 2, 0), wall_u=((U, 0.0, 0.0), (U, 0.0, 0.0)),
                improved=improved, rho_in_R=3.0, rho_in_B=1.0, alpha_R=aR, alpha_B=0.7,
                tau_R=P.tau_from_nu(nu_R, aR), tau_B=P.tau_from_nu(nu_B, 0.7), tau_e=1.0,
                tau_q=1.0, tau_pi=1.0, A_R=0.01, A_B=0.01, beta=0.5, delta=0.98)


def drop_shape(rR, rB, rin=(3.0, 1.0)):
    """(principal-axis ratio, x centroid) of the red region (rho^N > 0) of
    the first z layer; x is periodic (centroid from the circular mean)."""
    rn = ((rR / rin[0] - rB / rin[1]) / (rR / rin[0] + rB / rin[1]))[0]
    ny, nx = rn.shape
    ind = (rn > 0).astype(float)
    cx = (np.angle((ind.sum(0) * np.exp(2j * np.pi * np.arange(nx) / nx)).sum())
          % (2 * np.pi)) * nx / (2 * np.pi)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    m = ind.sum()
    cy = (ind * Y).sum() / m
    dx = (X - cx + nx / 2) % nx - nx / 2
    dy = Y - cy
    inertia = np.array([[(ind * dx * dx).sum(), (ind * dx * dy).sum()],
                        [(ind * dx * dy).sum(), (ind * dy * dy).sum()]]) / m
    ev = np.linalg.eigvalsh(inertia)
    return math.sqrt(ev[1] / ev[0]), cx


def run(improved=True, steps=120000, every=20000, device=None, log=None):
    dev = torch.device(device or "cuda")
    pd = case_params(improved)
    n, nz = pd["nx"], pd["nz"]
    rR, rB, u = wl.cylinder_z(n, n, nz, 30.0, 3.0, 1.0)
    stream = torch.cuda.Stream(dev)
    lat = lbm.Lattice(lbm.make_params(**pd), device=dev, stream=stream)
    rows = []
    try:
        lat.init_fields(rR, rB, u)
        done = 0
        while True:
            a, b, _ = (t.double().cpu().numpy() for t in lat.moments())
            ratio, cx = drop_shape(a, b)
            rows.append({"step": done, "aspect_ratio": ratio, "x_centroid": cx})
            if log:
                log("improved=%s step %d: aspect %.4f x %.2f" % (improved, done, ratio, cx))
            if done >= steps:
                break
            k = min(every, steps - done)
            lat.step(k)
            done += k
        diag = lat.diagnostics(raise_unstable=False)
    finally:
        lat.close()
    return {"improved": improved, "rows": rows, "nonfinite": diag[5], "mass_R": diag[0]}


def sphere_params(ratio, improved=True, n=128):
    """lbm_params keywords of the periodic 3D moving sphere (density ratio 1
    or 10, viscosity ratio 1 with both tau_v = 1)."""
    aB = 1.0 / 3.0 if ratio == 1 else 0.7
    aR = P.alpha_R_from_balance(float(ratio), 1.0, aB)
    A = P.A_from_sigma(0.005)
    return dict(nx=n, ny=n, nz=n, wall=(0, 0, 0), improved=improved, rho_in_R=float(ratio),
                rho_in_B=1.0, alpha_R=aR, alpha_B=aB, tau_R=1.0, tau_B=1.0, tau_e=1.0,
                tau_q=1.0, tau_pi=1.0, A_R=A, A_B=A, beta=0.7, delta=0.98)


def sphere_shape(rR, rB, rin):
    """(largest / smallest principal-axis ratio, centroid) of the red region
    (rho^N > 0) of a periodic 3D field (z, y, x); the centroid from circular
    means per axis."""
    rn = (rR / rin[0] - rB / rin[1]) / (rR / rin[0] + rB / rin[1])
    ind = (rn > 0).astype(float)
    shape = ind.shape  # (z, y, x)
    c = []
    for ax_cells, axis in ((shape[2], (0, 1)), (shape[1], (0, 2)), (shape[0], (1, 2))):
        prof = ind.sum(axis=axis)
        ang = np.angle((prof * np.exp(2j * np.pi * np.arange(ax_cells) / ax_cells)).sum())
        c.append((ang % (2 * np.pi)) * ax_cells / (2 * np.pi))
    Z, Y, X = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), np.arange(shape[2]),
                          indexing="ij")
    d = [(X - c[0] + shape[2] / 2) % shape[2] - shape[2] / 2,
         (Y - c[1] + shape[1] / 2) % shape[1] - shape[1] / 2,
         (Z - c[2] + shape[0] / 2) % shape[0] - shape[0] / 2]
    m = ind.sum()
    inertia = np.array([[(ind * d[i] * d[j]).sum() for j in range(3)] for i in range(3)]) / m
    ev = np.linalg.eigvalsh(inertia)
    return math.sqrt(ev[2] / ev[0]), c


def run_sphere(ratio, improved=True, steps=20000, every=5000, n=128, U=0.05, device=None,
               log=None):
    dev = torch.device(device or "cuda")
    pd = sphere_params(ratio, improved, n)
    rR, rB, u = wl.droplet(n, n, n, 20.0 * n / 128.0, float(ratio), 1.0, velocity=(U, 0.0, 0.0))
    stream = torch.cuda.Stream(dev)
    lat = lbm.Lattice(lbm.make_params(**pd), device=dev, stream=stream)
    rows = []
    rin = (float(ratio), 1.0)
    try:
        lat.init_fields(rR, rB, u)
        mass0 = lat.diagnostics(raise_unstable=False)[0]
        x0 = sphere_shape(rR, rB, rin)[1][0]
        done = 0
        while True:
            a, b, _ = (t.double().cpu().numpy() for t in lat.moments())
            ratio_ax, c = sphere_shape(a, b, rin)
            lag = ((x0 + U * done) - c[0] + n / 2) % n - n / 2
            diag = lat.diagnostics(raise_unstable=False)
            rows.append({"step": done, "axis_ratio": ratio_ax, "centroid_lag": lag,
                         "y": c[1], "z": c[2], "red_mass_rel_change": diag[0] / mass0 - 1.0,
                         "nonfinite": diag[5]})
            if log:
                log("ratio %g improved=%s step %d: axes %.4f lag %.3f" % (
                    ratio, improved, done, ratio_ax, lag))
            if done >= steps or diag[5] != 0:
                break
            k = min(every, steps - done)
            lat.step(k)
            done += k
    finally:
        lat.close()
    return {"density_ratio": ratio, "improved": improved, "rows": rows}


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="moving droplet between moving plates (Sec. IV.A)")
    ap.add_argument("--steps", type=int, default=120000)
    ap.add_argument("--every", type=int, default=20000)
    ap.add_argument("--sphere", action="store_true",
                    help="the 3D sphere in a periodic 128^3 uniform flow instead")
    args = ap.parse_args(argv)
    log = lambda m: print(m, flush=True)  # noqa: E731
    if args.sphere:
        out = [run_sphere(r, imp, args.steps, args.every, log=log)
               for r in (1, 10) for imp in (True, False)]
    else:
        out = [run(imp, args.steps, args.every, log=log) for imp in (True, False)]
    print(json.dumps(out))


if __name__ == "__main__":
    main()
