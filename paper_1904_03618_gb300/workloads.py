"""Seeded synthetic inputs: initial density and velocity fields, raw population
arrays, and the lattice shapes of the paper's test cases.

This module holds geometry and random numbers only -- no step of the method.
It is the one module that both the CUDA path's callers (tests, benchmark) and
the CPU oracle's callers use, so that both start from identical inputs.

Conventions: arrays are numpy float64 in C order with x fastest; scalar fields
have shape (nz, ny, nx), vector fields (3, nz, ny, nx), population arrays
(2, 19, nz, ny, nx) with colour 0 = red, 1 = blue.  Lattice cells sit at
integer coordinates; "centred" means the centre (n - 1) / 2 on each axis.
"""
from __future__ import annotations

import numpy as np


def _grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64),
                          np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def droplet(nx, ny, nz, radius, rho_in_R, rho_in_B, velocity=(0.0, 0.0, 0.0),
            center=None, noise=0.0, seed=0):
    """Sharp-interface sphere of the red fluid (density rho_in_R) in the blue
    fluid (rho_in_B), uniform velocity.  ``noise`` > 0 multiplies every
    non-zero density by (1 + U(-noise, noise)) drawn from ``seed``.
    Returns (rho_R, rho_B, u)."""
    x, y, z = _grid(nx, ny, nz)
    if center is None:
        center = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    r2 = (x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2
    inside = r2 <= radius * radius
    rho_R = np.where(inside, rho_in_R, 0.0)
    rho_B = np.where(inside, 0.0, rho_in_B)
    if noise > 0.0:
        rng = np.random.default_rng(seed)
        rho_R = rho_R * (1.0 + rng.uniform(-noise, noise, rho_R.shape))
        rho_B = rho_B * (1.0 + rng.uniform(-noise, noise, rho_B.shape))
    u = np.zeros((3, nz, ny, nx))
    for a in range(3):
        u[a] = velocity[a]
    return rho_R, rho_B, u


def cylinder_z(nx, ny, nz, radius, rho_in_R, rho_in_B, velocity=(0.0, 0.0, 0.0),
               center=None):
    """Red column along z (a 2D circular droplet extruded in z)."""
    x, y, _ = _grid(nx, ny, nz)
    if center is None:
        center = ((nx - 1) / 2.0, (ny - 1) / 2.0)
    inside = (x - center[0]) ** 2 + (y - center[1]) ** 2 <= radius * radius
    rho_R = np.where(inside, rho_in_R, 0.0)
    rho_B = np.where(inside, 0.0, rho_in_B)
    u = np.zeros((3, nz, ny, nx))
    for a in range(3):
        u[a] = velocity[a]
    return rho_R, rho_B, u


def layered(nx, ny, nz, a, rho_in_R, rho_in_B):
    """Layered channel between walls at y = -1/2 and y = ny - 1/2: red where
    |y_j| <= a with y_j = j + 1/2 - ny/2, blue elsewhere; at rest."""
    _, y, _ = _grid(nx, ny, nz)
    yc = y + 0.5 - ny / 2.0
    inside = np.abs(yc) <= a
    rho_R = np.where(inside, rho_in_R, 0.0)
    rho_B = np.where(inside, 0.0, rho_in_B)
    return rho_R, rho_B, np.zeros((3, nz, ny, nx))


def layered_nodes(nx, ny, nz, a, rho_in_R, rho_in_B):
    """Layered channel between no-slip plates lying on the first and last
    node of y: node j sits at y_j = j - (ny - 1)/2 (the plates at +-(ny - 1)/2),
    red where |y_j| <= a, blue elsewhere; at rest."""
    _, y, _ = _grid(nx, ny, nz)
    yc = y - (ny - 1) / 2.0
    inside = np.abs(yc) <= a
    rho_R = np.where(inside, rho_in_R, 0.0)
    rho_B = np.where(inside, 0.0, rho_in_B)
    return rho_R, rho_B, np.zeros((3, nz, ny, nx))


def rayleigh_taylor(nx, ny, nz, L, amplitude, z_interface, rho_in_R, rho_in_B,
                    dtype=np.float64):
    """Heavy red fluid above light blue fluid; interface height
    z_interface + h(x, y), h = amplitude * L * [cos(2 pi x / L) + cos(2 pi y / L)]
    (the single-mode perturbation of the paper's Rayleigh-Taylor case).
    Coordinates broadcast (no full grids), so lattices of 10^9 cells fit in
    host memory with dtype=np.float32."""
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    h = amplitude * L * (np.cos(2 * np.pi * x / L) + np.cos(2 * np.pi * y / L))
    upper = z >= z_interface + h
    rho_R = upper.astype(dtype) * dtype(rho_in_R)
    rho_B = (~upper).astype(dtype) * dtype(rho_in_B)
    return rho_R, rho_B, np.zeros((3, nz, ny, nx), dtype=dtype)


def random_populations(nx, ny, nz, seed=0, low=0.01, high=0.1):
    """Arbitrary positive populations, U(low, high) per entry: a far-from-
    equilibrium state for single-step algebra checks."""
    rng = np.random.default_rng(seed)
    return rng.uniform(low, high, (2, 19, nz, ny, nx))


def random_fields(nx, ny, nz, seed=0, rho_lo=0.2, rho_hi=1.0, umax=0.05):
    """Smooth-free random densities in [rho_lo, rho_hi] for both colours and
    velocities in [-umax, umax]: every cell is an interface cell."""
    rng = np.random.default_rng(seed)
    rho_R = rng.uniform(rho_lo, rho_hi, (nz, ny, nx))
    rho_B = rng.uniform(rho_lo, rho_hi, (nz, ny, nx))
    u = rng.uniform(-umax, umax, (3, nz, ny, nx))
    return rho_R, rho_B, u


def droplet_sweep(ncases, seed=1234, edges=(32, 48, 64, 96)):
    """Sampled parameters of a batched droplet sweep: per case a cubic box
    edge drawn uniformly from `edges`, a density ratio in [1, 20], a surface
    tension in [0.001, 0.02] and a speed in [0, 0.05] along x; every second
    case is static (speed 0).  Returns a list of dicts of raw samples."""
    rng = np.random.default_rng(seed)
    e = rng.choice(np.asarray(edges), size=ncases)
    ratio = rng.uniform(1.0, 20.0, ncases)
    sigma = rng.uniform(0.001, 0.02, ncases)
    speed = rng.uniform(0.0, 0.05, ncases)
    out = []
    for k in range(ncases):
        out.append(dict(edge=int(e[k]), density_ratio=float(ratio[k]),
                        sigma=float(sigma[k]),
                        speed=0.0 if k % 2 == 0 else float(speed[k])))
    return out
