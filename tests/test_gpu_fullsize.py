"""Parity at full size, in the library's default launch configuration, on
sampled cells.

One step at a cell reads the pre-step populations within two cells of it
(pulls from x - e_i; the Eq. 49 stencil of the moments at x +- e, which
pull from one cell further).  So the oracle can reproduce any single cell
exactly from the 5 x 5 x 5 window of the pre-step state around it: periodic
axes wrap the window, an axis with walls takes the window flush against the
wall and gives the oracle that wall (the window's far side is then also a
wall, which no cell within two of the centre can see).  Samples: random
cells, interface cells and wall cells.

Workloads (the paper's cases at the sizes the benchmark configurations
name): the 3-D Rayleigh-Taylor instability of Sec. IV.C on 256 x 256 x 1024
(Eq. 56 perturbation, Atwood number 0.5, walls in z), FP32 and FP16; a drop
impact after Sec. IV.D on 256 x 256 x 160 (R = 30, density ratio 50, We 100,
Re 200, floor wall with the 120-degree contact-angle rule); the 512-case batched droplet
sweep."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1904_03618_gb300 import lbm, params as P, workloads as wl
from paper_1904_03618_gb300 import surrogate as S

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _axis_window(c, n, wall):
    """Indices of the 5-cell window around c on an axis of n cells, the
    centre's position in it, and whether the oracle gets walls on it."""
    if wall and c < 2:
        return list(range(5)), c, True
    if wall and c > n - 3:
        return list(range(n - 5, n)), c - (n - 5), True
    return [(c - 2 + k) % n for k in range(5)], 2, False


def _window_check(pd, f0, f1, cells, bound_fn):
    """Oracle step of the window of every sampled cell; returns the worst
    ratio |gpu - oracle| / bound over the sampled cells."""
    worst = 0.0
    nx, ny, nz = pd["nx"], pd["ny"], pd["nz"]
    wall = pd.get("wall", (0, 0, 0))
    for (x, y, z) in cells:
        xi, cx, wx = _axis_window(x, nx, wall[0])
        yi, cy, wy = _axis_window(y, ny, wall[1])
        zi, cz, wz = _axis_window(z, nz, wall[2])
        zt = torch.tensor(zi, device=DEV)[:, None, None]
        yt = torch.tensor(yi, device=DEV)[None, :, None]
        xt = torch.tensor(xi, device=DEV)[None, None, :]
        win = f0[:, :, zt, yt, xt].double().cpu().numpy()
        got = f1[:, :, z, y, x].double().cpu().numpy()
        q = dict(pd)
        q.update(nx=5, ny=5, nz=5, wall=(int(wx), int(wy), int(wz)))
        ref = oracle.step(oracle.params_from(q), win, 1)[:, :, cz, cy, cx]
        err = np.abs(got - ref).max()
        worst = max(worst, err / bound_fn(np.abs(win).max()))
    return worst


def _samples(shape, rhoN, nrand, ninterface, walls, seed):
    """Random cells, cells with |rho^N| < 0.5 and cells on the wall layers."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    out = [tuple(int(v) for v in (rng.integers(nx), rng.integers(ny), rng.integers(nz)))
           for _ in range(nrand)]
    idx = torch.nonzero(rhoN.abs() < 0.5)
    if len(idx):
        pick = rng.choice(len(idx), size=min(ninterface, len(idx)), replace=False)
        for p in pick:
            z, y, x = (int(v) for v in idx[int(p)].tolist())
            out.append((x, y, z))
    for z in walls:
        for _ in range(4):
            out.append((int(rng.integers(nx)), int(rng.integers(ny)), z))
    return out


def _rhoN(lat, pd):
    rR, rB, _ = lat.moments()
    r, b = rR / pd["rho_in_R"], rB / pd["rho_in_B"]
    return (r - b) / (r + b)


def _rt_case():
    L = 256
    nu = L * math.sqrt(L * 1e-5) / 256.0                 # Re = L sqrt(L g) / nu = 256
    aR = P.alpha_R_from_balance(3.0, 1.0, 0.7)
    return dict(nx=L, ny=L, nz=4 * L, wall=(0, 0, 1), improved=True, rho_in_R=3.0,
                rho_in_B=1.0, alpha_R=aR, alpha_B=0.7, tau_R=P.tau_from_nu(nu, aR),
                tau_B=P.tau_from_nu(nu, 0.7), A_R=1e-3, A_B=1e-3, beta=0.7, delta=0.98,
                gravity=(0.0, 0.0, -1e-5))


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_rayleigh_taylor_256x256x1024(storage):
    pd = _rt_case()
    rR, rB, u = wl.rayleigh_taylor(pd["nx"], pd["ny"], pd["nz"], pd["nx"], 0.05,
                                   2 * pd["nx"], pd["rho_in_R"], pd["rho_in_B"])
    p = lbm.make_params(storage=storage, **pd)
    if storage != "f32":
        p.ref_R, p.ref_B = 0.0, 0.0
    lat = lbm.Lattice(p, device=DEV, stream=torch.cuda.Stream(DEV))
    try:
        lat.init_fields(rR, rB, u)
        del rR, rB, u
        lat.step(30)
        rhoN = _rhoN(lat, pd)
        f0 = lat.get_f()
        lat.step(1)
        f1 = lat.get_f()
        d = lat.diagnostics()
    finally:
        lat.close()
    cells = _samples((pd["nz"], pd["ny"], pd["nx"]), rhoN, 16, 24, (0, 1, 1022, 1023), 3)
    if storage == "f32":
        bound = lambda fmax: 1e-5 * fmax
    else:  # one rounding of the stored value (deviations from 0 here)
        bound = lambda fmax: (2.0 ** -11 + 1e-5) * fmax
    assert _window_check(pd, f0, f1, cells, bound) <= 1.0
    assert d[5] == 0


def test_drop_impact_256x256x160_with_wetting():
    # U0 = 0.01 keeps A_k small at density ratio 50 and We = 100
    setup = S.ImpactSetup(radius=30, box=(256, 256, 160), speed=0.01)
    sample = {"density_ratio": 50.0, "viscosity_ratio": 10.0, "weber": 100.0,
              "reynolds": 200.0, "theta_deg": 120.0}
    prm, fields = S.impact_case(sample, setup)
    pd = {f: getattr(prm, f) for f in ("nx", "ny", "nz", "improved", "rho_in_R", "rho_in_B",
                                       "alpha_R", "alpha_B", "tau_R", "tau_B", "tau_e", "tau_q",
                                       "tau_pi", "A_R", "A_B", "beta", "delta",
                                       "contact_angle_deg")}
    pd.update(wall=tuple(prm.wall), wetting=True, force=tuple(prm.force),
              gravity=tuple(prm.gravity))
    lat = lbm.Lattice(prm, device=DEV, stream=torch.cuda.Stream(DEV))
    try:
        lat.init_fields(*fields)
        lat.step(1000)          # the drop has reached the floor (10 cells of travel)
        rhoN = _rhoN(lat, pd)
        f0 = lat.get_f()
        lat.step(1)
        f1 = lat.get_f()
        d = lat.diagnostics()
        # the wetted footprint under the drop, where the contact-angle rule acts
        floor = torch.nonzero(rhoN[0] > 0)
    finally:
        lat.close()
    assert len(floor) > 100
    cells = _samples((pd["nz"], pd["ny"], pd["nx"]), rhoN, 12, 24, (0, 1, 158, 159), 5)
    rng = np.random.default_rng(9)
    for p in rng.choice(len(floor), size=12, replace=False):
        y, x = (int(v) for v in floor[int(p)].tolist())
        cells.append((x, y, 0))
    assert _window_check(pd, f0, f1, cells, lambda fmax: 1e-5 * fmax) <= 1.0
    assert d[5] == 0


def test_batched_sweep_512_cases():
    samples = wl.droplet_sweep(512, seed=1234)
    cases = [P.droplet_case(s) for s in samples]
    plist, fields = [], []
    for c, s in zip(cases, samples):
        n = c["nx"]
        fields.append(wl.droplet(n, n, n, 0.25 * n, c["rho_in_R"], 1.0,
                                 velocity=(s["speed"], 0.0, 0.0)))
        plist.append(lbm.make_params(**c))
    stream = torch.cuda.Stream(DEV)
    b = lbm.Batch(plist, device=DEV, stream=stream)
    try:
        for k, f in enumerate(fields):
            b.init_fields(k, *f)
        del fields
        b.step(10)
        picks = [0, 1, 2, 3, 100, 257, 400, 511]
        before = {k: (b.get_f(k), _rhoN_batch(b, k, cases[k])) for k in picks}
        b.step(1)
        worst = 0.0
        for k in picks:
            f0, rhoN = before[k]
            f1 = b.get_f(k)
            n = cases[k]["nx"]
            cells = _samples((n, n, n), rhoN, 3, 3, (), 11 + k)
            worst = max(worst, _window_check(cases[k], f0, f1, cells,
                                             lambda fmax: 1e-5 * fmax))
        assert worst <= 1.0
    finally:
        b.close()


def _rhoN_batch(b, k, c):
    rR, rB, _ = b.moments(k)
    r, bl = rR / c["rho_in_R"], rB / c["rho_in_B"]
    return (r - bl) / (r + bl)
