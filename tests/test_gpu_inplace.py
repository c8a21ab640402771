"""lbm_step_inplace: the step on one population array (AA access pattern).

Checks, against the FP64 oracle on the same input: the initial state
(equilibrium of the fields); every step of four from it -- both parities,
read back through lbm_inplace_read -- against the oracle stepped once from
the GPU's previous state, element by element, within the FP32 bar of the
other parity tests (relative L-infinity 1e-5 per step); the moments; the
odd layout as include/lbm.h documents it, read from the raw array; the
context API on the same input; FP16 / BF16 deviation storage against the
oracle with the same storage rounding and against the context's 16-bit
run; periodic, walled, gravity, wetting and BGK
lattices and lattices of one to three cells along an axis; and the
Rayleigh-Taylor lattice of the paper's Sec. IV.C at 512 x 512 x 2048 (537 M
cells, beyond the two-buffer kernels' 226 M-cell limit) on sampled cells
against the oracle's 5 x 5 x 5 windows, one step from each parity.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1904_03618_gb300 import lbm, params as P, workloads as wl
from storage_emulation import offsets, stored
from test_gpu_fullsize import _axis_window

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")

# D3Q19 in the order of Eq. 5 (the layout of include/lbm.h); opp pairs
# (1,2), (3,4), ..., (17,18).
EX = (0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0)
EY = (0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1)
EZ = (0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1)
OPP = tuple(0 if i == 0 else (i + 1 if i % 2 else i - 1) for i in range(19))


def test_velocity_table_is_the_oracles():
    """One unit population in direction i carries momentum e_i."""
    op = oracle.params(1, 1, 1)
    for i in range(19):
        f = np.zeros((2, 19, 1, 1, 1))
        f[0, i] = 1.0
        _, _, u = oracle.moments(op, f)
        assert np.allclose(u[:, 0, 0, 0], (EX[i], EY[i], EZ[i]), atol=1e-12)
        assert (EX[OPP[i]], EY[OPP[i]], EZ[OPP[i]]) == (-EX[i], -EY[i], -EZ[i])


def _pd(**kw):
    d = dict(wall=(0, 0, 0), improved=True, rho_in_R=3.0, rho_in_B=1.0, alpha_R=0.9,
             alpha_B=0.7, tau_R=0.8, tau_B=1.1, tau_e=1.0, tau_q=0.95, tau_pi=1.05,
             A_R=0.01, A_B=0.01, beta=0.7, delta=0.98, force=(2e-5, 0.0, 0.0),
             gravity=(0.0, 0.0, 0.0))
    d.update(kw)
    return d


def _rel_linf(a, b):
    a = a.double().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return np.abs(a - b).max() / np.abs(b).max()


def _fields(nx, ny, nz, seed):
    if min(nx, ny, nz) >= 8:
        r = 0.3 * min(nx, ny, nz)
        return wl.droplet(nx, ny, nz, r, 3.0, 1.0, velocity=(0.02, 0.01, -0.01),
                          noise=1e-3, seed=seed)
    return wl.random_fields(nx, ny, nz, seed=seed)


CASES = {
    # name: (nx, ny, nz, overrides); nx = 133 spans a full 128-thread block
    # and a ragged tail
    "periodic": (133, 11, 9, {}),
    "walls": (133, 11, 9, dict(wall=(1, 1, 1))),
    "z_walls_gravity": (133, 11, 9, dict(wall=(0, 0, 1), gravity=(0.0, 0.0, -1e-5))),
    "wetting": (40, 12, 10, dict(wall=(1, 1, 1), wetting=True, contact_angle_deg=60.0)),
    "bgk": (133, 11, 9, dict(wall=(0, 0, 1), collision="bgk")),
    "original_model": (37, 10, 8, dict(improved=False)),
    "one_cell_y_walls": (5, 1, 3, dict(wall=(0, 1, 0))),
    "two_cells": (2, 3, 2, {}),
    # several blocks along x (ragged) and more rows and planes
    "blocks_rows_planes": (170, 37, 19, {}),
    "blocks_rows_planes_walls": (170, 37, 19, dict(wall=(1, 1, 1))),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_inplace_steps_match_the_oracle(name):
    nx, ny, nz, kw = CASES[name]
    pd = _pd(**kw)
    p = lbm.make_params(nx, ny, nz, **pd)
    op = oracle.params_from(dict(pd, nx=nx, ny=ny, nz=nz))
    rR, rB, u = _fields(nx, ny, nz, seed=len(name))
    lat = lbm.InPlaceLattice(p, device=DEV)
    lat.init_fields(rR, rB, u)
    assert _rel_linf(lat.get_f(), oracle.init(op, rR, rB, u)) <= 1e-6
    for k in range(4):
        prev = lat.get_f().double().cpu().numpy()
        lat.step(1)
        assert lat.parity == (k + 1) % 2
        ref = oracle.step(op, prev, 1)
        assert _rel_linf(lat.get_f(), ref) <= 1e-5, (name, k)
        mR, mB, mu = lat.moments()
        oR, oB, ou = oracle.moments(op, ref)
        assert _rel_linf(mR, oR) <= 1e-5 and _rel_linf(mB, oB) <= 1e-5
        assert np.abs(mu.double().cpu().numpy() - ou).max() <= 1e-5 * max(1.0, np.abs(ou).max())


def test_several_steps_in_one_call_equal_single_calls():
    nx, ny, nz, kw = CASES["z_walls_gravity"]
    p = lbm.make_params(nx, ny, nz, **_pd(**kw))
    fields = _fields(nx, ny, nz, seed=5)
    a = lbm.InPlaceLattice(p, device=DEV)
    b = lbm.InPlaceLattice(p, device=DEV)
    a.init_fields(*fields)
    b.init_fields(*fields)
    a.step(3)
    for _ in range(3):
        b.step(1)
    assert a.parity == b.parity == 1
    assert torch.equal(a.f, b.f)
    f_before = a.f.clone()
    a.step(0)
    assert a.parity == 1 and torch.equal(a.f, f_before)


@pytest.mark.parametrize("wall", [(0, 0, 0), (1, 1, 1), (0, 1, 0)])
def test_odd_layout_is_the_documented_one(wall):
    """Odd state: f_i(x, t) at slot (opp(i), x - e_i), or (i, x) where
    x - e_i lies beyond a wall -- rebuilt here from the raw array."""
    nx, ny, nz = 19, 7, 6
    p = lbm.make_params(nx, ny, nz, **_pd(wall=wall))
    lat = lbm.InPlaceLattice(p, device=DEV)
    lat.init_fields(*_fields(nx, ny, nz, seed=2))
    lat.step(1)
    raw = lat.f.cpu().numpy()
    want = np.empty_like(raw)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for i in range(19):
                    s = [x - EX[i], y - EY[i], z - EZ[i]]
                    beyond = any(wall[a] and not 0 <= s[a] < n
                                 for a, n in enumerate((nx, ny, nz)))
                    if beyond:
                        want[:, i, z, y, x] = raw[:, i, z, y, x]
                    else:
                        want[:, i, z, y, x] = raw[:, OPP[i], s[2] % nz, s[1] % ny, s[0] % nx]
    assert np.array_equal(lat.get_f().cpu().numpy(), want)


def test_inplace_matches_the_context_api():
    nx, ny, nz, kw = CASES["z_walls_gravity"]
    p = lbm.make_params(nx, ny, nz, **_pd(**kw))
    fields = _fields(nx, ny, nz, seed=9)
    ctx = lbm.Lattice(p, device=DEV)
    ctx.init_fields(*fields)
    f0 = ctx.get_f()
    ctx.step(3)
    ref = ctx.get_f().double().cpu().numpy()
    ctx.close()
    lat = lbm.InPlaceLattice(p, device=DEV)
    lat.set_f(f0)
    lat.step(3)
    assert _rel_linf(lat.get_f(), ref) <= 3e-5


def test_inplace_rejects_bad_device_arguments():
    p = lbm.make_params(8, 8, 8)
    f = torch.zeros(38 * 512 + 64 * 4, device=DEV)
    with pytest.raises(lbm.LbmError) as ei:      # scratch inside f
        lbm.lbm_step_inplace(p, f, 0, 1, f[64:])
    assert "overlap" in str(ei.value)
    host = torch.zeros(38 * 512)
    scratch = torch.zeros(512 * 4, device=DEV)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_step_inplace(p, host, 0, 1, scratch)
    assert "device memory" in str(ei.value)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_inplace_read(p, f, 0, f_out=f[4:])
    assert "overlaps" in str(ei.value)
    with pytest.raises(lbm.LbmError) as ei:      # the FP32 input inside the state
        lbm.lbm_inplace_set(p, f[4:], f)
    assert "overlap" in str(ei.value)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_inplace_set(p, host, scratch.repeat(10))
    assert "device memory" in str(ei.value)
    p16 = lbm.make_params(8, 8, 8, storage="f16")
    raw = torch.zeros(38 * 512 + 8, dtype=torch.float16, device=DEV)
    fin = torch.zeros(38 * 512, device=DEV)
    with pytest.raises(lbm.LbmError) as ei:      # 16-bit values one byte off
        lbm._inplace_check(lbm._lib.lbm_inplace_set(
            lbm.ctypes.byref(p16), fin.data_ptr(), raw.data_ptr() + 1, None))
    assert "misaligned" in str(ei.value)
    lbm.lbm_inplace_set(p16, fin, raw[2:])       # 2-byte aligned 16-bit values: accepted
    torch.cuda.synchronize()


# ---------------------------------------------------------------------------
# FP16 / BF16 deviation storage in place.

@pytest.mark.parametrize("storage,bars", [("f16", dict(emu=5e-4, ctx=5e-4)),
                                          ("bf16", dict(emu=4e-3, ctx=4e-3))])
def test_inplace_16_bit_storage(storage, bars):
    """The in-place step on FP16 / BF16 deviations (the blue background
    offset by rho_in_B phi_i^B, red stored as is): set_f rounds exactly as
    the storage model of the two-buffer context does, and after 101 steps
    (ending on an odd state, read back through lbm_inplace_read) the state is
    within the FP32-versus-FP64 tie flips of the FP64 oracle with the same
    storage rounding after every step -- several times closer than to the
    unrounded oracle (on a GB300: FP16 relative L2 2.2e-4 against 1.4e-3,
    BF16 1.7e-3 against 1.8e-2) -- and as close to the two-buffer context's
    16-bit run from the same state.  Walls in z, gravity."""
    nx, ny, nz = 40, 24, 20
    pd = _pd(wall=(0, 0, 1), gravity=(0.0, 0.0, -1e-5))
    rR, rB, u = wl.droplet(nx, ny, nz, 7.0, 3.0, 1.0, velocity=(0.02, -0.01, 0.0),
                           noise=1e-3, seed=11)
    op = oracle.params_from(dict(nx=nx, ny=ny, nz=nz, **pd))
    ref_R, ref_B = 0.0, pd["rho_in_B"]
    off = offsets(pd, ref_R, ref_B)
    f0 = np.asarray(oracle.init(op, rR, rB, u), dtype=np.float32).astype(np.float64)
    p = lbm.make_params(nx, ny, nz, storage=storage, **pd)
    p.ref_R, p.ref_B = ref_R, ref_B
    steps = 101

    lat = lbm.InPlaceLattice(p, device=DEV)
    lat.set_f(torch.tensor(f0, dtype=torch.float32, device=DEV))
    held = lat.get_f().double().cpu().numpy()
    lat.step(steps)
    assert lat.parity == 1
    got = lat.get_f().double().cpu().numpy()
    lat.close()
    emu = stored(f0, storage, off)
    assert np.array_equal(held, emu)
    plain = emu.copy()
    for _ in range(steps):
        emu = stored(oracle.step(op, emu, 1), storage, off)
    plain = oracle.step(op, plain, steps)
    norm = np.linalg.norm(emu)
    e_emu = np.linalg.norm(got - emu) / norm
    e_plain = np.linalg.norm(got - plain) / norm
    assert e_emu <= bars["emu"] and e_emu <= 0.25 * e_plain, (e_emu, e_plain)

    ctx = lbm.Lattice(p, device=DEV)
    ctx.set_f(torch.tensor(f0, dtype=torch.float32, device=DEV))
    ctx.step(steps)
    two = ctx.get_f().double().cpu().numpy()
    ctx.close()
    e_ctx = np.linalg.norm(got - two) / norm
    print(storage, "in place: rel L2 vs emulated %.3e, vs unrounded %.3e, vs context %.3e"
          % (e_emu, e_plain, e_ctx))
    assert e_ctx <= bars["ctx"]


# ---------------------------------------------------------------------------
# Full size: Rayleigh-Taylor, 512 x 512 x 2048.

def _rt_pd(L):
    nu = L * math.sqrt(L * 1e-5) / 256.0                 # Re = L sqrt(L g) / nu = 256
    aR = P.alpha_R_from_balance(3.0, 1.0, 0.7)
    return dict(nx=L, ny=L, nz=4 * L, wall=(0, 0, 1), improved=True, rho_in_R=3.0,
                rho_in_B=1.0, alpha_R=aR, alpha_B=0.7, tau_R=P.tau_from_nu(nu, aR),
                tau_B=P.tau_from_nu(nu, 0.7), A_R=1e-3, A_B=1e-3, beta=0.7, delta=0.98,
                gravity=(0.0, 0.0, -1e-5))


def _rt_fields_on_device(nx, ny, nz, L, amplitude, z0, rho_R_in, rho_B_in):
    """The fields of workloads.rayleigh_taylor, built on the device (the host
    generator's float64 grids would take tens of GB at this size)."""
    x = torch.arange(nx, device=DEV, dtype=torch.float64)
    y = torch.arange(ny, device=DEV, dtype=torch.float64)
    h = amplitude * L * (torch.cos(2 * math.pi * x / L)[None, :] +
                         torch.cos(2 * math.pi * y / L)[:, None])
    rR = torch.empty((nz, ny, nx), device=DEV, dtype=torch.float32)
    rB = torch.empty_like(rR)
    for z in range(0, nz, 256):
        zz = torch.arange(z, min(z + 256, nz), device=DEV, dtype=torch.float64)
        upper = zz[:, None, None] >= (z0 + h)[None]
        rR[z:z + len(zz)] = torch.where(upper, rho_R_in, 0.0).float()
        rB[z:z + len(zz)] = torch.where(upper, 0.0, rho_B_in).float()
    return rR, rB, torch.zeros((3, nz, ny, nx), device=DEV, dtype=torch.float32), h


def _gather(f, parity, wall, dims, zt, yt, xt):
    """f_i^k(x, t) at the cells (zt, yt, xt) (broadcasting index tensors) of
    an in-place state of the given parity, by the documented layout."""
    if parity == 0:
        return f[:, :, zt, yt, xt]
    nx, ny, nz = dims
    shape = torch.broadcast_shapes(zt.shape, yt.shape, xt.shape)
    vals = []
    for i in range(19):
        sx, sy, sz = xt - EX[i], yt - EY[i], zt - EZ[i]
        beyond = torch.zeros(shape, dtype=torch.bool, device=f.device)
        for s, n, w in ((sx, nx, wall[0]), (sy, ny, wall[1]), (sz, nz, wall[2])):
            if w:
                beyond = beyond | (s < 0) | (s >= n)
        nb = f[:, OPP[i], sz % nz, sy % ny, sx % nx]
        me = f[:, i, zt, yt, xt]
        vals.append(torch.where(beyond, me, nb))
    return torch.stack(vals, dim=1)


def test_rayleigh_taylor_512x512x2048_in_place():
    pd = _rt_pd(512)
    nx, ny, nz = pd["nx"], pd["ny"], pd["nz"]
    N = nx * ny * nz
    free, _ = torch.cuda.mem_get_info(DEV)
    need = N * (152 + 16 + 20) + (8 << 30)
    if free < need:
        pytest.skip("needs %.0f GB of free device memory, %.0f free" % (need / 1e9, free / 1e9))
    p = lbm.make_params(**pd)
    with pytest.raises(lbm.LbmError):                 # beyond the two-buffer limit
        lbm.lbm_create(p)
    lat = lbm.InPlaceLattice(p, device=DEV, stream=torch.cuda.Stream(DEV))
    rR, rB, u, h = _rt_fields_on_device(nx, ny, nz, nx, 0.05, 2 * nx, pd["rho_in_R"],
                                        pd["rho_in_B"])
    lat.init_fields(rR, rB, u)
    del rR, rB, u
    torch.cuda.empty_cache()

    rng = np.random.default_rng(11)
    cells = [(int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz)))
             for _ in range(12)]
    for _ in range(16):                                # interface cells
        x, y = int(rng.integers(nx)), int(rng.integers(ny))
        zi = int(math.ceil(2 * nx + float(h[y, x])))
        cells.append((x, y, zi - 1 + int(rng.integers(2))))
    for z in (0, 1, nz - 2, nz - 1):                   # wall layers
        cells += [(int(rng.integers(nx)), int(rng.integers(ny)), z) for _ in range(3)]
    cells += [(0, 0, nz // 2), (nx - 1, ny - 1, nz // 2), (0, ny - 1, 2 * nx)]  # seams
    # block boundaries along x (128-thread blocks)
    cells += [(127, 15, 127), (128, 16, 128), (255, 47, 255), (256, 48, 256)]
    wall = pd["wall"]
    dims = (nx, ny, nz)
    for start in (0, 1):                               # step 1 from even, step 2 from odd
        assert lat.parity == start
        wins, where = [], []
        for (x, y, z) in cells:
            xi, cx, wx = _axis_window(x, nx, wall[0])
            yi, cy, wy = _axis_window(y, ny, wall[1])
            zi, cz, wz = _axis_window(z, nz, wall[2])
            zt = torch.tensor(zi, device=DEV)[:, None, None]
            yt = torch.tensor(yi, device=DEV)[None, :, None]
            xt = torch.tensor(xi, device=DEV)[None, None, :]
            wins.append(_gather(lat.f, lat.parity, wall, dims, zt, yt, xt).double().cpu().numpy())
            where.append((cx, cy, cz, wx, wy, wz))
        lat.step(1)
        lat.stream.synchronize()
        worst = 0.0
        for (x, y, z), win, (cx, cy, cz, wx, wy, wz) in zip(cells, wins, where):
            t = lambda v: torch.tensor([v], device=DEV)
            got = _gather(lat.f, lat.parity, wall, dims, t(z), t(y), t(x))[:, :, 0]
            q = dict(pd, nx=5, ny=5, nz=5, wall=(int(wx), int(wy), int(wz)))
            ref = oracle.step(oracle.params_from(q), win, 1)[:, :, cz, cy, cx]
            err = np.abs(got.double().cpu().numpy() - ref).max()
            worst = max(worst, err / (1e-5 * np.abs(win).max()))
        assert worst <= 1.0, (start, worst)
