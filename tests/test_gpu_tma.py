"""The TMA-staged fused step (hold 7: two stages, hold 8: one stage; tile_y 8
= 32 x 8 threads, 16 = 16 x 16, 15 = 34 x 15): same populations as the oracle and
as the shared-memory-hold kernel it restages (hold 2), on lattices with
several tiles, ragged tails, periodic seams and walls.  The two kernels run
the same arithmetic; the compiler may contract different products into
FMAs, so they agree to FP32 rounding (a few ulp), not bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_1904_03618_gb300 import lbm, workloads as wl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def base(nx, ny, nz, **kw):
    d = dict(nx=nx, ny=ny, nz=nz, wall=(0, 0, 0), improved=True, rho_in_R=3.0,
             rho_in_B=1.0, alpha_R=0.9, alpha_B=0.7, tau_R=0.8, tau_B=1.1,
             tau_e=1.0, tau_q=0.95, tau_pi=1.05, A_R=0.01, A_B=0.01, beta=0.7,
             delta=0.98, force=(2e-5, 0.0, 0.0), gravity=(0.0, 0.0, -1e-5))
    d.update(kw)
    return d


def state(pd, radius, velocity, seed=0):
    rR, rB, u = wl.droplet(pd["nx"], pd["ny"], pd["nz"], radius, pd["rho_in_R"],
                           pd["rho_in_B"], velocity=velocity, noise=1e-3, seed=seed)
    f = oracle.init(oracle.params_from(pd), rR, rB, u)
    return np.asarray(f, dtype=np.float32).astype(np.float64)


TMA = [(8, 7), (8, 8), (16, 7), (16, 8), (15, 7), (15, 8)]


def run(pd, f0, steps, hold, zchunk=0, storage="f32", tile_y=8):
    p = lbm.make_params(storage=storage, **pd)
    if storage != "f32":
        p.ref_R, p.ref_B = 0.0, pd["rho_in_B"]
    lat = lbm.Lattice(p, device=DEV)
    lbm.lbm_set_fused_config(lat.ctx, tile_y, zchunk, hold)
    lat.set_f(torch.tensor(f0, dtype=torch.float32, device=DEV))
    lat.step(steps)
    out = lat.get_f().double().cpu().numpy()
    diag = lat.diagnostics()
    lat.close()
    return out, diag


CASES = {
    "periodic": dict(nx=72, ny=37, nz=19),
    "z_walls": dict(nx=64, ny=23, nz=14, wall=(0, 0, 1)),
    "all_walls_original": dict(nx=36, ny=20, nz=12, wall=(1, 1, 1), improved=False),
    "y_walls_wetting": dict(nx=40, ny=26, nz=10, wall=(0, 1, 0), wetting=True,
                            contact_angle_deg=60.0),
    "thin": dict(nx=4, ny=7, nz=3),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("zchunk", [0, 5])
@pytest.mark.parametrize("tile_y,hold", TMA)
def test_tma_matches_oracle_and_hold2(name, zchunk, tile_y, hold):
    kw = dict(CASES[name])
    pd = base(**{k: kw.pop(k) for k in ("nx", "ny", "nz")}, **kw)
    f0 = state(pd, min(pd["nx"], pd["ny"], pd["nz"]) / 3.0, (0.02, 0.01, 0.005))
    got, diag = run(pd, f0, 3, hold, zchunk, tile_y=tile_y)
    ref_gpu, _ = run(pd, f0, 3, 2, zchunk)
    ref = oracle.step(oracle.params_from(pd), f0, 3)
    assert np.abs(got - ref).max() / np.abs(ref).max() <= 1e-5
    assert np.abs(got - ref_gpu).max() / np.abs(ref_gpu).max() <= 1e-6
    assert diag[5] == 0


SEAM_CASES = [(72, 37, 19), (34, 15, 6), (36, 16, 5), (130, 44, 11), (64, 28, 9)]


@pytest.mark.parametrize("zwall", [0, 1])
@pytest.mark.parametrize("tile_y,hold", [(15, 8), (12, 7)])
@pytest.mark.parametrize("nx,ny,nz", SEAM_CASES)
def test_seam_form_matches_oracle_across_the_periodic_seams(nx, ny, nz, tile_y, hold, zwall):
    """On a periodic FP32 lattice the 34 x 15 one-stage form and the 34 x 12
    two-stage form (the library default there) stage the cells beyond the x
    and y seams by tensor copies of the lattice's far side.  A drop centred
    on the corner (0, 0) puts the interface across both seams and their
    corner.  With walls in z (zwall = 1) the first and last plane are pulled
    from global memory, the rest staged."""
    pd = base(nx, ny, nz, wall=(0, 0, zwall))
    rR, rB, u = wl.droplet(nx, ny, nz, 6.0, pd["rho_in_R"], pd["rho_in_B"],
                           velocity=(0.02, -0.01, 0.005), center=(0.5, 0.5, nz / 2.0),
                           noise=1e-3, seed=3)
    f0 = np.asarray(oracle.init(oracle.params_from(pd), rR, rB, u),
                    dtype=np.float32).astype(np.float64)
    got, diag = run(pd, f0, 3, hold, 0, tile_y=tile_y)
    ref_gpu, _ = run(pd, f0, 3, 2, 0)
    ref = oracle.step(oracle.params_from(pd), f0, 3)
    assert np.abs(got - ref).max() / np.abs(ref).max() <= 1e-5
    assert np.abs(got - ref_gpu).max() / np.abs(ref_gpu).max() <= 1e-6
    assert diag[5] == 0


def test_two_stage_seam_tile_is_accepted_only_where_it_applies():
    for storage in ("f32", "f16", "bf16"):
        ok = lbm.Lattice(lbm.make_params(storage=storage, **base(64, 30, 9, wall=(0, 0, 1))),
                         device=DEV)
        lbm.lbm_set_fused_config(ok.ctx, 12, 0, 7)
        assert lbm.lbm_get_fused_config(ok.ctx)[0] == 12
        ok.close()
    refused = [dict(base(64, 30, 9, wall=(1, 0, 0))),            # x walls
               dict(base(64, 30, 9), collision="bgk"),           # BGK: shared-memory hold
               dict(base(30, 30, 9)),                            # nx < 34
               dict(base(64, 30, 9), storage="f16", wall=(0, 1, 0)),  # 16-bit, y walls
               dict(base(66, 30, 9), storage="f16")]             # 16-bit, nx % 4 != 0
    for d in refused:
        storage = d.pop("storage", "f32")
        lat = lbm.Lattice(lbm.make_params(storage=storage, **d), device=DEV)
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_set_fused_config(lat.ctx, 12, 0, 7)
        assert ei.value.status == lbm.LBM_ERR_ARG
        for hold in (2, 8):
            with pytest.raises(lbm.LbmError):
                lbm.lbm_set_fused_config(lat.ctx, 12, 0, hold)
        lat.close()


def test_seam_form_is_the_default_on_a_periodic_fp32_cube():
    lat = lbm.Lattice(lbm.make_params(**base(128, 128, 128)), device=DEV)
    assert tuple(lbm.lbm_get_fused_config(lat.ctx))[::2] == (12, 7)
    lat.close()


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("tile_y,hold", TMA)
def test_tma_reduced_precision(storage, tile_y, hold):
    """Same stored values as hold 2 up to one rounding step of the storage
    format (a few FP32-ulp differences can flip a rounding)."""
    pd = base(72, 31, 17, wall=(0, 0, 1))
    f0 = state(pd, 8.0, (0.02, 0.0, 0.01))
    got, _ = run(pd, f0, 4, hold, storage=storage, tile_y=tile_y)
    ref, _ = run(pd, f0, 4, 2, storage=storage)
    ulp = 2.0 ** -10 if storage == "f16" else 2.0 ** -7
    assert np.abs(got - ref).max() <= ulp * np.abs(ref).max()


@pytest.mark.parametrize("tile_y,hold", TMA)
def test_tma_long_run_matches_hold2(tile_y, hold):
    """200 steps: the two kernels stay within the FP32 parity bar."""
    pd = base(96, 48, 40)
    f0 = state(pd, 12.0, (0.03, 0.0, 0.0))
    got, d1 = run(pd, f0, 200, hold, tile_y=tile_y)
    ref, d2 = run(pd, f0, 200, 2)
    assert np.abs(got - ref).max() / np.abs(ref).max() <= 1e-5
    assert abs(d1[0] - d2[0]) <= 1e-6 * d2[0] and abs(d1[1] - d2[1]) <= 1e-6 * d2[1]


def test_tma_rejected_where_rows_are_not_16_byte_multiples():
    for nx, storage in [(71, "f32"), (70, "f16")]:
        lat = lbm.Lattice(lbm.make_params(**base(nx, 12, 8), storage=storage), device=DEV)
        try:
            for tile_y, hold in TMA:
                with pytest.raises(lbm.LbmError):
                    lbm.lbm_set_fused_config(lat.ctx, tile_y, 0, hold)
        finally:
            lat.close()
    # the 34 x 15 tile exists only in the TMA form
    lat = lbm.Lattice(lbm.make_params(**base(72, 12, 8)), device=DEV)
    try:
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_fused_config(lat.ctx, 15, 0, 2)
    finally:
        lat.close()


SEAM16_CASES = [(72, 37, 19), (36, 16, 5), (132, 44, 11), (64, 28, 9), (100, 33, 7)]


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("tile_y", [15, 12])
@pytest.mark.parametrize("zwall", [0, 1])
@pytest.mark.parametrize("nx,ny,nz", SEAM16_CASES)
def test_seam16_form_across_the_periodic_seams(nx, ny, nz, tile_y, zwall, storage):
    """The 16-bit SEAM form (34 x 15 or 34 x 12 threads, two stages; strips
    four pairs wide from the lattice's far side): a drop centred on the
    corner (0, 0) puts the interface across both seams and their corner.
    Three steps against the shared-memory hold within one rounding step of
    the storage format, and one step against the oracle fed the stored
    (rounded) state within the storage-ulp bar of the other 16-bit tests."""
    pd = base(nx, ny, nz, wall=(0, 0, zwall))
    rR, rB, u = wl.droplet(nx, ny, nz, 6.0, pd["rho_in_R"], pd["rho_in_B"],
                           velocity=(0.02, -0.01, 0.005), center=(0.5, 0.5, nz / 2.0),
                           noise=1e-3, seed=3)
    f0 = np.asarray(oracle.init(oracle.params_from(pd), rR, rB, u),
                    dtype=np.float32).astype(np.float64)
    got, diag = run(pd, f0, 3, 7, 0, storage=storage, tile_y=tile_y)
    ref_gpu, _ = run(pd, f0, 3, 2, 0, storage=storage)
    ulp = 2.0 ** -10 if storage == "f16" else 2.0 ** -7
    assert np.abs(got - ref_gpu).max() <= ulp * np.abs(ref_gpu).max()
    assert diag[5] == 0
    # one step from the stored state against the oracle
    p = lbm.make_params(storage=storage, **pd)
    p.ref_R, p.ref_B = 0.0, pd["rho_in_B"]
    lat = lbm.Lattice(p, device=DEV)
    lbm.lbm_set_fused_config(lat.ctx, tile_y, 0, 7)
    lat.set_f(torch.tensor(f0, dtype=torch.float32, device=DEV))
    s0 = lat.get_f().double().cpu().numpy()
    lat.step(1)
    s1 = lat.get_f().double().cpu().numpy()
    lat.close()
    ref = oracle.step(oracle.params_from(pd), s0, 1)
    unit = 2.0 ** -11 if storage == "f16" else 2.0 ** -8   # the stored format's ulp
    bar = unit * (1.0 + pd["rho_in_B"] * pd["alpha_B"] / np.abs(ref).max()) + 1e-5
    assert np.abs(s1 - ref).max() / np.abs(ref).max() <= bar


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_seam16_form_is_the_default_on_a_periodic_16_bit_cube(storage):
    p = lbm.make_params(storage=storage, **base(128, 128, 128))
    lat = lbm.Lattice(p, device=DEV)
    assert tuple(lbm.lbm_get_fused_config(lat.ctx))[::2] == (15, 7)
    lat.close()
