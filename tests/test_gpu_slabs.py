"""z-slab decomposition on the GPU (one device, several slabs in one
process: SlabsOnOneDevice): every step advances each slab's context, then
lbm_get_planes / lbm_set_planes copy each slab's two outermost own planes
into its neighbours' ghost planes.  The assembled moments must equal the
undivided lattice's: exactly with walls in z (the slabs run the same kernel
instantiation as the whole lattice), within FP32 rounding for a lattice
periodic in z (the slabs' local z walls select the walled instantiation,
whose code generation may contract other multiply-adds).  The multi-GPU
transfer itself is tested over gloo on CPU (tests/test_slabs.py)."""
import numpy as np
import pytest
import torch

from paper_1904_03618_gb300 import lbm, slabs, workloads as wl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _case(walls):
    pd = dict(nx=40, ny=36, nz=48, wall=(0, 0, 1 if walls else 0), improved=True,
              rho_in_R=3.0, rho_in_B=1.0, alpha_R=0.9, alpha_B=0.7, tau_R=0.9, tau_B=1.1,
              A_R=0.001, A_B=0.001, beta=0.7, gravity=(0.0, 0.0, -1e-5) if walls else (0, 0, 0),
              force=(0.0, 0.0, 0.0) if walls else (1e-5, 0.0, 0.0))
    if walls:
        f = wl.rayleigh_taylor(40, 36, 48, 40, 0.05, 24, 3.0, 1.0)
    else:
        f = wl.droplet(40, 36, 48, 9.0, 3.0, 1.0, velocity=(0.02, 0.01, 0.03), noise=1e-3)
    return pd, tuple(np.ascontiguousarray(a, dtype=np.float32) for a in f)


def _whole(pd, fields, storage, refs, steps):
    p = lbm.make_params(storage=storage, **pd)
    p.ref_R, p.ref_B = refs
    lat = lbm.Lattice(p, device=DEV)
    lat.init_fields(*fields)
    lat.step(steps)
    out = lat.moments()
    lat.close()
    return out


@pytest.mark.parametrize("walls", [True, False])
@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_slabs_on_one_device_equal_the_undivided_lattice(walls, world, storage):
    pd, fields = _case(walls)
    refs = (0.0, 0.0) if storage == "f32" else (3.0, 1.0) if walls else (0.0, 1.0)
    steps = 8
    ref = _whole(pd, fields, storage, refs, steps)
    s = slabs.SlabsOnOneDevice(pd, world, device=DEV, storage=storage, refs=refs)
    try:
        s.init_fields(fields)
        s.step(steps)
        got = s.moments()
    finally:
        s.close()
    for g, r in zip(got, ref):
        if walls:
            assert torch.equal(g, r)
        else:
            err = (g.double() - r.double()).abs().max().item() / r.double().abs().max().item()
            assert err < 1e-5, err


def test_plane_copies_round_trip_and_refuse_bad_ranges():
    pd, fields = _case(True)
    p = lbm.make_params(**pd)
    lat = lbm.Lattice(p, device=DEV)
    try:
        lat.init_fields(*fields)
        pb = lbm.lbm_plane_bytes(lat.ctx)
        assert pb == 19 * pd["nx"] * pd["ny"] * 8
        planes = torch.empty(3 * pb // 4, dtype=torch.int32, device=DEV)
        lbm.lbm_get_planes(lat.ctx, 10, 3, planes)
        whole = torch.empty(lbm.lbm_population_bytes(lat.ctx) // 4, dtype=torch.int32,
                            device=DEV)
        lbm.lbm_get_populations(lat.ctx, whole)
        plane_pairs = (pd["nx"] * pd["ny"] * pd["nz"] + 63) // 64 * 64
        cells = pd["nx"] * pd["ny"]
        w = whole.view(19, -1)[:, : plane_pairs * 2].reshape(19, plane_pairs, 2)
        want = w[:, 10 * cells:13 * cells].reshape(-1)
        assert torch.equal(planes, want)
        # writing them back elsewhere and reading again gives the same bytes
        lbm.lbm_set_planes(lat.ctx, 30, 3, planes)
        again = torch.empty_like(planes)
        lbm.lbm_get_planes(lat.ctx, 30, 3, again)
        torch.cuda.synchronize()
        assert torch.equal(again, planes)
        host = np.empty(3 * pb // 4, dtype=np.int32)
        lbm.lbm_get_planes(lat.ctx, 30, 3, host)
        torch.cuda.synchronize()
        assert np.array_equal(host, planes.cpu().numpy())
        for z0, n in [(-1, 2), (47, 2), (0, 0)]:
            with pytest.raises(lbm.LbmError) as ei:
                lbm.lbm_get_planes(lat.ctx, z0, n, planes)
            assert ei.value.status == lbm.LBM_ERR_ARG
    finally:
        lat.close()
