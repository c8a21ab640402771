"""lbm_step_noalloc: the allocation-free step entry point.

It exists for callers that cannot call cudaMalloc (device memory fixed at
start-up, embedders owning all buffers).
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone in a fresh
process.  The checks: two calls in a row, each compared with the context
API (lbm_set_f, lbm_step, lbm_get_f) on the same input, and with the FP64
oracle, within the FP32 parity bar used by the other tests (relative
L-infinity 1e-5).
"""
import numpy as np
import pytest
import torch

from paper_1904_03618_gb300 import lbm, workloads as wl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _params(nx, ny, nz, **kw):
    d = dict(wall=(0, 0, 1), improved=True, rho_in_R=3.0, rho_in_B=1.0, alpha_R=0.9,
             alpha_B=0.7, tau_R=0.8, tau_B=1.1, tau_e=1.0, tau_q=0.95, tau_pi=1.05,
             A_R=0.01, A_B=0.01, beta=0.7, delta=0.98, force=(2e-5, 0.0, 0.0),
             gravity=(0.0, 0.0, -1e-5))
    d.update(kw)
    return lbm.make_params(nx, ny, nz, **d)


def _initial_state(params, nx, ny, nz):
    rR, rB, u = wl.droplet(nx, ny, nz, 5.0, 3.0, 1.0, velocity=(0.02, 0.01, 0.0),
                           noise=1e-3, seed=0)
    lat = lbm.Lattice(params, device=DEV)
    lat.init_fields(rR, rB, u)
    f0 = lat.get_f()
    lat.close()
    return f0


def _rel_linf(a, b):
    return (a.double() - b.double()).abs().max().item() / b.double().abs().max().item()


@pytest.mark.parametrize("wall", [(0, 0, 1), (0, 0, 0), (1, 1, 1)])
def test_noalloc_matches_context_api_on_two_consecutive_calls(wall):
    nx, ny, nz = 37, 21, 13
    params = _params(nx, ny, nz, wall=wall)
    f0 = _initial_state(params, nx, ny, nz)

    lat = lbm.Lattice(params, device=DEV)
    lat.set_f(f0)
    lat.step(1)
    ref1 = lat.get_f()
    lat.step(1)
    ref2 = lat.get_f()
    lat.close()

    stream = torch.cuda.current_stream(DEV)
    f1 = torch.empty_like(f0)
    f2 = torch.empty_like(f0)
    lbm.lbm_step_noalloc(params, f0, f1, stream.cuda_stream)
    lbm.lbm_step_noalloc(params, f1, f2, stream.cuda_stream)
    stream.synchronize()
    assert _rel_linf(f1, ref1) <= 1e-5
    assert _rel_linf(f2, ref2) <= 1e-5


@pytest.mark.parametrize("wall", [(0, 0, 1), (1, 1, 1)])
def test_noalloc_matches_the_oracle_on_two_consecutive_calls(wall):
    """The same two calls checked directly against the FP64 oracle stepped
    from the same (float32-rounded) state: per-step relative L-infinity
    1e-5."""
    import oracle
    nx, ny, nz = 29, 18, 11
    params = _params(nx, ny, nz, wall=wall)
    f0 = _initial_state(params, nx, ny, nz)
    pd = dict(nx=nx, ny=ny, nz=nz, wall=wall, improved=True, rho_in_R=3.0, rho_in_B=1.0,
              alpha_R=0.9, alpha_B=0.7, tau_R=0.8, tau_B=1.1, tau_e=1.0, tau_q=0.95,
              tau_pi=1.05, A_R=0.01, A_B=0.01, beta=0.7, delta=0.98,
              force=(2e-5, 0.0, 0.0), gravity=(0.0, 0.0, -1e-5))
    p = oracle.params_from(pd)
    fo0 = f0.double().cpu().numpy()
    fo1 = oracle.step(p, fo0, 1)
    fo2 = oracle.step(p, fo1, 1)
    stream = torch.cuda.current_stream(DEV)
    f1 = torch.empty_like(f0)
    f2 = torch.empty_like(f0)
    lbm.lbm_step_noalloc(params, f0, f1, stream.cuda_stream)
    lbm.lbm_step_noalloc(params, f1, f2, stream.cuda_stream)
    stream.synchronize()
    for got, ref in ((f1, fo1), (f2, fo2)):
        g = got.double().cpu().numpy().reshape(ref.shape)
        assert np.abs(g - ref).max() / np.abs(ref).max() <= 1e-5


def test_noalloc_rejects_lattices_beyond_its_scratch():
    params = _params(65, 64, 64, wall=(0, 0, 0))   # 266,240 cells > 262,144
    f = torch.zeros(1, device=DEV)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_step_noalloc(params, f, f)
    assert ei.value.status == lbm.LBM_ERR_ARG
    assert "262144" in str(ei.value)


def test_noalloc_rejects_overlapping_arrays():
    params = _params(8, 8, 8)
    f = torch.zeros(2 * 38 * 512, device=DEV)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_step_noalloc(params, f, f[100:])
    assert ei.value.status == lbm.LBM_ERR_ARG
