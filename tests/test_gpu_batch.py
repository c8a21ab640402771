"""Batched contexts: many independent lattices advanced by one launch per
step, replayed through a CUDA graph.  Each case must equal the same lattice
stepped on its own within rounding: the per-cell arithmetic is the same
source, but the batched kernel is a different compiled function (case
parameters from shared memory, wall handling compiled in when any case has
walls), so the compiler's multiply-add contractions may differ by an ulp.
One case is also checked against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1904_03618_gb300 import lbm, workloads as wl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _case(nx, ny, nz, **kw):
    d = dict(nx=nx, ny=ny, nz=nz, wall=(0, 0, 0), improved=True, rho_in_R=3.0,
             rho_in_B=1.0, alpha_R=0.9, alpha_B=0.7, tau_R=0.8, tau_B=1.1, tau_e=1.0,
             tau_q=0.95, tau_pi=1.05, A_R=0.01, A_B=0.01, beta=0.7, delta=0.98,
             force=(0.0, 0.0, 0.0), gravity=(0.0, 0.0, 0.0))
    d.update(kw)
    return d


CASES = [
    _case(32, 32, 32, rho_in_R=1.0, alpha_R=1 / 3, alpha_B=1 / 3, A_R=0.0225, A_B=0.0225),
    _case(45, 17, 23, wall=(0, 0, 1), gravity=(0, 0, -1e-5)),
    _case(61, 13, 9, wall=(1, 1, 0), improved=False, force=(1e-5, 0, 0)),
    _case(1, 40, 1, wall=(0, 1, 0), rho_in_R=0.8, rho_in_B=0.1, alpha_B=0.2,
          alpha_R=1 - 0.8 * 0.1 / 0.8, force=(1e-6, 0, 0)),
    _case(20, 20, 20, rho_in_R=10.0, alpha_R=0.97, A_R=0.01125, A_B=0.01125),
]


def _fields(d, seed):
    R = max(2.0, min(d["nx"], d["ny"], d["nz"]) * 0.25)
    return wl.droplet(d["nx"], d["ny"], d["nz"], R, d["rho_in_R"], d["rho_in_B"],
                      velocity=(0.02, -0.01, 0.01), noise=1e-3, seed=seed)


def _run_single(d, steps, cfg=None, storage="f32"):
    stream = torch.cuda.Stream(DEV)
    lat = lbm.Lattice(lbm.make_params(storage=storage, **d), device=DEV, stream=stream)
    if cfg:
        lbm.lbm_set_fused_config(lat.ctx, *cfg)
    lat.init_fields(*_fields(d, 7))
    lat.step(steps)
    out = lat.get_f()
    lat.close()
    return out


@pytest.mark.parametrize("cfg", [(8, 0, 2), (8, 5, 0), (16, 7, 1)])
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_cases_equal_single_lattices(cfg, storage):
    stream = torch.cuda.Stream(DEV)
    params = [lbm.make_params(storage=storage, **d) for d in CASES]
    b = lbm.Batch(params, device=DEV, stream=stream)
    lbm.lbm_set_fused_config(b.ctx, *cfg)
    for k, d in enumerate(CASES):
        b.init_fields(k, *_fields(d, 7))
    b.step(7)   # graph path: 2 plain steps, then graph replays, then 1 plain
    for k, d in enumerate(CASES):
        got = b.get_f(k)
        ref = _run_single(d, 7, storage=storage)
        # FP32: the parity bar; FP16: an ulp of the stored deviation
        tol = 1e-5 if storage == "f32" else 2.0 ** -10
        err = (got.double() - ref.double()).abs().max() / ref.double().abs().max()
        assert err.item() <= tol, (k, err.item())
    b.close()


# every case with a 16-byte multiple x row in FP32 and 16-bit storage, so
# that the batch has tensor maps for the TMA-staged forms
TMA_CASES = [
    _case(32, 32, 32, rho_in_R=1.0, alpha_R=1 / 3, alpha_B=1 / 3, A_R=0.0225, A_B=0.0225),
    _case(44, 17, 23, wall=(0, 0, 1), gravity=(0, 0, -1e-5)),
    _case(64, 13, 9, wall=(1, 1, 0), improved=False, force=(1e-5, 0, 0)),
    _case(4, 40, 4, wall=(0, 1, 0), rho_in_R=0.8, rho_in_B=0.1, alpha_B=0.2,
          alpha_R=1 - 0.8 * 0.1 / 0.8, force=(1e-6, 0, 0)),
    _case(20, 20, 20, rho_in_R=10.0, alpha_R=0.97, A_R=0.01125, A_B=0.01125),
    _case(36, 24, 12, wall=(0, 0, 1), wetting=True, contact_angle_deg=120.0),
]


@pytest.mark.parametrize("cfg", [(8, 0, 7), (8, 5, 8), (15, 0, 7), (15, 5, 8), (15, 3, 7)])
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_tma_cases_equal_single_lattices(cfg, storage):
    """The batched TMA-staged step: tensor maps per case from a device
    table, persistent CTAs over (case, chunk, tile) items, the stage
    mbarrier phases carried across items."""
    stream = torch.cuda.Stream(DEV)
    params = [lbm.make_params(storage=storage, **d) for d in TMA_CASES]
    b = lbm.Batch(params, device=DEV, stream=stream)
    lbm.lbm_set_fused_config(b.ctx, *cfg)
    for k, d in enumerate(TMA_CASES):
        b.init_fields(k, *_fields(d, 7))
    b.step(7)
    d0 = b.diagnostics(0)
    for k, d in enumerate(TMA_CASES):
        got = b.get_f(k)
        ref = _run_single(d, 7, storage=storage)
        tol = 1e-5 if storage == "f32" else 2.0 ** -10
        err = (got.double() - ref.double()).abs().max() / ref.double().abs().max()
        assert err.item() <= tol, (k, err.item())
    assert d0[5] == 0
    b.close()


def test_batch_tma_rejected_without_maps():
    """A batch with a case whose x row is not a 16-byte multiple has no
    tensor maps: the TMA forms are refused, the others run."""
    params = [lbm.make_params(**d) for d in CASES]
    b = lbm.Batch(params, device=DEV)
    try:
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_fused_config(b.ctx, 15, 0, 7)
        lbm.lbm_set_fused_config(b.ctx, 8, 0, 2)
    finally:
        b.close()


def test_batch_case_against_oracle():
    d = CASES[1]
    b = lbm.Batch([lbm.make_params(**dd) for dd in CASES], device=DEV,
                  stream=torch.cuda.Stream(DEV))
    for k, dd in enumerate(CASES):
        b.init_fields(k, *_fields(dd, 7))
    f0 = b.get_f(1).double().cpu().numpy()
    b.step(1)
    got = b.get_f(1).double().cpu().numpy()
    b.close()
    ref = oracle.step(oracle.params_from(d), f0, 1)
    assert np.abs(got - ref).max() / np.abs(ref).max() <= 1e-5


def test_graph_replay_equals_plain_launches():
    d = CASES[1]
    outs = []
    for graphs in (True, False):
        stream = torch.cuda.Stream(DEV)
        lat = lbm.Lattice(lbm.make_params(**d), device=DEV, stream=stream)
        lbm.lbm_set_graphs(lat.ctx, graphs)
        lat.init_fields(*_fields(d, 3))
        lat.step(3)
        lat.step(10)
        lat.step(5)
        outs.append(lat.get_f())
        assert lat.diagnostics()[12] == 18
        lat.close()
    assert torch.equal(outs[0], outs[1])


def test_batch_diagnostics_and_moments_per_case():
    stream = torch.cuda.Stream(DEV)
    b = lbm.Batch([lbm.make_params(**d) for d in CASES], device=DEV, stream=stream)
    for k, d in enumerate(CASES):
        b.init_fields(k, *_fields(d, 11))
    b.step(4)
    for k, d in enumerate(CASES):
        f = b.get_f(k).double()
        diag = b.diagnostics(k)
        assert diag[0] == pytest.approx(f[0].sum().item(), rel=1e-12)
        assert diag[1] == pytest.approx(f[1].sum().item(), rel=1e-12)
        rR, rB, u = b.moments(k)
        assert torch.allclose(rR.double(), f[0].sum(0), rtol=1e-6, atol=1e-6)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_batch_get_f(b.ctx, len(CASES), torch.empty(1, device=DEV))
    assert ei.value.status == lbm.LBM_ERR_ARG
    b.close()


def test_batch_step_before_all_cases_are_initialised():
    b = lbm.Batch([lbm.make_params(**d) for d in CASES[:2]], device=DEV)
    b.init_fields(0, *_fields(CASES[0], 1))
    with pytest.raises(lbm.LbmError) as ei:
        b.step(1)
    assert ei.value.status == lbm.LBM_ERR_STATE
    b.close()


# FP32 cases periodic in x and y: the batched SEAM form (34 x 12 tile, two
# stages, the periodic seams staged by strip copies), an autotuner option
# for such batches.  Cases narrower than the tile's 32 x 10 interior in x or y (a
# tile spanning both seams of the axis) pull the far seam's sources from
# global memory.
SEAM_CASES = [
    _case(32, 32, 32, rho_in_R=1.0, alpha_R=1 / 3, alpha_B=1 / 3, A_R=0.0225, A_B=0.0225),
    _case(44, 17, 23, wall=(0, 0, 1), gravity=(0, 0, -1e-5)),
    _case(64, 13, 9, improved=False, force=(1e-5, 0, 0)),
    _case(20, 20, 20, rho_in_R=10.0, alpha_R=0.97, A_R=0.01125, A_B=0.01125),
    _case(36, 24, 12, wall=(0, 0, 1), wetting=True, contact_angle_deg=120.0),
    _case(2, 6, 5, force=(0.0, 1e-5, 0.0)),
    _case(48, 48, 16),
]


@pytest.mark.parametrize("zchunk", [0, 5, 32])
def test_batch_seam_cases_equal_single_lattices(zchunk):
    stream = torch.cuda.Stream(DEV)
    params = [lbm.make_params(**d) for d in SEAM_CASES]
    b = lbm.Batch(params, device=DEV, stream=stream)
    lbm.lbm_set_fused_config(b.ctx, 12, zchunk, 7)
    for k, d in enumerate(SEAM_CASES):
        b.init_fields(k, *_fields(d, 7))
    b.step(7)
    assert b.diagnostics(0)[5] == 0
    for k, d in enumerate(SEAM_CASES):
        got = b.get_f(k)
        ref = _run_single(d, 7)
        err = (got.double() - ref.double()).abs().max() / ref.double().abs().max()
        assert err.item() <= 1e-5, (k, err.item())
    b.close()


@pytest.mark.parametrize("k", [0, 3, 5])
def test_batch_seam_double_seam_case_against_oracle(k):
    """Cases narrower than the tile (32^3, 20^3, 2 x 6 x 5): one step of the
    batched SEAM form against the oracle."""
    b = lbm.Batch([lbm.make_params(**dd) for dd in SEAM_CASES], device=DEV,
                  stream=torch.cuda.Stream(DEV))
    lbm.lbm_set_fused_config(b.ctx, 12, 0, 7)
    for j, dd in enumerate(SEAM_CASES):
        b.init_fields(j, *_fields(dd, 7))
    f0 = b.get_f(k).double().cpu().numpy()
    b.step(1)
    got = b.get_f(k).double().cpu().numpy()
    b.close()
    ref = oracle.step(oracle.params_from(SEAM_CASES[k]), f0, 1)
    assert np.abs(got - ref).max() / np.abs(ref).max() <= 1e-5
