"""lbm_step_monitored: every step reports the diagnostics of the state it
reads.  On the seam forms' default tiles the step kernel sums them itself
(FP32 per warp, FP64 across warps and CTAs); elsewhere the diagnostics pass
runs before each step.  Checked against lbm_diagnostics of the same states
taken by a twin context that steps one step at a time, and the monitored
steps must leave the same populations as plain ones."""
import numpy as np
import pytest
import torch

from paper_1904_03618_gb300 import lbm, workloads as wl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
BASE = dict(rho_in_R=3.0, rho_in_B=1.0, alpha_R=0.9, alpha_B=0.7, tau_R=0.8, tau_B=1.1,
            A_R=0.01, A_B=0.01, beta=0.7, force=(2e-5, 0.0, 0.0))

# name: (nx, ny, nz, keywords, whether the in-kernel form applies)
CASES = {
    "fp32_seam": (64, 48, 40, {}, True),
    "fp32_seam_zwalls_gravity": (64, 30, 24, dict(wall=(0, 0, 1), gravity=(0.0, 0.0, -1e-5)),
                                 True),
    "f16_seam": (68, 32, 20, dict(storage="f16"), True),
    "bf16_seam_zwalls": (68, 30, 18, dict(storage="bf16", wall=(0, 0, 1)), True),
    "fp32_xwalls_fallback": (40, 20, 10, dict(wall=(1, 0, 0)), False),
    "two_pass_fallback": (24, 18, 10, dict(kernel="two_pass"), False),
}


def _lattice(nx, ny, nz, kw):
    kw = dict(BASE, **kw)
    p = lbm.make_params(nx, ny, nz, **kw)
    if kw.get("storage", "f32") != "f32":
        p.ref_R, p.ref_B = 0.0, 1.0
    lat = lbm.Lattice(p, device=DEV)
    lat.init_fields(*wl.droplet(nx, ny, nz, 0.3 * min(nx, ny, nz), 3.0, 1.0,
                                velocity=(0.03, 0.01, 0.0), noise=1e-3, seed=nx))
    return lat


@pytest.mark.parametrize("name", sorted(CASES))
def test_monitored_steps_report_the_states_they_read(name):
    nx, ny, nz, kw, fused = CASES[name]
    n = 5
    a = _lattice(nx, ny, nz, kw)
    b = _lattice(nx, ny, nz, kw)
    try:
        out = torch.zeros((n, 16), dtype=torch.float64).pin_memory()
        lbm.lbm_step_monitored(a.ctx, n, out)
        lbm.lbm_sync(a.ctx)
        got = out.numpy()
        for k in range(n):
            ref = b.diagnostics(raise_unstable=False)
            g = got[k]
            assert g[12] == ref[12] == k
            for s in (5, 6, 8, 13, 14):                   # counts and the error word
                assert g[s] == ref[s], (k, s, g[s], ref[s])
            mass = abs(ref[0]) + abs(ref[1])
            tol = 2e-6 if fused else 1e-12
            assert abs(g[0] - ref[0]) <= tol * abs(ref[0])
            assert abs(g[1] - ref[1]) <= tol * abs(ref[1])
            for s in (2, 3, 4):                            # momentum
                assert abs(g[s] - ref[s]) <= tol * mass, (k, s, g[s], ref[s])
            assert abs(g[7] - ref[7]) <= 1e-6 * ref[7]      # max |u|
            for s in (9, 10, 11):                           # red-mass centroid
                assert abs(g[s] - ref[s]) <= 10 * tol * max(nx, ny, nz), (k, s, g[s], ref[s])
            b.step(1)
        # the monitored form is a kernel of its own: where the compiler
        # contracts an operation differently its FP32 results differ in the
        # last bits (a few ulp after five steps; a 16-bit store can then
        # round the other way: one storage ulp)
        fa = a.get_f().double().cpu().numpy()
        fb = b.get_f().double().cpu().numpy()
        storage = kw.get("storage", "f32")
        ulp = {"f32": 1e-6, "f16": 2.0 ** -10, "bf16": 2.0 ** -7}[storage]
        assert np.abs(fa - fb).max() <= ulp * np.abs(fb).max()
    finally:
        a.close()
        b.close()


def test_monitored_output_in_device_memory_and_batches_refused():
    a = _lattice(64, 48, 40, {})
    try:
        out = torch.zeros((3, 16), dtype=torch.float64, device=DEV)
        lbm.lbm_step_monitored(a.ctx, 3, out)
        lbm.lbm_sync(a.ctx)
        assert out[:, 12].cpu().tolist() == [0.0, 1.0, 2.0]
        assert float(out[:, 0].min()) > 0.0
    finally:
        a.close()
    ps = [lbm.make_params(32, 32, 32, **BASE) for _ in range(2)]
    bt = lbm.Batch(ps, device=DEV)
    try:
        for k in range(2):
            bt.init_fields(k, *wl.droplet(32, 32, 32, 8.0, 3.0, 1.0))
        out = torch.zeros((1, 16), dtype=torch.float64, device=DEV)
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_step_monitored(bt.ctx, 1, out)
        assert ei.value.status == lbm.LBM_ERR_ARG
    finally:
        bt.close()
