"""The stated workloads of the moving-droplet configuration on the GPU, at
their full sizes and step counts.

  * Layered two-phase channel on a 4 x 128 x 4 lattice, halfway bounce-back
    walls in y (the walls half a cell outside the first and last row),
    body force 1e-6 along x, viscosity ratios M = mu_R / mu_B = 1, 10, 100:
    equal densities (alpha 1/3 for both, so the improved and the original
    equilibria coincide and the test is of the collision, the forcing, the
    walls and the viscosity interpolation of Eq. 52), red where |y_j| <= 32,
    the smaller relaxation time 1 (tau_B = 1, tau_R = 1/2 + M / 2), compared
    with Eq. 54-55 (a = 32, b = 64).  The FP64 oracle, from the analytic
    profile to steady state (100,000 steps on 1 x 128 x 1), gives E_u =
    3.05e-5, 0.665 % and 0.933 %; the GPU, from rest (200,000 steps), must
    land within 10 % of the oracle for M = 10 and 100, and below 3e-4 for
    M = 1 (FP32 steady-state rounding).
  * The 128^3 periodic moving sphere (R = 20, U = (0.05, 0, 0), density
    ratios 1 and 10, viscosity ratio 1, sigma = 0.005, 20,000 steps,
    paper_1904_03618_gb300/moving_droplet.py): the drop translates with the
    flow and stays spherical with the improved model.
"""
import numpy as np
import pytest
import torch

from paper_1904_03618_gb300 import lbm, workloads as wl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _layered_128(M, steps=200000):
    ny, a, b, G = 128, 32.0, 64.0, 1e-6
    tB, tR = 1.0, 0.5 + 0.5 * M
    mu_B, mu_R = (tB - 0.5) / 3.0, (tR - 0.5) / 3.0
    y = np.arange(ny) + 0.5 - ny / 2
    A1, A2 = -G / (2 * mu_R), -G / (2 * mu_B)
    B2 = 2 * (A1 * M - A2) * a
    C1 = (A2 - A1) * a * a - B2 * (b - a) - A2 * b * b
    C2 = -A2 * b * b - B2 * b
    ua = np.where(np.abs(y) <= a, A1 * y * y + C1, A2 * y * y + B2 * np.abs(y) + C2)
    p = lbm.make_params(4, ny, 4, wall=(0, 1, 0), improved=True, rho_in_R=1.0, rho_in_B=1.0,
                        alpha_R=1 / 3, alpha_B=1 / 3, tau_R=tR, tau_B=tB, A_R=1e-4, A_B=1e-4,
                        beta=0.7, force=(G, 0.0, 0.0))
    lat = lbm.Lattice(p, device=DEV, stream=torch.cuda.Stream(DEV))
    lat.init_fields(*wl.layered(4, ny, 4, a, 1.0, 1.0))
    lat.step(steps)
    _, _, u = (t.double().cpu().numpy() for t in lat.moments())
    d = lat.diagnostics(raise_unstable=False)
    lat.close()
    assert d[5] == 0
    ux = u[0, 1, :, 2]
    assert np.abs(u[0] - ux[None, :, None]).max() <= 1e-6 * np.abs(ux).max()  # uniform in x, z
    return np.abs(ux - ua).sum() / np.abs(ua).sum()


@pytest.mark.parametrize("M,oracle_eu", [(10.0, 0.006646), (100.0, 0.009328)])
def test_layered_channel_128_viscosity_ratios(M, oracle_eu):
    e = _layered_128(M)
    assert abs(e / oracle_eu - 1) < 0.10, (M, e, oracle_eu)


def test_layered_channel_128_equal_viscosity():
    assert _layered_128(1.0) < 3e-4


def test_moving_sphere_128_density_ratio_1():
    """Ratio 1 (alpha 1/3 for both: the two models coincide): after 20,000
    steps (1000 cells travelled) the axis ratio stays below 1.01 (measured
    1.0009) and the centroid within 3 cells of x0 + U t (1.78)."""
    from paper_1904_03618_gb300 import moving_droplet as md
    r = md.run_sphere(1, True, steps=20000, every=10000, device=DEV)
    last = r["rows"][-1]
    assert last["nonfinite"] == 0
    assert max(row["axis_ratio"] for row in r["rows"]) < 1.01
    assert abs(last["centroid_lag"]) < 3.0


def test_moving_sphere_128_density_ratio_10_improved_against_original():
    """Ratio 10 (alpha 0.97 / 0.7), U = 0.05 (Mach 0.4 in the drop, whose
    (c_s)^2 is 0.015): the improved model's drop stays near-spherical
    (largest over the records of the axis ratio 1.066, 1.050 after 20,000
    steps) and lags the flow by 15 cells over 1000; the original model's
    turns into an ellipsoid (axis ratio up to 1.68) and lags by tens of
    cells.  Bars: improved below 1.1 and a lag below 20 cells, original
    above 1.3."""
    from paper_1904_03618_gb300 import moving_droplet as md
    imp = md.run_sphere(10, True, steps=20000, every=5000, device=DEV)
    orig = md.run_sphere(10, False, steps=20000, every=5000, device=DEV)
    assert imp["rows"][-1]["nonfinite"] == 0 and orig["rows"][-1]["nonfinite"] == 0
    assert max(row["axis_ratio"] for row in imp["rows"]) < 1.1
    assert abs(imp["rows"][-1]["centroid_lag"]) < 20.0
    assert max(row["axis_ratio"] for row in orig["rows"]) > 1.3
    assert abs(imp["rows"][-1]["red_mass_rel_change"]) < 1e-3
