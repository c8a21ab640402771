"""Physics of the CUDA path at scales the CPU oracle cannot afford, as bands
around what the paper reports (figures only, no printed values, except the
layered channel's E_u) and what the continuum theory fixes.

  * Galilean invariance (Sec. IV.A): a drop of density ratio 3 carried by a
    uniform flow keeps its circular shape with the improved model and turns
    elliptic with the original model -- in a periodic uniform flow, and in
    the paper's own setup, dragged by two moving plates (Zou-He velocity
    nodes) on a 140 x 140 x 4 lattice.
  * Laplace law: pressure jump 2 sigma / R with sigma = 2 (A_R + A_B) / 9,
    approached as the drop is resolved better.
  * Layered two-phase channel (Sec. IV.B, Eq. 54-55) on the paper's lattice.
"""
import json
import os

import numpy as np
import pytest
import torch

from paper_1904_03618_gb300 import lbm, params as P, workloads as wl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _aspect_ratio(rR, rB, rin):
    """Principal-axis ratio of the red region (rho^N > 0) of a quasi-2D
    periodic field (1, ny, nx), centroid from circular means."""
    rn = ((rR / rin[0] - rB / rin[1]) / (rR / rin[0] + rB / rin[1]))[0]
    ny, nx = rn.shape
    ind = (rn > 0).astype(float)
    cx = (np.angle((ind.sum(0) * np.exp(2j * np.pi * np.arange(nx) / nx)).sum())
          % (2 * np.pi)) * nx / (2 * np.pi)
    cy = (np.angle((ind.sum(1) * np.exp(2j * np.pi * np.arange(ny) / ny)).sum())
          % (2 * np.pi)) * ny / (2 * np.pi)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    dx = (X - cx + nx / 2) % nx - nx / 2
    dy = (Y - cy + ny / 2) % ny - ny / 2
    m = ind.sum()
    I = np.array([[(ind * dx * dx).sum(), (ind * dx * dy).sum()],
                  [(ind * dx * dy).sum(), (ind * dy * dy).sum()]]) / m
    ev = np.linalg.eigvalsh(I)
    return np.sqrt(ev[1] / ev[0])


def _moving_drop(improved, U=0.02, n=128, steps=20000):
    # Sec. IV.A: rho_in 3 / 1, alpha 0.9 / 0.7, A = 0.01, beta = 0.5, other
    # relaxation times 1, mu_R = mu_B = 0.075 (tau_v = 1 for both fluids)
    pd = dict(wall=(0, 0, 0), improved=improved, rho_in_R=3.0, rho_in_B=1.0,
              alpha_R=0.9, alpha_B=0.7, tau_R=1.0, tau_B=1.0, A_R=0.01, A_B=0.01,
              beta=0.5)
    assert P.alpha_R_from_balance(3.0, 1.0, 0.7) == pytest.approx(0.9)
    rR, rB, u = wl.cylinder_z(n, n, 1, 30.0, 3.0, 1.0, velocity=(U, 0.0, 0.0))
    lat = lbm.Lattice(lbm.make_params(n, n, 1, **pd), device=DEV, stream=torch.cuda.Stream(DEV))
    lat.init_fields(rR, rB, u)
    lat.step(steps)
    r1, r2, _ = (t.double().cpu().numpy() for t in lat.moments())
    d = lat.diagnostics(raise_unstable=False)
    lat.close()
    return _aspect_ratio(r1, r2, (3.0, 1.0)), d


def test_galilean_invariance_improved_keeps_the_drop_round():
    a_imp, d = _moving_drop(True)
    a_orig, _ = _moving_drop(False)
    assert d[5] == 0
    assert a_imp < 1.02          # measured 1.001 - 1.008 over 20,000 steps
    assert a_orig > 1.2          # measured 1.47: the original model deforms


def test_galilean_invariance_between_moving_plates_paper_setup():
    """Sec. IV.A as printed: 140 x 140 x 4, plates in y moving at 0.02.
    Once the plates have set the whole fluid in motion (about 60,000 steps)
    the improved model's drop stays round (measured 1.005 - 1.009 from
    60,000 to 120,000 steps) and the original model's is elliptic (1.22 -
    1.23)."""
    from paper_1904_03618_gb300 import moving_droplet as md
    imp = md.run(True, steps=80000, every=80000, device=DEV)
    orig = md.run(False, steps=80000, every=80000, device=DEV)
    assert imp["nonfinite"] == 0 and orig["nonfinite"] == 0
    assert imp["rows"][-1]["aspect_ratio"] < 1.02
    assert orig["rows"][-1]["aspect_ratio"] > 1.15
    # the drop travels with the plates (80,000 steps at up to 0.02)
    moved = (imp["rows"][-1]["x_centroid"] - imp["rows"][0]["x_centroid"]) % 140
    assert moved > 1.0


@pytest.mark.parametrize("R,band", [(8.0, 0.08), (10.0, 0.05)])
def test_laplace_law_3d(R, band):
    n = 32
    pd = dict(rho_in_R=1.0, rho_in_B=1.0, alpha_R=1 / 3, alpha_B=1 / 3,
              A_R=P.A_from_sigma(0.01), A_B=P.A_from_sigma(0.01), beta=0.7)
    rR, rB, u = wl.droplet(n, n, n, R, 1.0, 1.0)
    lat = lbm.Lattice(lbm.make_params(n, n, n, **pd), device=DEV, stream=torch.cuda.Stream(DEV))
    lat.init_fields(rR, rB, u)
    lat.step(2000)
    r1, r2, uu = (t.double().cpu().numpy() for t in lat.moments())
    lat.close()
    pr = (r1 + r2) / 3.0  # p = sum_k rho_k c_s^2, alpha = 1/3
    x = np.arange(n) - (n - 1) / 2
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    rr = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    Re = (3 * r1.sum() / (4 * np.pi)) ** (1 / 3)
    dp = pr[rr < Re - 3].mean() - pr[rr > Re + 4].mean()
    assert abs(dp * Re / 2 / 0.01 - 1.0) < band
    assert np.abs(uu).max() < 1e-3   # spurious currents


def _layered(name, improved, steps=2000000):
    c = json.load(open(os.path.join(GOLD, "printed_numbers.json")))["layered_flow"]["cases"][name]
    rR, rB, aB, Mr = c["rho_in_R"], c["rho_in_B"], c["alpha_B"], c["M"]
    aR = P.alpha_R_from_balance(rR, rB, aB)
    csR, csB = P.cs2(aR), P.cs2(aB)
    if rR * csR / (rB * csB) > Mr:
        tB, muB = 1.0, rB * csB * 0.5
        muR = Mr * muB
        tR = 0.5 + muR / (rR * csR)
    else:
        tR, muR = 1.0, rR * csR * 0.5
        muB = muR / Mr
        tB = 0.5 + muB / (rB * csB)
    ny, a, b, G = 100, 25.0, 50.0, 1.5e-8
    pd = dict(wall=(0, 1, 0), improved=improved, rho_in_R=rR, rho_in_B=rB, alpha_R=aR,
              alpha_B=aB, tau_R=tR, tau_B=tB, A_R=1e-4, A_B=1e-4, beta=0.7, force=(G, 0, 0))
    y = np.arange(ny) + 0.5 - ny / 2
    A1, A2 = -G / (2 * muR), -G / (2 * muB)
    B2 = 2 * (A1 * Mr - A2) * a
    C1 = (A2 - A1) * a * a - B2 * (b - a) - A2 * b * b
    C2 = -A2 * b * b - B2 * b
    ua = np.where(np.abs(y) <= a, A1 * y * y + C1, A2 * y * y + B2 * np.abs(y) + C2)
    fR, fB, u = wl.layered(1, ny, 1, a, rR, rB)
    lat = lbm.Lattice(lbm.make_params(1, ny, 1, **pd), device=DEV, stream=torch.cuda.Stream(DEV))
    lat.init_fields(fR, fB, u)   # from rest, as a user would start
    lat.step(steps)
    _, _, uu = (t.double().cpu().numpy() for t in lat.moments())
    lat.close()
    return np.abs(uu[0, 0, :, 0] - ua).sum() / np.abs(ua).sum()


def test_layered_channel_on_the_paper_lattice():
    """Sec. IV.B cases A and B at steady state (paper: improved 0.66 % /
    1.42 %, original 44.6 % / 59.7 %), from rest, 2,000,000 steps (case B's
    slowest mode decays by e every ~220,000 steps).  tau and beta are not
    printed (larger relaxation time 1, beta 0.7), hence bands."""
    eA, eB = _layered("A", True), _layered("B", True)
    assert eA < 0.05 and eB < 0.02
    assert _layered("A", False) > 0.20 and _layered("B", False) > 0.50
