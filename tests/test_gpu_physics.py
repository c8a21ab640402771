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
import numpy as np
import pytest
import torch

from paper_1904_03618_gb300 import lbm, params as P, workloads as wl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


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


def _layered(name, improved, steps=600000, gscale=10.0):
    """(u_x profile, E_u) of the GPU step from rest."""
    import layered_channel as lc
    g0 = lc.G
    try:
        lc.G = g0 * gscale
        d, muR, muB = lc.case_params(name, improved)
        ua = lc.analytic_profile(muR, muB, lc.printed_case(name)["M"])
    finally:
        lc.G = g0
    d = {k: v for k, v in d.items() if k not in ("nx", "ny", "nz")}
    lat = lbm.Lattice(lbm.make_params(1, lc.NY, 1, **d), device=DEV,
                      stream=torch.cuda.Stream(DEV))
    lat.init_fields(*lc.initial_fields(name, from_profile=False))   # from rest
    lat.step(steps)
    _, _, uu = (t.double().cpu().numpy() for t in lat.moments())
    lat.close()
    return uu[0, 0, :, 0], lc.e_u(uu[0, 0, :, 0], ua)


def test_layered_channel_on_the_paper_lattice():
    """Sec. IV.B cases A, B and C from rest to steady state (600,000 steps)
    on the paper's lattice, read as in tests/layered_channel.py (Zou-He
    no-slip wet nodes, the smaller relaxation time 1, beta 0.7), against the
    FP64 oracle's steady profile of the same case (from the analytic
    profile, in spawned CPU workers).  Paper: improved 0.66 / 1.42 / 0.36 %,
    original 44.6 / 59.7 / 6904 %; the oracle: improved 0.449 / 1.498 /
    0.584 %, original 31.0 / 64.0 / 27.6 %.  The body force is ten times the
    printed G = 1.5e-8 (E_u does not depend on G in this Stokes regime: the
    oracle gives 0.4488 % for case A at G, 10 G and 100 G): at the printed G
    the velocities are at most 3e-4 and the FP32 steady state carries a
    rounding bias of the order of E_u itself.  Even at 10 G it shifts the
    profile by a few 1e-3 of its peak (case A: E_u 0.31 % against the
    oracle's 0.45 %), so the bar for the improved model is on the profile:
    max |u_GPU - u_oracle| <= 5e-3 max |u_oracle|; for the original model,
    whose steady state balances large spurious stresses (its profile moves
    by 1 % of its peak in FP32), E_u within 10 % of the oracle's (measured
    30.66 % against 30.97 % for case A)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import layered_channel as lc
    keys = [("A", True, 50000), ("B", True, 200000), ("C", True, 200000),
            ("A", False, 50000), ("B", False, 50000), ("C", False, 50000)]
    with cf.ProcessPoolExecutor(max_workers=len(keys),
                                mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(lc.oracle_profile, n, imp, st, 10.0) for n, imp, st in keys]
        ref = [f.result() for f in futs]
    for (name, imp, _), (u_ref, e_ref) in zip(keys, ref):
        u_gpu, e_gpu = _layered(name, imp)
        dev = np.abs(u_gpu - u_ref).max() / np.abs(u_ref).max()
        if imp:
            assert dev <= 5e-3, (name, imp, dev, e_gpu, e_ref)
        else:
            assert abs(e_gpu / e_ref - 1) < 0.10, (name, e_gpu, e_ref)
