"""Pins of the FP64 oracle's full step (no GPU needed).

  * two independent restatements agree: the C oracle (moment space, Eq. 41)
    and the numpy one (velocity space, Eq. 40 and 53 with dense Lambda);
  * conservation laws the method fixes exactly (per-colour mass, momentum
    balance F per cell per step);
  * special cases that reduce to textbook results (BGK with tau = 1; exact
    Poiseuille with halfway bounce-back at the two-relaxation-time "magic"
    parameter);
  * the paper's own experiments, as bands: the layered two-phase channel
    (Sec. IV.B, Eq. 54-55) and the Laplace law for the surface tension
    sigma = 2 (A_R + A_B) / 9 (Sec. III.B).
"""
import json
import os

import numpy as np
import pytest

import oracle
import oracle.naive as naive
from paper_1904_03618_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")
E = naive.E


def _pd(nx, ny, nz, **kw):
    d = dict(nx=nx, ny=ny, nz=nz, wall=(0, 0, 0), improved=True, rho_in_R=3.0,
             rho_in_B=1.0, alpha_R=0.9, alpha_B=0.7, tau_R=0.8, tau_B=1.2,
             tau_e=1.1, tau_q=0.9, tau_pi=1.3, A_R=0.01, A_B=0.02, beta=0.5,
             delta=0.98, force=(1e-3, 2e-4, -3e-4), gravity=(0, 1e-4, 2e-4))
    d.update(kw)
    return d


@pytest.mark.parametrize("wall", [(0, 0, 0), (0, 1, 0), (1, 0, 1), (1, 1, 1)])
@pytest.mark.parametrize("improved", [True, False])
def test_c_oracle_matches_numpy_restatement(wall, improved):
    pd = _pd(5, 6, 4, wall=wall, improved=improved)
    p = oracle.params_from(pd)
    rR, rB, u = wl.random_fields(5, 6, 4, seed=11)
    f = oracle.init(p, rR, rB, u)
    f = f * (1 + 0.05 * np.random.default_rng(5).uniform(-1, 1, f.shape))
    a = oracle.step(p, f, 3)
    b = naive.step(pd, f, 3)
    assert np.abs(a - b).max() < 1e-13


def test_c_oracle_matches_numpy_on_far_from_equilibrium_state():
    pd = _pd(4, 3, 5, wall=(0, 0, 1))
    p = oracle.params_from(pd)
    f = wl.random_populations(4, 3, 5, seed=2)
    assert np.abs(oracle.step(p, f, 2) - naive.step(pd, f, 2)).max() < 1e-13


@pytest.mark.parametrize("wall", [(0, 0, 0), (1, 1, 1)])
def test_per_colour_mass_is_conserved_exactly(wall):
    pd = _pd(10, 9, 8, wall=wall, force=(0, 0, 0), gravity=(0, 0, 0))
    p = oracle.params_from(pd)
    rR, rB, u = wl.droplet(10, 9, 8, 3.0, 3.0, 1.0, velocity=(0.02, 0, 0),
                           noise=1e-2, seed=3)
    f = oracle.init(p, rR, rB, u)
    g = oracle.step(p, f, 30)
    for k in range(2):
        assert abs(g[k].sum() - f[k].sum()) / f[k].sum() < 1e-13


def test_momentum_balance_under_body_force():
    """Periodic lattice: each step adds F per cell to sum_x sum_i e_i f_i,
    with F = force + rho g and the total mass fixed."""
    pd = _pd(6, 5, 7)
    p = oracle.params_from(pd)
    rR, rB, u = wl.droplet(6, 5, 7, 2.0, 3.0, 1.0, noise=1e-2, seed=4)
    f = oracle.init(p, rR, rB, u)
    n = 25
    g = oracle.step(p, f, n)
    j0 = np.einsum("ia,kizyx->a", E, f)
    j1 = np.einsum("ia,kizyx->a", E, g)
    mass = f.sum()
    N = 6 * 5 * 7
    expect = n * (np.array(pd["force"]) * N + np.array(pd["gravity"]) * mass)
    assert np.allclose(j1 - j0, expect, rtol=0, atol=1e-13)


def test_single_phase_bgk_tau_one_is_textbook_streaming_of_equilibrium():
    """A = beta = 0, no blue fluid, alpha = 1/3 and every rate 1 make the
    step f_i(x + e_i, t + 1) = f_i^eq(rho, u)(x) with the textbook D3Q19
    equilibrium rho omega_i (1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u^2)."""
    nx, ny, nz = 4, 5, 3
    pd = _pd(nx, ny, nz, alpha_R=1 / 3, alpha_B=1 / 3, tau_R=1, tau_B=1, tau_e=1,
             tau_q=1, tau_pi=1, A_R=0, A_B=0, beta=0, force=(0, 0, 0),
             gravity=(0, 0, 0), rho_in_R=1.0, rho_in_B=1.0)
    p = oracle.params_from(pd)
    f = wl.random_populations(nx, ny, nz, seed=9)
    f[1] = 0.0
    g = oracle.step(p, f, 1)
    rho = f[0].sum(axis=0)
    u = np.einsum("ia,izyx->azyx", E, f[0]) / rho
    w = naive.W
    for i in range(19):
        eu = np.einsum("a,azyx->zyx", E[i], u)
        feq = rho * w[i] * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * (u ** 2).sum(0))
        moved = np.roll(feq, shift=(int(E[i, 2]), int(E[i, 1]), int(E[i, 0])),
                        axis=(0, 1, 2))
        assert np.allclose(g[0, i], moved, atol=1e-15)
    assert np.all(g[1] == 0.0)


# ---- BGK variant with the correction term (Eq. 20) -------------------------

@pytest.mark.parametrize("wall", [(0, 0, 0), (1, 0, 1)])
@pytest.mark.parametrize("improved", [True, False])
def test_bgk_equals_mrt_with_every_rate_equal(wall, improved):
    """The paper: Eq. 40 with Lambda = I / tau is Eq. 20, and Eq. 53 the
    perturbation divided by tau.  The C oracle's BGK branch (velocity space,
    no M, S or Lambda in the relaxation) against its MRT branch (moment
    space) with tau_e = tau_q = tau_pi = tau_R = tau_B: same total f*, so the
    same step, with force, gravity, surface tension and walls."""
    tau = 0.87
    pd = _pd(5, 6, 4, wall=wall, improved=improved, tau_R=tau, tau_B=tau, tau_e=tau,
             tau_q=tau, tau_pi=tau)
    rR, rB, u = wl.random_fields(5, 6, 4, seed=3)
    p_mrt = oracle.params_from(pd)
    f = oracle.init(p_mrt, rR, rB, u)
    f = f * (1 + 0.05 * np.random.default_rng(8).uniform(-1, 1, f.shape))
    a = oracle.step(p_mrt, f, 3)
    b = oracle.step(oracle.params_from(dict(pd, collision="bgk")), f, 3)
    assert np.abs(a - b).max() < 1e-13
    # and the rates do matter: a different tau_q changes the MRT step
    c = oracle.step(oracle.params_from(dict(pd, tau_q=1.2)), f, 3)
    assert np.abs(a - c).max() > 1e-6


@pytest.mark.parametrize("wall", [(0, 0, 0), (0, 1, 1), (1, 1, 1)])
def test_bgk_c_oracle_matches_numpy_restatement(wall):
    """Variable tau_v (Eq. 52 across the interface): the C branch against
    the numpy one with Lambda = I / tau_v per cell."""
    pd = _pd(5, 4, 6, wall=wall, collision="bgk")
    p = oracle.params_from(pd)
    rR, rB, u = wl.random_fields(5, 4, 6, seed=21)
    f = oracle.init(p, rR, rB, u)
    f = f * (1 + 0.05 * np.random.default_rng(6).uniform(-1, 1, f.shape))
    assert np.abs(oracle.step(p, f, 3) - naive.step(pd, f, 3)).max() < 1e-13


def test_bgk_tau_one_is_textbook_streaming_of_equilibrium():
    """The BGK branch alone, at tau = 1 with one colour and alpha = 1/3:
    f_i(x + e_i, t + 1) = rho omega_i (1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u^2)."""
    nx, ny, nz = 4, 3, 5
    pd = _pd(nx, ny, nz, alpha_R=1 / 3, alpha_B=1 / 3, tau_R=1, tau_B=1, A_R=0, A_B=0,
             beta=0, force=(0, 0, 0), gravity=(0, 0, 0), rho_in_R=1.0, rho_in_B=1.0,
             collision="bgk")
    f = wl.random_populations(nx, ny, nz, seed=12)
    f[1] = 0.0
    g = oracle.step(oracle.params_from(pd), f, 1)
    rho = f[0].sum(axis=0)
    u = np.einsum("ia,izyx->azyx", E, f[0]) / rho
    for i in range(19):
        eu = np.einsum("a,azyx->zyx", E[i], u)
        feq = rho * naive.W[i] * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * (u ** 2).sum(0))
        moved = np.roll(feq, shift=(int(E[i, 2]), int(E[i, 1]), int(E[i, 0])),
                        axis=(0, 1, 2))
        assert np.allclose(g[0, i], moved, atol=1e-15)


# ---- moving plates: Zou-He velocity nodes (Sec. IV.A) -----------------------

PLATES = ((0.03, 0.01, -0.02), (-0.01, -0.005, 0.02))   # low / high plate of the axis


def _plates_pd(ax, **kw):
    wall = [0, 0, 0]
    wall[ax] = 2
    return _pd(5, 6, 4, wall=tuple(wall), wall_u=PLATES, **kw)


@pytest.mark.parametrize("ax", [0, 1, 2])
@pytest.mark.parametrize("impl", ["c", "numpy"])
def test_zou_he_nodes_carry_the_plate_velocity(ax, impl):
    """The scheme's defining property: at every node of a plate and for each
    colour, sum_i e_i f_i^k = rho_k u_w with rho_k = sum_i f_i^k (normal and
    tangential components, inflow through the plate included)."""
    pd = _plates_pd(ax)
    p = oracle.params_from(pd)
    rR, rB, u = wl.random_fields(5, 6, 4, seed=31)
    f = oracle.init(p, rR, rB, u)
    g = oracle.step(p, f, 2) if impl == "c" else naive.step(pd, f, 2)
    for side in range(2):
        face = [slice(None)] * 3
        face[2 - ax] = 0 if side == 0 else g.shape[2 + 2 - ax] - 1
        for k in range(2):
            fk = g[(k, slice(None)) + tuple(face)]
            rho = fk.sum(axis=0)
            j = np.einsum("ia,i...->a...", E, fk)
            want = rho[None] * np.asarray(PLATES[side])[(slice(None),) + (None,) * rho.ndim]
            assert np.abs(j - want).max() < 1e-14


@pytest.mark.parametrize("ax", [0, 1, 2])
def test_zou_he_c_oracle_matches_numpy_restatement(ax):
    """Closed form (C) against the linear-system statement (numpy)."""
    pd = _plates_pd(ax)
    p = oracle.params_from(pd)
    rR, rB, u = wl.random_fields(5, 6, 4, seed=32)
    f = oracle.init(p, rR, rB, u)
    f = f * (1 + 0.05 * np.random.default_rng(4).uniform(-1, 1, f.shape))
    assert np.abs(oracle.step(p, f, 3) - naive.step(pd, f, 3)).max() < 1e-13


def _couette(U, tau, collision="mrt", ny=17, steps=6000):
    pd = _pd(1, ny, 1, wall=(0, 2, 0), wall_u=((-U, 0, 0), (U, 0, 0)), alpha_R=1 / 3,
             alpha_B=1 / 3, tau_R=tau, tau_B=tau, tau_e=1, tau_q=1, tau_pi=1, A_R=0,
             A_B=0, beta=0, force=(0, 0, 0), gravity=(0, 0, 0), rho_in_R=1.0,
             rho_in_B=1.0, collision=collision)
    p = oracle.params_from(pd)
    rR = np.ones((1, ny, 1))
    f = oracle.init(p, rR, np.zeros_like(rR), np.zeros((3, 1, ny, 1)))
    g = oracle.step(p, f, steps)
    j = np.einsum("ia,kizyx->azyx", E, g)
    ux = j[0] / g.sum(axis=(0, 1))
    exact = U * (2 * np.arange(ny) / (ny - 1) - 1)
    return np.abs(ux[0, :, 0] - exact).max(), np.abs(j[1:]).max(), abs(g.sum() - f.sum()) / f.sum()


@pytest.mark.parametrize("collision", ["mrt", "bgk"])
def test_couette_flow_between_moving_plates_is_linear(collision):
    """Single phase between plates moving at -U and +U (the other axes
    periodic), every rate 1: the steady velocity is exactly linear through
    the plate nodes, u_x(y) = U (2 y / (ny - 1) - 1), v = w = 0, and no mass
    crosses the plates."""
    err, cross, dm = _couette(0.02, 1.0, collision)
    assert err < 1e-14 and cross < 1e-14 and dm < 1e-13


def test_couette_deviation_away_from_tau_one_is_third_order_in_u():
    """At tau_v = 0.8 the steady profile departs from the line by the D3Q19
    equilibrium's O(u^3) error, not by a boundary error: halving U divides
    the deviation by 8."""
    e1, _, _ = _couette(0.02, 0.8)
    e2, _, _ = _couette(0.01, 0.8)
    assert e1 < 1e-5 * 0.02
    assert 7.5 < e1 / e2 < 8.5


def test_poiseuille_is_exact_at_the_trt_magic_parameter():
    """Single phase, halfway bounce-back walls at y = -1/2 and ny - 1/2,
    uniform force G: with (tau_v - 1/2)(tau_q - 1/2) = 3/16 and
    tau_e = tau_pi = tau_v the steady profile is the exact parabola
    u_x = G / (2 mu) (b^2 - y^2), mu = rho (tau_v - 1/2) / 3, b = ny / 2.
    This pins the collision, the forcing (u shift and (I - S/2) F) and the
    bounce-back together."""
    ny, G, tv = 12, 1e-5, 0.9
    tq = 0.5 + (3 / 16) / (tv - 0.5)
    pd = _pd(1, ny, 1, wall=(0, 1, 0), alpha_R=1 / 3, alpha_B=1 / 3, tau_R=tv,
             tau_B=tv, tau_e=tv, tau_pi=tv, tau_q=tq, A_R=0, A_B=0, beta=0,
             force=(G, 0, 0), gravity=(0, 0, 0), rho_in_R=1.0, rho_in_B=1.0)
    p = oracle.params_from(pd)
    rR = np.ones((1, ny, 1))
    rB = np.zeros((1, ny, 1))
    f = oracle.init(p, rR, rB, np.zeros((3, 1, ny, 1)))
    f = oracle.step(p, f, 12000)
    _, _, u = oracle.moments(p, f)
    y = np.arange(ny) + 0.5 - ny / 2
    ua = G / (2 * (tv - 0.5) / 3) * ((ny / 2) ** 2 - y ** 2)
    assert np.abs(u[0, 0, :, 0] - ua).max() / ua.max() < 1e-10
    assert np.abs(u[1:]).max() < 1e-14


def _layered_case(name, improved, eq18_coef=oracle.EQ18_COEF, steps=50000):
    c = json.load(open(os.path.join(GOLD, "printed_numbers.json")))["layered_flow"]["cases"][name]
    rR, rB, aB, Mr = c["rho_in_R"], c["rho_in_B"], c["alpha_B"], c["M"]
    aR = oracle.alpha_R_from_balance(rR, rB, aB)
    csR, csB = oracle.cs2(aR), oracle.cs2(aB)
    # The paper gives only M = mu_R / mu_B: the larger relaxation time is 1.
    if rR * csR * 0.5 / (rB * csB * 0.5) > Mr:
        tB = 1.0
        muB = rB * csB * 0.5
        muR = Mr * muB
        tR = 0.5 + muR / (rR * csR)
    else:
        tR = 1.0
        muR = rR * csR * 0.5
        muB = muR / Mr
        tB = 0.5 + muB / (rB * csB)
    ny, a, b, G = 100, 25.0, 50.0, 1.5e-8
    pd = _pd(1, ny, 1, wall=(0, 1, 0), improved=improved, rho_in_R=rR, rho_in_B=rB,
             alpha_R=aR, alpha_B=aB, tau_R=tR, tau_B=tB, tau_e=1, tau_q=1, tau_pi=1,
             A_R=1e-4, A_B=1e-4, beta=0.7, force=(G, 0, 0), gravity=(0, 0, 0),
             eq18_coef=eq18_coef)
    p = oracle.params_from(pd)
    y = np.arange(ny) + 0.5 - ny / 2
    A1, A2 = -G / (2 * muR), -G / (2 * muB)
    B2 = 2 * (A1 * Mr - A2) * a
    C1 = (A2 - A1) * a * a - B2 * (b - a) - A2 * b * b
    C2 = -A2 * b * b - B2 * b
    ua = np.where(np.abs(y) <= a, A1 * y * y + C1, A2 * y * y + B2 * np.abs(y) + C2)  # Eq. 54-55
    rho_R, rho_B, u = wl.layered(1, ny, 1, a, rR, rB)
    u[0] = ua[None, :, None]  # start from the analytic profile to converge fast
    f = oracle.step(p, oracle.init(p, rho_R, rho_B, u), steps)
    _, _, uu = oracle.moments(p, f)
    return np.abs(uu[0, 0, :, 0] - ua).sum() / np.abs(ua).sum()


@pytest.mark.slow
def test_layered_channel_improved_model_is_accurate_and_original_is_not():
    """Sec. IV.B: the improved model follows the analytic profile (paper:
    E_u = 0.66 % and 1.42 % for cases A and B) while the original model is
    far off (44.6 % and 59.7 %).  Started from the analytic profile and
    measured after 50,000 steps (case A is at steady state by then; case B's
    slowest mode is still decaying -- the GPU test runs it to steady state).
    The paper leaves tau and beta unstated, so this is a band: improved below
    5 % and 1.5 %, original above 20 % and 50 %, and the Eq. 18 coefficient
    as printed (3/2) clearly worse than 3."""
    eA = _layered_case("A", True)
    eB = _layered_case("B", True)
    assert eA < 0.05 and eB < 0.015
    assert _layered_case("A", False) > 0.20
    assert _layered_case("B", False) > 0.50
    assert _layered_case("A", True, eq18_coef=oracle.EQ18_COEF_PRINTED) > 3 * eA


@pytest.mark.slow
def test_laplace_law_static_droplet():
    """32^3 periodic, R = 8, A_R = A_B = 0.0225 (sigma = 0.01), beta = 0.7,
    500 steps: the pressure jump gives sigma within 10 %, and the mass of
    each colour is unchanged to round-off."""
    n, R, A = 32, 8.0, 0.0225
    pd = _pd(n, n, n, rho_in_R=1.0, rho_in_B=1.0, alpha_R=1 / 3, alpha_B=1 / 3,
             tau_R=1, tau_B=1, tau_e=1, tau_q=1, tau_pi=1, A_R=A, A_B=A, beta=0.7,
             force=(0, 0, 0), gravity=(0, 0, 0))
    p = oracle.params_from(pd)
    rR, rB, u = wl.droplet(n, n, n, R, 1.0, 1.0)
    f0 = oracle.init(p, rR, rB, u)
    f = oracle.step(p, f0, 500)
    r1, r2, _ = oracle.moments(p, f)
    pr = (r1 + r2) / 3.0  # p = sum_k rho_k c_s^2 with alpha = 1/3
    x = np.arange(n) - (n - 1) / 2
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    rr = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    Re = (3 * r1.sum() / (4 * np.pi)) ** (1 / 3)
    dp = pr[rr < Re - 3].mean() - pr[rr > Re + 4].mean()
    sigma = oracle.surface_tension(A, A)
    assert abs(dp * Re / 2 / sigma - 1) < 0.10
    for k in range(2):
        assert abs(f[k].sum() - f0[k].sum()) / f0[k].sum() < 1e-12


def test_wetting_switch_is_inert_without_walls():
    """Periodic lattice: no wall-adjacent cells, so the wetting rule changes
    nothing."""
    pd = _pd(6, 5, 7)
    rR, rB, u = wl.droplet(6, 5, 7, 2.0, 3.0, 1.0, noise=1e-2, seed=4)
    p0 = oracle.params_from(pd)
    p1 = oracle.params_from(dict(pd, wetting=True, contact_angle_deg=60.0))
    f = oracle.init(p0, rR, rB, u)
    assert np.array_equal(oracle.step(p0, f, 3), oracle.step(p1, f, 3))


def test_wetting_rule_changes_only_wall_adjacent_cells_in_one_step():
    pd = _pd(8, 7, 6, wall=(0, 0, 1))
    rR, rB, u = wl.droplet(8, 7, 6, 3.0, 3.0, 1.0, center=(3.5, 3.0, 0.0), noise=1e-2, seed=6)
    p0 = oracle.params_from(pd)
    p1 = oracle.params_from(dict(pd, wetting=True, contact_angle_deg=45.0))
    f = oracle.init(p0, rR, rB, u)
    a, b = oracle.step(p0, f, 1), oracle.step(p1, f, 1)
    diff = np.abs(a - b).max(axis=(0, 1, 3, 4))  # per z plane
    # the rule acts at z = 0 and z = 5; streaming carries it one plane inward
    assert diff[0] > 1e-6 and diff[2] == 0.0 and diff[3] == 0.0
