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


def _layered_all_fn(fn, jobs):
    """fn(*job) for every job, side by side in spawned single-threaded
    workers (fn sets the worker's OpenMP thread count before the oracle
    loads)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(fn, *j) for j in jobs]
        return [f.result() for f in futs]


def _layered_all(jobs):
    import layered_channel as lc
    return _layered_all_fn(lc.oracle_e_u, jobs)


@pytest.mark.slow
def test_layered_channel_matches_the_printed_errors():
    """Sec. IV.B, Eq. 54-55, cases A, B and C at steady state, from the
    analytic profile, under the readings stated in tests/layered_channel.py
    (Zou-He no-slip wet nodes, the smaller relaxation time 1, beta 0.7).
    The paper prints E_u = 0.66 %, 1.42 % and 0.36 % for the improved model
    and 44.6 %, 59.7 % and 6904 % for the original one.  The oracle gives
    0.449 %, 1.498 % and 0.580 % (improved) and 31.0 %, 64.0 % and 27.5 %
    (original); the bands are those values within a factor 1.5, which also
    holds each improved value within a factor 1.65 of the printed one and
    the original A and B within 1.5.  Case C's original-model error (the
    paper's density ratio 1000) is not reproduced: under this reading the
    original model's blue phase is 833 times too viscous (its third moments
    carry rho/3 instead of p_k, Eq. 17), which pins its velocity near zero
    rather than far above the profile.  The printed Eq. 18 coefficient 3/2
    gives several times the error of 3."""
    import layered_channel as lc
    jobs = [("A", True, 50000), ("B", True, 200000), ("C", True, 200000),
            ("A", False, 50000), ("B", False, 50000), ("C", False, 50000),
            ("A", True, 50000, oracle.EQ18_COEF_PRINTED)]
    eA, eB, eC, oA, oB, oC, pA = _layered_all(jobs)
    measured = {"A": (eA, 0.00449, 0.66), "B": (eB, 0.01498, 1.42), "C": (eC, 0.00580, 0.36)}
    for name, (e, ref, printed) in measured.items():
        assert ref / 1.5 < e < ref * 1.5, (name, e)
        assert printed / 100 / 1.65 < e < printed / 100 * 1.65, (name, e, printed)
    for name, e, ref in (("A", oA, 0.310), ("B", oB, 0.640), ("C", oC, 0.275)):
        assert ref / 1.5 < e < ref * 1.5, (name, e)
    assert 0.446 / 1.5 < oA < 0.446 * 1.5 and 0.597 / 1.5 < oB < 0.597 * 1.5
    assert oC > 10 * eC
    assert pA > 3 * eA


@pytest.mark.slow
def test_layered_channel_is_the_exact_parabola_at_equal_viscosity():
    """The channel's steady state pins the improved equilibrium across a
    density jump.  With case A's densities (0.1 / 0.8, alpha 0.2 / 0.9, equal
    pressures p_k = rho_k (c_s^k)^2 = 0.04) and equal relaxation times
    (M = 1), the improved model's off-diagonal third moments carry p_k u
    (Eq. 19), the same in both phases, so the exact solution is the
    single-phase Poiseuille parabola; the original model's carry rho_k u / 3
    (Eq. 17), whose jump across the interface bends the profile.  The
    relaxation times sit at (tau_v - 1/2)(tau_q - 1/2) = 3/16, where a
    single-phase D3Q19 MRT channel with halfway bounce-back is exact.  From
    the parabola, 100,000 steps: the improved model is within 5.2e-6 of it
    (2.3e-7 after 400,000 steps), the original 60 % off."""
    import layered_channel as lc
    e_imp, e_orig = _layered_all_fn(lc.equal_viscosity_error, [(True, 100000), (False, 20000)])
    assert e_imp < 2e-5, e_imp
    assert e_orig > 0.3, e_orig


@pytest.mark.slow
def test_galilean_invariance_drop_moves_with_the_flow():
    """Sec. IV.A on a smaller lattice: a red disc (R = 12, density ratio 3,
    alpha 0.9 / 0.7, A_R = A_B = 0.01, beta 0.5, tau 1 in both fluids, the
    paper's parameters) in a uniform flow U = 0.02 along x on a periodic
    48 x 48 x 1 lattice.  Galilean invariance: the drop is carried with the
    flow and keeps its shape.  After 2000 steps (40 cells travelled) the
    improved model's centroid is within 0.3 cells of x0 + U t (measured
    0.24) and its axis ratio below 1.01 (1.008); the original model's drop
    lags by more than 5 cells (9.6) and turns elliptic (1.066)."""
    n, R, U, steps = 48, 12.0, 0.02, 2000
    out = {}
    for improved in (True, False):
        pd = _pd(n, n, 1, improved=improved, rho_in_R=3.0, rho_in_B=1.0, alpha_R=0.9,
                 alpha_B=0.7, tau_R=1.0, tau_B=1.0, tau_e=1.0, tau_q=1.0, tau_pi=1.0,
                 A_R=0.01, A_B=0.01, beta=0.5, force=(0, 0, 0), gravity=(0, 0, 0))
        p = oracle.params_from(pd)
        rR, rB, u = wl.cylinder_z(n, n, 1, R, 3.0, 1.0, velocity=(U, 0.0, 0.0))
        a0, cx0, _ = _disc_shape(rR, rB, (3.0, 1.0))
        f = oracle.step(p, oracle.init(p, rR, rB, u), steps)
        r1, r2, _ = oracle.moments(p, f)
        a, cx, cy = _disc_shape(r1, r2, (3.0, 1.0))
        lag = ((cx0 + U * steps) - cx + n / 2) % n - n / 2
        out[improved] = (a, lag, cy)
        assert abs(f[0].sum() - oracle.init(p, rR, rB, u)[0].sum()) < 1e-9 * f[0].sum()
    (a_i, lag_i, cy_i), (a_o, lag_o, _) = out[True], out[False]
    assert abs(a0 - 1) < 1e-3
    assert abs(lag_i) < 0.3 and a_i < 1.01, out
    assert lag_o > 5.0 and a_o > 1.04, out
    assert abs(cy_i - (n - 1) / 2) < 1e-6


def _disc_shape(rR, rB, rin):
    """(principal-axis ratio, centroid x, centroid y) of the red region
    (rho^N > 0) of a quasi-2D periodic field (1, ny, nx); the centroid from
    circular means."""
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
    inertia = np.array([[(ind * dx * dx).sum(), (ind * dx * dy).sum()],
                        [(ind * dx * dy).sum(), (ind * dy * dy).sum()]]) / m
    ev = np.linalg.eigvalsh(inertia)
    return np.sqrt(ev[1] / ev[0]), cx, cy


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
