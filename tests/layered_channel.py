"""The layered two-phase channel of Sec. IV.B (Eq. 54-55) as the tests read
it: helpers shared by the oracle pin and the GPU test.

Readings of what the paper leaves unstated (each chosen by a sweep of the
oracle, recorded beside the readings of the paper in the design notes):
  * walls: the paper's no-slip condition is the Zou-He scheme of its Ref.
    [45], i.e. wet nodes.  The 100 lattice spacings between the plates give
    101 nodes y_j = j - 50 with the plates on the first and last node (b = 50),
    the red fluid on the nodes |y_j| <= a = 25;
  * relaxation times: the smaller of tau_R, tau_B is 1, the other follows from
    M = mu_R / mu_B with mu_k = rho_k (c_s^k)^2 (tau_k - 1/2) (Eq. 51);
  * beta = 0.7, tau_e = tau_q = tau_pi = 1 (as in Sec. IV.A), delta = 0.98;
  * E_u = sum_y |u_x - u_x^a| / sum_y |u_x^a| over every node (Sec. IV.B).
"""
from __future__ import annotations

import json
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NY, A_HALF, B_HALF, G = 101, 25.0, 50.0, 1.5e-8


def printed_case(name):
    return json.load(open(os.path.join(GOLD, "printed_numbers.json")))["layered_flow"]["cases"][name]


def case_params(name, improved=True, beta=0.7, eq18_coef=None):
    """(params dict in the shared names, mu_R, mu_B) of case A, B or C."""
    c = printed_case(name)
    rR, rB, aB, M = c["rho_in_R"], c["rho_in_B"], c["alpha_B"], c["M"]
    aR = 1.0 - (1.0 - aB) * rB / rR              # rho_R / rho_B = (1 - a_B) / (1 - a_R)
    pR, pB = rR * 0.5 * (1.0 - aR), rB * 0.5 * (1.0 - aB)   # rho_k (c_s^k)^2
    if pR / pB > M:   # equal relaxation times would make mu_R / mu_B too large
        tR, tB = 1.0, 0.5 + pR * 0.5 / M / pB
    else:
        tB, tR = 1.0, 0.5 + M * pB * 0.5 / pR
    d = dict(nx=1, ny=NY, nz=1, wall=(0, 2, 0), improved=improved, rho_in_R=rR,
             rho_in_B=rB, alpha_R=aR, alpha_B=aB, tau_R=tR, tau_B=tB, tau_e=1.0,
             tau_q=1.0, tau_pi=1.0, A_R=1e-4, A_B=1e-4, beta=beta, delta=0.98,
             force=(G, 0.0, 0.0), gravity=(0.0, 0.0, 0.0))
    if eq18_coef is not None:
        d["eq18_coef"] = eq18_coef
    return d, pR * (tR - 0.5), pB * (tB - 0.5)


def analytic_profile(muR, muB, M):
    """u_x^a(y_j) of Eq. 54-55 on the nodes y_j = j - 50."""
    y = np.arange(NY) - (NY - 1) / 2.0
    a, b = A_HALF, B_HALF
    A1, A2 = -G / (2 * muR), -G / (2 * muB)
    B2 = 2 * (A1 * M - A2) * a
    C1 = (A2 - A1) * a * a - B2 * (b - a) - A2 * b * b
    C2 = -A2 * b * b - B2 * b
    return np.where(np.abs(y) <= a, A1 * y * y + C1, A2 * y * y + B2 * np.abs(y) + C2)


def initial_fields(name, from_profile):
    """(rho_R, rho_B, u) on the 1 x 101 x 1 lattice: the layers, at rest or
    moving with the analytic profile (which shortens the run to steady state)."""
    from paper_1904_03618_gb300 import workloads as wl
    c = printed_case(name)
    rho_R, rho_B, u = wl.layered_nodes(1, NY, 1, A_HALF, c["rho_in_R"], c["rho_in_B"])
    if from_profile:
        d, muR, muB = case_params(name)
        u[0] = analytic_profile(muR, muB, c["M"])[None, :, None]
    return rho_R, rho_B, u


def e_u(ux, ua):
    return float(np.abs(ux - ua).sum() / np.abs(ua).sum())


def oracle_e_u(name, improved, steps, eq18_coef=None, threads=1):
    """E_u of the FP64 oracle after `steps` steps from the analytic profile.
    Sets the OpenMP thread count of the process before the oracle loads
    (meant for a spawned worker: a 101-cell lattice runs fastest on one
    thread, and independent cases run side by side)."""
    os.environ["OMP_NUM_THREADS"] = str(threads)
    import oracle
    d, muR, muB = case_params(name, improved, eq18_coef=eq18_coef)
    p = oracle.params_from(d)
    f = oracle.step(p, oracle.init(p, *initial_fields(name, True)), steps)
    _, _, u = oracle.moments(p, f)
    return e_u(u[0, 0, :, 0], analytic_profile(muR, muB, printed_case(name)["M"]))


def oracle_profile(name, improved, steps, gscale=1.0, threads=1):
    """(u_x on the 101 nodes, E_u) of the FP64 oracle after `steps` steps
    from the analytic profile, with the body force G * gscale."""
    global G
    os.environ["OMP_NUM_THREADS"] = str(threads)
    import oracle
    g0 = G
    try:
        G = g0 * gscale
        d, muR, muB = case_params(name, improved)
        ua = analytic_profile(muR, muB, printed_case(name)["M"])
        fields = initial_fields(name, True)
    finally:
        G = g0
    p = oracle.params_from(d)
    f = oracle.step(p, oracle.init(p, *fields), steps)
    _, _, u = oracle.moments(p, f)
    return u[0, 0, :, 0].copy(), e_u(u[0, 0, :, 0], ua)


def equal_viscosity_error(improved, steps, threads=1):
    """Max |u_x - u_x^a| / max u_x^a of the oracle for the channel with case
    A's densities (0.1 / 0.8, alpha_R 0.2, alpha_B 0.9: p_R = p_B = 0.04) and
    equal relaxation times, after `steps` steps from the Poiseuille parabola
    u^a = G (50^2 - y^2) / (2 mu), mu = p_k (tau - 1/2).  Halfway bounce-back
    walls at y = +-50 (100 cells, y_j = j + 1/2 - 50), red where |y_j| <= 25,
    G = 1e-7, tau_v = 7/8 and tau_q = 1 ((tau_v - 1/2)(tau_q - 1/2) = 3/16)."""
    os.environ["OMP_NUM_THREADS"] = str(threads)
    import oracle
    from paper_1904_03618_gb300 import workloads as wl
    ny, g = 100, 1e-7
    tau = 0.5 + 3.0 / 16.0 / 0.5
    mu = 0.04 * (tau - 0.5)
    y = np.arange(ny) + 0.5 - ny / 2
    ua = g / (2 * mu) * (50.0 ** 2 - y ** 2)
    p = oracle.params(1, ny, 1, wall=(0, 1, 0), improved=improved, rho_in_R=0.1,
                      rho_in_B=0.8, alpha_R=0.2, alpha_B=0.9, tau_R=tau, tau_B=tau,
                      tau_e=1.0, tau_q=1.0, tau_pi=1.0, A_R=1e-4, A_B=1e-4, beta=0.7,
                      force=(g, 0.0, 0.0))
    rR, rB, u = wl.layered(1, ny, 1, 25.0, 0.1, 0.8)
    u[0] = ua[None, :, None]
    f = oracle.step(p, oracle.init(p, rR, rB, u), steps)
    _, _, uu = oracle.moments(p, f)
    return float(np.abs(uu[0, 0, :, 0] - ua).max() / ua.max())
