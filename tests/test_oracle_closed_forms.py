"""Pins of the FP64 oracle's building blocks against what the paper prints
and what the mathematics fixes (no GPU needed).

Each test compares the oracle's velocity-space computation with an
independent statement: a matrix or number printed in the paper (golden
fixtures), a moment identity stated in the paper (Eq. 16, 17, 19, 21, 34-37,
Appendix), or a textbook special case.
"""
import json
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_matrix(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([int(v) for v in line.split()])
    return np.array(rows, dtype=np.float64)


E = _read_matrix("eq5_velocities.txt").T           # (19, 3), Eq. 5
M_PRINTED = _read_matrix("appendix_M.txt")          # Appendix
PRINTED = json.load(open(os.path.join(GOLD, "printed_numbers.json")))
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def _frac(v):
    return v[0] / v[1]


def test_weights_and_B_match_printed_values():
    w = PRINTED["weights"]
    # The oracle's equilibrium at u = 0 with alpha = 1/3 is rho * omega_i.
    f = oracle.feq(1.0, 1.0 / 3.0, (0, 0, 0))
    assert f[0] == pytest.approx(_frac(w["w0"]), abs=1e-15)
    assert np.allclose(f[1:7], _frac(w["w1_6"]), atol=1e-15)
    assert np.allclose(f[7:], _frac(w["w7_18"]), atol=1e-15)
    # B_i: Omega2 along a direction with (e.n)^2 = 0 gives -(A/2)|g| B_i.
    g = np.array([0.0, 0.0, 2.0])
    om = oracle.perturbation(1.0, g)
    b = PRINTED["B_i"]
    assert om[0] == pytest.approx(-0.5 * 2.0 * _frac(b["B0"]), abs=1e-15)
    assert om[1] == pytest.approx(-0.5 * 2.0 * _frac(b["B1_6"]), abs=1e-15)
    assert om[7] == pytest.approx(-0.5 * 2.0 * _frac(b["B7_18"]), abs=1e-15)


def test_transformation_matrix_equals_appendix():
    M = oracle.matrix_M()
    assert np.array_equal(M, M_PRINTED)
    Minv = oracle.matrix_Minv()
    assert np.allclose(Minv @ M, np.eye(19), atol=1e-13)
    assert np.allclose(Minv, np.linalg.inv(M_PRINTED), atol=1e-13)


def test_opposite_pairs_of_eq5():
    # Directions (1,2), (3,4), ..., (17,18) are opposite pairs.
    for i in range(1, 19, 2):
        assert np.array_equal(E[i], -E[i + 1])


def _moments(f):
    return M_PRINTED @ f


@pytest.mark.parametrize("alpha", [1 / 3, 0.2, 0.7, 0.9, 0.992])
def test_equilibrium_moments_match_appendix_rows_0_to_15(alpha):
    rho = 1.7
    u = np.array([0.031, -0.047, 0.022])
    f = oracle.feq(rho, alpha, u, improved=True)
    m = _moments(f)
    p = 0.5 * rho * (1 - alpha)
    ux, uy, uz = u
    uu = u @ u
    expected = [rho, rho * ux, rho * uy, rho * uz, 3 * p + rho * uu,
                rho * (2 * ux ** 2 - uy ** 2 - uz ** 2), rho * (uy ** 2 - uz ** 2),
                rho * ux * uy, rho * ux * uz, rho * uy * uz,
                p * uy, p * ux, p * uz, p * ux, p * uz, p * uy]
    assert np.allclose(m[:16], expected, rtol=0, atol=1e-14)


def test_equilibrium_rows_16_to_18_follow_M_feq_not_the_printed_form():
    rho, alpha = 2.3, 0.6
    u = np.array([0.05, -0.02, 0.04])
    f = oracle.feq(rho, alpha, u, improved=True)
    m = _moments(f)
    ux, uy, uz = u
    uu = u @ u
    # Direct sum over the four directions with e_x^2 e_y^2 = 1 (etc.).
    for row, (a, b, c) in zip((16, 17, 18), ((ux, uy, uz), (ux, uz, uy), (uy, uz, ux))):
        mf = rho * ((1 - alpha) + 2 * a * a + 2 * b * b - c * c) / 6
        printed = (rho * (1 - alpha - uu) + 2 * rho * (a * a + b * b)) / 6
        assert m[row] == pytest.approx(mf, abs=1e-15)
        assert abs(m[row] - printed) > 1e-5  # the printed row differs at O(u^2)


@pytest.mark.parametrize("improved", [True, False])
def test_second_moments_eq16(improved):
    rho, alpha = 0.8, 0.2
    u = np.array([0.02, 0.01, -0.03])
    f = oracle.feq(rho, alpha, u, improved=improved)
    p = 0.5 * rho * (1 - alpha)
    Pi = np.einsum("ia,ib,i->ab", E, E, f)
    assert np.allclose(Pi, rho * np.outer(u, u) + p * np.eye(3), atol=1e-15)


def _third(f):
    return np.einsum("ia,ib,ic,i->abc", E, E, E, f)


def test_third_moments_eq17_original_and_eq19_improved():
    rho, alpha = 1.3, 0.9
    u = np.array([0.04, -0.01, 0.02])
    p = 0.5 * rho * (1 - alpha)
    d = np.eye(3)
    sym = (np.einsum("a,bc->abc", u, d) + np.einsum("b,ac->abc", u, d)
           + np.einsum("c,ab->abc", u, d))
    T0 = _third(oracle.feq(rho, alpha, u, improved=False))
    assert np.allclose(T0, rho / 3 * sym, atol=1e-15)         # Eq. 17
    T1 = _third(oracle.feq(rho, alpha, u, improved=True))
    for a in range(3):
        for b in range(3):
            for c in range(3):
                want = (rho / 3 if a == b == c else p) * sym[a, b, c]  # Eq. 19
                assert T1[a, b, c] == pytest.approx(want, abs=1e-15)


def test_printed_eq18_coefficient_misses_eq19():
    """With the coefficient printed in Eq. 18 (3/2) the off-diagonal third
    moments land half way between rho/3 u and p u: Eq. 19 fails."""
    rho, alpha = 1.0, 0.9
    u = np.array([0.0, 0.05, 0.0])
    p = 0.5 * rho * (1 - alpha)
    f = oracle.feq(rho, alpha, u, improved=True,
                   eq18_coef=oracle.EQ18_COEF_PRINTED)
    T = _third(f)
    assert T[0, 0, 1] == pytest.approx(0.5 * (rho / 3 + p) * u[1], abs=1e-15)
    assert abs(T[0, 0, 1] - p * u[1]) > 1e-3


def test_improved_equals_original_for_standard_pressure_weights():
    """alpha = 1/3 makes phi = omega and c_s^2 = 1/3, so the Eq. 18 term
    vanishes and the equilibrium is the textbook D3Q19 one."""
    rho = 1.1
    u = np.array([0.03, 0.02, -0.05])
    a = oracle.feq(rho, 1 / 3, u, improved=True)
    b = oracle.feq(rho, 1 / 3, u, improved=False)
    eu = E @ u
    textbook = rho * W * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * (u @ u))
    assert np.allclose(a, textbook, atol=1e-15)
    assert np.allclose(b, textbook, atol=1e-15)


def test_correction_term_constraints_eq21_34_37():
    Q = np.array([1.3e-3, -0.7e-3, 2.1e-3])
    C = oracle.correction(Q)
    G = np.linalg.solve(M_PRINTED, C)            # G = M^-1 C (Eq. 45)
    assert abs(G.sum()) < 1e-15                   # Eq. 21
    assert np.allclose(E.T @ G, 0, atol=1e-15)    # Eq. 21
    P = np.einsum("ia,ib,i->ab", E, E, G)
    assert abs(P[0, 1]) < 1e-15 and abs(P[0, 2]) < 1e-15 and abs(P[1, 2]) < 1e-15  # Eq. 34
    assert np.allclose(np.diag(P), Q, atol=1e-15)  # Eq. 35-37
    # the high-order moments of G are zero by construction (below Eq. 48)
    assert np.allclose((M_PRINTED @ G)[7:], 0, atol=1e-15)


@pytest.mark.parametrize("g", [(0.3, 0.0, 0.0), (0.1, -0.2, 0.05), (1e-3, 2e-3, -4e-3)])
def test_perturbation_moments(g):
    """Eq. 8 carries no mass or momentum; its moments have the closed form
    (A/2)|g| pi(n) with pi_4 = -4/9, pi_5 = 2(3n_x^2-1)/9, pi_6 = 2(n_y^2-n_z^2)/9,
    pi_7..9 = 2 n_a n_b / 9, pi_16..18 = -n_z^2/9, -n_y^2/9, -n_x^2/9."""
    A = 0.02
    g = np.array(g)
    om = oracle.perturbation(A, g)
    m = M_PRINTED @ om
    gn = np.linalg.norm(g)
    n = g / gn
    pi = np.zeros(19)
    pi[4] = -4 / 9
    pi[5] = 2 * (3 * n[0] ** 2 - 1) / 9
    pi[6] = 2 * (n[1] ** 2 - n[2] ** 2) / 9
    pi[7], pi[8], pi[9] = 2 * n[0] * n[1] / 9, 2 * n[0] * n[2] / 9, 2 * n[1] * n[2] / 9
    pi[16], pi[17], pi[18] = -n[2] ** 2 / 9, -n[1] ** 2 / 9, -n[0] ** 2 / 9
    assert np.allclose(m, 0.5 * A * gn * pi, atol=1e-16)


def test_perturbation_zero_below_threshold():
    assert np.all(oracle.perturbation(1.0, (1e-14, 0, 0)) == 0.0)


def test_guo_force_moments():
    F = np.array([1e-3, -2e-3, 5e-4])
    u = np.array([0.04, 0.01, -0.02])
    Fi = oracle.force_guo(F, u)
    assert abs(Fi.sum()) < 1e-17
    assert np.allclose(E.T @ Fi, F, atol=1e-17)
    P = np.einsum("ia,ib,i->ab", E, E, Fi)
    assert np.allclose(P, np.outer(u, F) + np.outer(F, u), atol=1e-17)


def test_tau_v_interpolation_eq52():
    tR, tB, d = 1.0, 0.5625, 0.98
    h = 2 * tR * tB / (tR + tB)
    assert oracle.tau_v(0.0, tR, tB, d) == pytest.approx(h)
    assert oracle.tau_v(0.99, tR, tB, d) == tR
    assert oracle.tau_v(-0.99, tR, tB, d) == tB
    # continuity and zero slope at +-delta
    assert oracle.tau_v(d, tR, tB, d) == pytest.approx(tR, abs=1e-14)
    assert oracle.tau_v(-d, tR, tB, d) == pytest.approx(tB, abs=1e-14)
    eps = 1e-6
    assert (oracle.tau_v(d, tR, tB, d) - oracle.tau_v(d - eps, tR, tB, d)) / eps < 1e-5
    assert (oracle.tau_v(-d + eps, tR, tB, d) - oracle.tau_v(-d, tR, tB, d)) / eps < 1e-5
    xs = np.linspace(-1, 1, 401)
    ts = np.array([oracle.tau_v(x, tR, tB, d) for x in xs])
    assert np.all(np.diff(ts) >= -1e-15)  # monotone between tau_B and tau_R


def test_recolouring_weights_have_zero_mass():
    """sum_i cos(phi_i) phi_i^k = 0 for any direction (odd x even), which is
    what makes the recolouring of Eq. 10-11 conserve each colour's mass."""
    n = np.array([0.3, -0.5, 0.8])
    n /= np.linalg.norm(n)
    elen = np.linalg.norm(E, axis=1)
    cos = np.where(elen > 0, (E @ n) / np.where(elen > 0, elen, 1), 0)
    for alpha in (0.2, 0.9):
        phi = oracle.feq(1.0, alpha, (0, 0, 0))
        assert abs(cos @ phi) < 1e-16


def test_printed_parameter_identities():
    pr = PRINTED
    md = pr["moving_droplet"]
    assert oracle.alpha_R_from_balance(md["rho_in_R"], md["rho_in_B"], md["alpha_B"]) \
        == pytest.approx(md["alpha_R"])
    imp = pr["droplet_impact"]
    assert oracle.surface_tension(imp["A"], imp["A"]) == pytest.approx(imp["sigma"])
    We = imp["rho_in_R"] * imp["U0"] ** 2 * imp["D0"] / imp["sigma"]
    assert We == pytest.approx(imp["We"])
    # the layered-flow cases: all have equal pressures p_R = p_B
    for c in pr["layered_flow"]["cases"].values():
        aR = oracle.alpha_R_from_balance(c["rho_in_R"], c["rho_in_B"], c["alpha_B"])
        assert c["rho_in_R"] * oracle.cs2(aR) == pytest.approx(
            c["rho_in_B"] * oracle.cs2(c["alpha_B"]))


@pytest.mark.parametrize("theta", [30.0, 60.0, 90.0, 120.0, 150.0])
@pytest.mark.parametrize("side", [(0, 0, 1), (0, -1, 0), (1, 0, 0)])
def test_wetting_rule_sets_the_contact_angle(theta, side):
    """The rotated gradient keeps its magnitude and its direction along the
    wall, and makes the angle pi - theta with the inward wall normal."""
    g = np.array([0.07, -0.03, 0.05])
    out = oracle.wetting(side, theta, g)
    n = np.array(side, dtype=float)
    assert np.linalg.norm(out) == pytest.approx(np.linalg.norm(g), rel=1e-14)
    ang = np.degrees(np.arccos(out @ n / np.linalg.norm(out)))
    assert ang == pytest.approx(180.0 - theta, abs=1e-9)
    t_in = g - (g @ n) * n
    t_out = out - (out @ n) * n
    assert np.allclose(t_out / np.linalg.norm(t_out), t_in / np.linalg.norm(t_in), atol=1e-14)


def test_wetting_rule_edge_cases():
    # no wall contact: unchanged; purely normal gradient: unchanged
    g = np.array([0.1, 0.2, 0.3])
    assert np.array_equal(oracle.wetting((0, 0, 0), 60.0, g), g)
    assert np.array_equal(oracle.wetting((0, 0, 1), 60.0, [0.0, 0.0, 0.4]), [0.0, 0.0, 0.4])
    # 90 degrees: the normal component is removed
    out = oracle.wetting((0, 0, 1), 90.0, g)
    assert abs(out[2]) < 1e-15 and np.linalg.norm(out) == pytest.approx(np.linalg.norm(g))
    # edge cell: normal along the diagonal of the two walls
    out = oracle.wetting((1, 0, 1), 45.0, g)
    n = np.array([1.0, 0.0, 1.0]) / np.sqrt(2.0)
    assert np.degrees(np.arccos(out @ n / np.linalg.norm(out))) == pytest.approx(135.0)
