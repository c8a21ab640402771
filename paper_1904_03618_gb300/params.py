"""Parameter helpers of the product side (the oracle keeps its own copies).

alpha from the pressure balance of Eq. 13 (equal pressures
rho_k (1 - alpha_k) / 2 in the two bulk phases), relaxation time from a
kinematic viscosity (nu_k = (c_s^k)^2 (tau_k - 1/2), below Eq. 52), and the
perturbation amplitude from a surface tension (sigma = 2 (A_R + A_B) / 9
for the perturbation applied through the collision matrix, Eq. 53).
"""
from __future__ import annotations


def alpha_R_from_balance(rho_in_R: float, rho_in_B: float, alpha_B: float) -> float:
    return 1.0 - (1.0 - alpha_B) * rho_in_B / rho_in_R


def cs2(alpha: float) -> float:
    return 0.5 * (1.0 - alpha)


def tau_from_nu(nu: float, alpha: float) -> float:
    return 0.5 + nu / cs2(alpha)


def A_from_sigma(sigma: float) -> float:
    """A_R = A_B giving surface tension sigma."""
    return 9.0 * sigma / 4.0


def droplet_case(sample: dict, alpha_B: float = 0.7, beta: float = 0.7) -> dict:
    """lbm_params keywords of one sampled droplet case (see
    workloads.droplet_sweep): red drop of density ratio `density_ratio` in
    blue of density 1, both relaxation times 1, periodic cube."""
    n = sample["edge"]
    ratio = sample["density_ratio"]
    A = A_from_sigma(sample["sigma"])
    return dict(nx=n, ny=n, nz=n, wall=(0, 0, 0), improved=True, rho_in_R=ratio,
                rho_in_B=1.0, alpha_R=alpha_R_from_balance(ratio, 1.0, alpha_B),
                alpha_B=alpha_B, tau_R=1.0, tau_B=1.0, tau_e=1.0, tau_q=1.0,
                tau_pi=1.0, A_R=A, A_B=A, beta=beta, delta=0.98)
