"""Second FP64 restatement of the step, in numpy, in velocity space.

TEST INFRASTRUCTURE ONLY (same import rule as the ``oracle`` package).

This one deliberately takes a different route from ``lbm_oracle.c`` so that
the two check each other:
  * the transformation matrix is the one printed in the Appendix (read from
    the transcription in ``tests/golden/appendix_M.txt``), and its inverse is
    ``numpy.linalg.inv``;
  * the collision is applied in velocity space, Eq. 40, with the dense
    collision matrix Lambda = M^-1 S M formed per cell; the correction term is
    G^k = M^-1 C^k (Eq. 45) and the perturbation uses Eq. 53 as Lambda Omega2;
  * streaming uses ``numpy.roll`` plus explicit halfway bounce-back.
With ``collision="bgk"`` the collision matrix is Lambda = I / tau_v, which
the paper states turns Eq. 40 into Eq. 20, and Eq. 53 into the perturbation
divided by tau.
Moving plates (``wall`` entry 2, Zou-He velocity nodes): the five entering
populations of each colour and the colour density are the solution of the
six linear conditions that define the scheme -- mass, the two tangential
momenta equal to rho_k u_t, the normal axis population bouncing back its
non-equilibrium part (f_n - f_-n = rho_k u_n / 3), and the same for each
pair of diagonals (their sum) -- solved with ``numpy.linalg.solve``, not
through the closed form the C oracle uses.

It is vectorised over cells and intended for lattices of a few hundred cells.
The readings it takes are the same as the C oracle's (see its header).
"""
from __future__ import annotations

import os

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_GOLD = os.path.join(_ROOT, "tests", "golden")


def _read_int_matrix(name):
    rows = []
    with open(os.path.join(_GOLD, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(v) for v in line.split()])
    return np.array(rows, dtype=np.float64)


M = _read_int_matrix("appendix_M.txt")          # Appendix
E = _read_int_matrix("eq5_velocities.txt").T    # Eq. 5, shape (19, 3)
MINV = np.linalg.inv(M)
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)       # below Eq. 6
BP = np.array([-1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)     # below Eq. 8
OPP = np.array([int(np.where((E == -E[i]).all(axis=1))[0][0]) for i in range(19)])
ELEN = np.sqrt((E ** 2).sum(axis=1))
GRAD_EPS = 1e-12


def _phi(alpha):
    """phi_i^k of Eq. 13, shape (19,)."""
    return np.array([alpha] + [(1 - alpha) / 12] * 6 + [(1 - alpha) / 24] * 12)


def _neighbour(psi, e, wall):
    """psi(x + e) with periodic wrap; beyond a wall, the centre value."""
    out = psi
    for ax, d in enumerate(e):
        d = int(d)
        if d == 0:
            continue
        arr_axis = 2 - ax  # arrays are (z, y, x)
        out = np.roll(out, -d, axis=arr_axis)
    for ax, d in enumerate(e):
        d = int(d)
        if d == 0 or not wall[ax]:
            continue
        arr_axis = 2 - ax
        n = psi.shape[arr_axis]
        idx = [slice(None)] * 3
        idx[arr_axis] = n - 1 if d > 0 else 0
        out = out.copy()
        out[tuple(idx)] = psi[tuple(idx)]
    return out


def _grad(psi, wall):
    """Eq. 49 applied to a scalar field: returns (3, nz, ny, nx)."""
    g = np.zeros((3,) + psi.shape)
    for i in range(1, 19):
        nb = _neighbour(psi, E[i], wall)
        for a in range(3):
            if E[i, a] != 0:
                g[a] += W[i] * nb * E[i, a]
    return 3.0 * g


def _feq(rho_k, alpha, u, improved, coef):
    """Eq. 18 (improved) or Eq. 6 (original); returns (19, cells...)."""
    cs2 = 0.5 * (1 - alpha)
    eu = np.einsum("ia,a...->i...", E, u)
    uu = (u ** 2).sum(axis=0)
    ee = (E ** 2).sum(axis=1)
    br = 3 * eu + 4.5 * eu ** 2 - 1.5 * uu[None]
    if improved:
        br = br + coef * eu * (3 * cs2 - 1) * (3 * ee - 5)[:, None, None, None]
    return rho_k[None] * (_phi(alpha)[:, None, None, None]
                          + W[:, None, None, None] * br)


def _tau_v(rhoN, tR, tB, delta):
    """Eq. 52 with the parabolic interpolants (same reading as the C oracle)."""
    s = 2 * tR * tB / (tR + tB)
    a = 2 * (tR - s) / delta
    b = 2 * (s - tB) / delta
    gR = s + a * rhoN - a / (2 * delta) * rhoN ** 2
    gB = s + b * rhoN + b / (2 * delta) * rhoN ** 2
    return np.where(rhoN > delta, tR,
                    np.where(rhoN > 0, gR, np.where(rhoN >= -delta, gB, tB)))


def step(pd: dict, f: np.ndarray, nsteps: int = 1) -> np.ndarray:
    """Advance f (2, 19, nz, ny, nx) by nsteps.  ``pd`` holds the parameters
    under the same names as the C oracle's ``or_params``."""
    wall = tuple(int(v) for v in pd.get("wall", (0, 0, 0)))
    improved = bool(pd.get("improved", True))
    coef = float(pd.get("eq18_coef", 3.0))
    rin = (float(pd["rho_in_R"]), float(pd["rho_in_B"]))
    alpha = (float(pd["alpha_R"]), float(pd["alpha_B"]))
    Ak = (float(pd.get("A_R", 0.0)), float(pd.get("A_B", 0.0)))
    beta = float(pd.get("beta", 0.7))
    delta = float(pd.get("delta", 0.98))
    force = np.asarray(pd.get("force", (0, 0, 0)), dtype=np.float64)
    grav = np.asarray(pd.get("gravity", (0, 0, 0)), dtype=np.float64)
    tau_e, tau_q, tau_pi = (float(pd.get("tau_e", 1.0)), float(pd.get("tau_q", 1.0)),
                            float(pd.get("tau_pi", 1.0)))
    f = np.array(f, dtype=np.float64, copy=True)
    shp = f.shape[2:]
    for _ in range(nsteps):
        rk = f.sum(axis=1)                       # (2, ...) Eq. 4
        rho = rk.sum(axis=0)
        j = np.einsum("ia,i...->a...", E, f.sum(axis=0))
        F = force[:, None, None, None] + grav[:, None, None, None] * rho[None]
        u = (j + 0.5 * F) / rho[None]
        a_, b_ = rk[0] / rin[0], rk[1] / rin[1]
        rhoN = (a_ - b_) / (a_ + b_)
        g = _grad(rhoN, wall)
        gnorm = np.sqrt((g ** 2).sum(axis=0))
        big = gnorm >= GRAD_EPS
        safe = np.where(big, gnorm, 1.0)
        n = g / safe[None]
        tv = _tau_v(rhoN, float(pd["tau_R"]), float(pd["tau_B"]), delta)
        s = np.empty((19,) + shp)
        s[0:4] = 1.0
        s[4] = 1.0 / tau_e
        s[5:10] = 1.0 / tv[None]
        s[10:16] = 1.0 / tau_q
        s[16:19] = 1.0 / tau_pi
        if pd.get("collision", "mrt") == "bgk":
            # Lambda = I / tau_v per cell (Eq. 20)
            Lam = np.einsum("c,ij->cij", 1.0 / tv.reshape(-1), np.eye(19))
        else:
            # Lambda = M^-1 S M per cell, as (cells, 19, 19)
            sc = s.reshape(19, -1).T
            Lam = np.einsum("ir,cr,rj->cij", MINV, sc, M)
        fstar = np.zeros((19,) + shp)
        for k in range(2):
            cs2 = 0.5 * (1 - alpha[k])
            qbar = rk[k][None] * u * (1 - 3 * cs2)
            Q = np.stack([_grad(qbar[a], wall)[a] for a in range(3)])
            C = np.zeros((19,) + shp)
            if improved:
                C[4] = Q[0] + Q[1] + Q[2]
                C[5] = 2 * Q[0] - Q[1] - Q[2]
                C[6] = Q[1] - Q[2]
            G = np.einsum("ir,r...->i...", MINV, C)               # Eq. 45
            Fk = F * (rk[k] / rho)[None]
            eu = np.einsum("ia,a...->i...", E, u)
            eF = np.einsum("ia,a...->i...", E, Fk)
            uF = (u * Fk).sum(axis=0)
            FG = W[:, None, None, None] * (3 * (eF - uF[None]) + 9 * eu * eF)
            fk = f[k]
            fe = _feq(rk[k], alpha[k], u, improved, coef)
            src = (G + FG).reshape(19, -1).T
            neq = (fk - fe).reshape(19, -1).T
            om1 = (-np.einsum("cij,cj->ci", Lam, neq)
                   + src - 0.5 * np.einsum("cij,cj->ci", Lam, src))  # Eq. 40
            en = np.einsum("ia,a...->i...", E, n)
            om2 = np.where(big[None], 0.5 * Ak[k] * gnorm[None]
                           * (W[:, None, None, None] * en ** 2
                              - BP[:, None, None, None]), 0.0)       # Eq. 8
            om2n = np.einsum("cij,cj->ci", Lam, om2.reshape(19, -1).T)  # Eq. 53
            fstar += fk + om1.T.reshape((19,) + shp) + om2n.T.reshape((19,) + shp)
        # Eq. 10-11
        cosphi = np.where(big[None], np.einsum("ia,a...->i...", E, n)
                          / np.where(ELEN > 0, ELEN, 1.0)[:, None, None, None], 0.0)
        cosphi[0] = 0.0
        feq0 = (rk[0][None] * _phi(alpha[0])[:, None, None, None]
                + rk[1][None] * _phi(alpha[1])[:, None, None, None])
        seg = beta * (rk[0] * rk[1] / rho ** 2)[None] * cosphi * feq0
        fp = np.stack([(rk[0] / rho)[None] * fstar + seg,
                       (rk[1] / rho)[None] * fstar - seg])
        # streaming with periodic wrap and halfway bounce-back
        new = np.empty_like(fp)
        for i in range(19):
            v = fp[:, i]
            for ax in range(3):
                d = int(E[i, ax])
                if d:
                    v = np.roll(v, d, axis=3 - ax)
            new[:, i] = v
        for i in range(19):
            for ax in range(3):
                d = int(E[i, ax])
                if d == 0 or not wall[ax]:
                    continue
                n_ax = shp[2 - ax]
                idx = [slice(None)] * 4
                idx[3 - ax] = 0 if d > 0 else n_ax - 1
                new[(slice(None), i) + tuple(idx[1:])] = \
                    fp[(slice(None), OPP[i]) + tuple(idx[1:])]
        for ax in range(3):
            if wall[ax] == 2:
                _zou_he(new, ax, pd["wall_u"])
        f = new
    return f


def _zou_he(f, ax, wall_u):
    """Velocity nodes on both faces of axis ax, in place (see the header)."""
    nax = 3 - ax                     # array axis of lattice axis ax in (k, i, z, y, x)
    t1, t2 = (ax + 1) % 3, (ax + 2) % 3
    for side in range(2):
        s = 1 if side == 0 else -1
        u = np.asarray(wall_u[side], dtype=np.float64)
        un = s * u[ax]
        en = s * E[:, ax]
        unk = [i for i in range(19) if en[i] == 1]
        axis_i = [i for i in unk if E[i, t1] == 0 and E[i, t2] == 0][0]
        A = np.zeros((6, 6))
        A[0, :5] = 1.0
        A[0, 5] = -1.0                                   # mass
        for r, t in ((1, t1), (2, t2)):                  # tangential momenta
            A[r, :5] = [E[i, t] for i in unk]
            A[r, 5] = -u[t]
        A[3, unk.index(axis_i)] = 1.0
        A[3, 5] = -un / 3.0                              # normal bounce-back
        for r, t in ((4, t1), (5, t2)):                  # diagonal pair sums
            for i in unk:
                if E[i, t] != 0:
                    A[r, unk.index(i)] = 1.0
            A[r, 5] = -un / 3.0
        idx = [slice(None)] * 5
        idx[2 + (2 - ax)] = 0 if side == 0 else f.shape[2 + (2 - ax)] - 1
        face = f[tuple(idx)]                             # (2, 19, a, b)
        known = [i for i in range(19) if en[i] != 1]
        for k in range(2):
            fk = face[k]
            b = np.zeros((6,) + fk.shape[1:])
            b[0] = -sum(fk[i] for i in known)
            for r, t in ((1, t1), (2, t2)):
                b[r] = -sum(E[i, t] * fk[i] for i in known)
            b[3] = fk[OPP[axis_i]]
            for r, t in ((4, t1), (5, t2)):
                b[r] = sum(fk[OPP[i]] for i in unk if E[i, t] != 0)
            sol = np.linalg.solve(A, b.reshape(6, -1)).reshape(b.shape)
            for j, i in enumerate(unk):
                fk[i] = sol[j]
        f[tuple(idx)] = face
