"""FP64 CPU oracle for the improved 3D colour-gradient MRT-LB step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (``paper_1904_03618_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, per-colour literal
form of Wen, Li, Yu & Luo, arXiv:1904.03618, Sec. II-III and the Appendix).
This module only marshals numpy arrays through ctypes, plus the oracle's own
parameter helpers (Eq. 13 pressure balance, Eq. 51 viscosity, the surface
tension relation stated below Eq. 52).

Array layouts (numpy, C order):
    f        (2, 19, nz, ny, nx)   k = 0 red, 1 blue; f_i^k(x, t) after streaming
    rho      (nz, ny, nx)
    u        (3, nz, ny, nx)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``lbm_oracle.c`` into ``oracle/_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(
                 os.path.join(_HERE, "lbm_oracle.h")))
    if force or stale:
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OracleParams(ctypes.Structure):
    """Mirror of ``or_params`` in ``lbm_oracle.h``."""
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("wall", ctypes.c_int * 3),
        ("improved", ctypes.c_int), ("pad_", ctypes.c_int),
        ("rho_in_R", ctypes.c_double), ("rho_in_B", ctypes.c_double),
        ("alpha_R", ctypes.c_double), ("alpha_B", ctypes.c_double),
        ("tau_R", ctypes.c_double), ("tau_B", ctypes.c_double),
        ("tau_e", ctypes.c_double), ("tau_q", ctypes.c_double),
        ("tau_pi", ctypes.c_double),
        ("A_R", ctypes.c_double), ("A_B", ctypes.c_double),
        ("beta", ctypes.c_double), ("delta", ctypes.c_double),
        ("force", ctypes.c_double * 3), ("gravity", ctypes.c_double * 3),
        ("eq18_coef", ctypes.c_double),
        ("wetting", ctypes.c_int), ("pad2_", ctypes.c_int),
        ("contact_angle_deg", ctypes.c_double),
        ("collision", ctypes.c_int), ("pad3_", ctypes.c_int),
        ("wall_u", (ctypes.c_double * 3) * 2),
    ]


# Collision operators: the MRT form (Eq. 40-44, perturbation by Eq. 53) and
# the BGK form with the correction term (Eq. 20, perturbation divided by tau).
COLLISION = {"mrt": 0, "bgk": 1}


# Coefficient of the high-order term of Eq. 18.  As printed it is 3/2; the
# value that yields the third moments of Eq. 19 and the Appendix is 3.
EQ18_COEF_PRINTED = 1.5
EQ18_COEF = 3.0


def params(nx, ny, nz, *, wall=(0, 0, 0), improved=True, rho_in_R=1.0,
           rho_in_B=1.0, alpha_R=1.0 / 3.0, alpha_B=1.0 / 3.0, tau_R=1.0,
           tau_B=1.0, tau_e=1.0, tau_q=1.0, tau_pi=1.0, A_R=0.0, A_B=0.0,
           beta=0.7, delta=0.98, force=(0.0, 0.0, 0.0),
           gravity=(0.0, 0.0, 0.0), eq18_coef=EQ18_COEF, wetting=False,
           contact_angle_deg=90.0, collision="mrt",
           wall_u=((0.0, 0.0, 0.0), (0.0, 0.0, 0.0))) -> OracleParams:
    p = OracleParams()
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    for a in range(3):
        p.wall[a] = int(wall[a])
        p.force[a] = float(force[a])
        p.gravity[a] = float(gravity[a])
    p.improved = 1 if improved else 0
    p.rho_in_R, p.rho_in_B = float(rho_in_R), float(rho_in_B)
    p.alpha_R, p.alpha_B = float(alpha_R), float(alpha_B)
    p.tau_R, p.tau_B = float(tau_R), float(tau_B)
    p.tau_e, p.tau_q, p.tau_pi = float(tau_e), float(tau_q), float(tau_pi)
    p.A_R, p.A_B = float(A_R), float(A_B)
    p.beta, p.delta = float(beta), float(delta)
    p.eq18_coef = float(eq18_coef)
    p.wetting = 1 if wetting else 0
    p.contact_angle_deg = float(contact_angle_deg)
    p.collision = COLLISION[collision] if isinstance(collision, str) else int(collision)
    for side in range(2):
        for a in range(3):
            p.wall_u[side][a] = float(wall_u[side][a])
    return p


def params_from(d: dict) -> OracleParams:
    """Build oracle params from a plain dict of the shared parameter names."""
    kw = dict(d)
    nx, ny, nz = kw.pop("nx"), kw.pop("ny"), kw.pop("nz")
    for k in ("storage", "kernel", "ref_R", "ref_B"):
        kw.pop(k, None)
    return params(nx, ny, nz, **kw)


# ---- the oracle's own parameter helpers ------------------------------------

def alpha_R_from_balance(rho_in_R, rho_in_B, alpha_B):
    """Pressure balance rho_R^in / rho_B^in = (1 - alpha_B) / (1 - alpha_R)
    (Sec. IV.A, Eq. 13)."""
    return 1.0 - (1.0 - alpha_B) * rho_in_B / rho_in_R


def cs2(alpha):
    """(c_s^k)^2 = (1 - alpha_k) / 2 (Eq. 13, c = 1)."""
    return 0.5 * (1.0 - alpha)


def tau_from_nu(nu, alpha):
    """nu_k = (c_s^k)^2 (tau_v^k - 1/2) (below Eq. 52)."""
    return 0.5 + nu / cs2(alpha)


def surface_tension(A_R, A_B):
    """sigma = 2 (A_R + A_B) / 9 for the perturbation of Eq. 53."""
    return 2.0 * (A_R + A_B) / 9.0


# ---- ctypes bindings --------------------------------------------------------

_dp = ctypes.POINTER(ctypes.c_double)


def _lib_handle():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(OracleParams)
        lib.or_matrix_M.argtypes = [_dp]
        lib.or_matrix_Minv.argtypes = [_dp]
        lib.or_matrix_Minv.restype = ctypes.c_int
        lib.or_feq.argtypes = [ctypes.c_double, ctypes.c_double, _dp,
                               ctypes.c_int, ctypes.c_double, _dp]
        lib.or_force_guo.argtypes = [_dp, _dp, _dp]
        lib.or_perturbation.argtypes = [ctypes.c_double, _dp, _dp]
        lib.or_correction.argtypes = [_dp, _dp]
        lib.or_wetting.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_double, _dp]
        lib.or_tau_v.argtypes = [ctypes.c_double] * 4
        lib.or_tau_v.restype = ctypes.c_double
        lib.or_moments.argtypes = [P, _dp, _dp, _dp, _dp]
        lib.or_moments.restype = ctypes.c_int
        lib.or_init.argtypes = [P, _dp, _dp, _dp, _dp]
        lib.or_init.restype = ctypes.c_int
        lib.or_step.argtypes = [P, _dp, _dp, ctypes.c_int]
        lib.or_step.restype = ctypes.c_int
        lib.or_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _vec(v, n):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(n))
    return a


def matrix_M() -> np.ndarray:
    out = np.zeros((19, 19))
    _lib_handle().or_matrix_M(_ptr(out))
    return out


def matrix_Minv() -> np.ndarray:
    out = np.zeros((19, 19))
    rc = _lib_handle().or_matrix_Minv(_ptr(out))
    assert rc == 0
    return out


def feq(rho_k, alpha_k, u, improved=True, eq18_coef=EQ18_COEF) -> np.ndarray:
    out = np.zeros(19)
    uu = _vec(u, 3)
    _lib_handle().or_feq(float(rho_k), float(alpha_k), _ptr(uu),
                         1 if improved else 0, float(eq18_coef), _ptr(out))
    return out


def force_guo(F, u) -> np.ndarray:
    out = np.zeros(19)
    FF, uu = _vec(F, 3), _vec(u, 3)
    _lib_handle().or_force_guo(_ptr(FF), _ptr(uu), _ptr(out))
    return out


def perturbation(A_k, grad) -> np.ndarray:
    out = np.zeros(19)
    g = _vec(grad, 3)
    _lib_handle().or_perturbation(float(A_k), _ptr(g), _ptr(out))
    return out


def correction(Q) -> np.ndarray:
    out = np.zeros(19)
    q = _vec(Q, 3)
    _lib_handle().or_correction(_ptr(q), _ptr(out))
    return out


def wetting(wall_side, theta_deg, grad) -> np.ndarray:
    g = _vec(grad, 3).copy()
    side = (ctypes.c_int * 3)(*[int(v) for v in wall_side])
    _lib_handle().or_wetting(side, float(theta_deg), _ptr(g))
    return g


def tau_v(rhoN, tau_R, tau_B, delta=0.98) -> float:
    return _lib_handle().or_tau_v(float(rhoN), float(tau_R), float(tau_B),
                                  float(delta))


def init(p: OracleParams, rho_R, rho_B, u) -> np.ndarray:
    shape = (p.nz, p.ny, p.nx)
    rR = np.ascontiguousarray(np.asarray(rho_R, dtype=np.float64).reshape(shape))
    rB = np.ascontiguousarray(np.asarray(rho_B, dtype=np.float64).reshape(shape))
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape((3,) + shape))
    f = np.zeros((2, 19) + shape)
    rc = _lib_handle().or_init(ctypes.byref(p), _ptr(rR), _ptr(rB), _ptr(uu),
                               _ptr(f))
    assert rc == 0
    return f


def step(p: OracleParams, f: np.ndarray, nsteps: int = 1) -> np.ndarray:
    shape = (2, 19, p.nz, p.ny, p.nx)
    fin = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(shape))
    fout = np.empty(shape)
    rc = _lib_handle().or_step(ctypes.byref(p), _ptr(fin), _ptr(fout),
                               int(nsteps))
    if rc != 0:
        raise RuntimeError("or_step failed with %d" % rc)
    return fout


def moments(p: OracleParams, f: np.ndarray):
    shape = (p.nz, p.ny, p.nx)
    fin = np.ascontiguousarray(
        np.asarray(f, dtype=np.float64).reshape((2, 19) + shape))
    rR, rB = np.empty(shape), np.empty(shape)
    u = np.empty((3,) + shape)
    rc = _lib_handle().or_moments(ctypes.byref(p), _ptr(fin), _ptr(rR),
                                  _ptr(rB), _ptr(u))
    assert rc == 0
    return rR, rB, u


def num_threads() -> int:
    return int(_lib_handle().or_num_threads())
