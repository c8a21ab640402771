"""Python binding of the C ABI in ``include/lbm.h`` (ctypes).

Argument marshalling only: every step of the computation runs in the CUDA
library ``_lib/liblbm.so`` built by ``__graft_entry__.build()`` (or the
build named by the environment variable ``LBM_LIBRARY``, e.g. the
index-checked ``_lib/liblbm_checked.so`` of
``__graft_entry__.build_checked()``).  If that library is missing this
module raises on import -- there is no CPU fallback.

Functions carry the C names (``lbm_create``, ``lbm_init_fields``,
``lbm_step``, ``lbm_moments``, ``lbm_diagnostics``, ``lbm_get_f``,
``lbm_set_f``, ``lbm_get_populations``, ``lbm_set_populations``,
``lbm_destroy``, ``lbm_last_error``, the in-place ``lbm_inplace_init``,
``lbm_step_inplace``, ``lbm_inplace_read`` and the others of the header);
:class:`Lattice` is a small convenience wrapper holding a context, its torch
stream and output tensors, :class:`InPlaceLattice` the same for the in-place
step (its population array, scratch and parity).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(_HERE, "_lib", "liblbm.so")

if not os.path.exists(LIB_PATH):
    raise RuntimeError(
        "CUDA library %s is missing: run __graft_entry__.build() first "
        "(there is no CPU fallback)" % LIB_PATH)

_lib = ctypes.CDLL(LIB_PATH)

LBM_OK, LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA = 0, -1, -2, -3
LBM_ERR_UNSTABLE, LBM_ERR_TIMEOUT, LBM_ERR_STATE = -4, -5, -6
LBM_F32, LBM_F16, LBM_BF16 = 0, 1, 2
LBM_KERNEL_FUSED, LBM_KERNEL_TWO_PASS = 0, 1
STORAGE = {"f32": LBM_F32, "f16": LBM_F16, "bf16": LBM_BF16}
LBM_COLLISION_MRT, LBM_COLLISION_BGK = 0, 1
COLLISION = {"mrt": LBM_COLLISION_MRT, "bgk": LBM_COLLISION_BGK}


class LbmParams(ctypes.Structure):
    """Mirror of ``lbm_params``."""
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("wall", ctypes.c_int * 3),
        ("improved", ctypes.c_int), ("storage", ctypes.c_int),
        ("kernel", ctypes.c_int), ("wetting", ctypes.c_int),
        ("rho_in_R", ctypes.c_double), ("rho_in_B", ctypes.c_double),
        ("alpha_R", ctypes.c_double), ("alpha_B", ctypes.c_double),
        ("tau_R", ctypes.c_double), ("tau_B", ctypes.c_double),
        ("tau_e", ctypes.c_double), ("tau_q", ctypes.c_double),
        ("tau_pi", ctypes.c_double),
        ("A_R", ctypes.c_double), ("A_B", ctypes.c_double),
        ("beta", ctypes.c_double), ("delta", ctypes.c_double),
        ("force", ctypes.c_double * 3), ("gravity", ctypes.c_double * 3),
        ("ref_R", ctypes.c_double), ("ref_B", ctypes.c_double),
        ("contact_angle_deg", ctypes.c_double),
        ("collision", ctypes.c_int), ("reserved", ctypes.c_int),
        ("wall_u", (ctypes.c_double * 3) * 2),
    ]


class LbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("lbm status %d: %s" % (status, message))
        self.status = status


_ctx_p = ctypes.c_void_p
_fp = ctypes.c_void_p

_lib.lbm_create.argtypes = [ctypes.POINTER(LbmParams), ctypes.c_void_p,
                            ctypes.POINTER(ctypes.c_void_p)]
_lib.lbm_create.restype = ctypes.c_int
_lib.lbm_init_fields.argtypes = [_ctx_p, _fp, _fp, _fp, _fp]
_lib.lbm_init_fields.restype = ctypes.c_int
_lib.lbm_step.argtypes = [_ctx_p, ctypes.c_int]
_lib.lbm_step.restype = ctypes.c_int
_lib.lbm_moments.argtypes = [_ctx_p, _fp, _fp, _fp]
_lib.lbm_moments.restype = ctypes.c_int
_lib.lbm_diagnostics.argtypes = [_ctx_p, ctypes.POINTER(ctypes.c_double)]
_lib.lbm_diagnostics.restype = ctypes.c_int
_lib.lbm_step_diagnostics_async.argtypes = [_ctx_p, ctypes.c_int, _fp]
_lib.lbm_step_diagnostics_async.restype = ctypes.c_int
_lib.lbm_step_monitored.argtypes = [_ctx_p, ctypes.c_int, _fp]
_lib.lbm_step_monitored.restype = ctypes.c_int
_lib.lbm_sync.argtypes = [_ctx_p]
_lib.lbm_sync.restype = ctypes.c_int
_lib.lbm_get_f.argtypes = [_ctx_p, _fp]
_lib.lbm_get_f.restype = ctypes.c_int
_lib.lbm_set_f.argtypes = [_ctx_p, _fp]
_lib.lbm_set_f.restype = ctypes.c_int
_lib.lbm_population_bytes.argtypes = [_ctx_p]
_lib.lbm_population_bytes.restype = ctypes.c_size_t
_lib.lbm_get_populations.argtypes = [_ctx_p, _fp]
_lib.lbm_get_populations.restype = ctypes.c_int
_lib.lbm_set_populations.argtypes = [_ctx_p, _fp]
_lib.lbm_set_populations.restype = ctypes.c_int
_lib.lbm_plane_bytes.argtypes = [_ctx_p]
_lib.lbm_plane_bytes.restype = ctypes.c_size_t
_lib.lbm_get_planes.argtypes = [_ctx_p, ctypes.c_int, ctypes.c_int, _fp]
_lib.lbm_get_planes.restype = ctypes.c_int
_lib.lbm_set_planes.argtypes = [_ctx_p, ctypes.c_int, ctypes.c_int, _fp]
_lib.lbm_set_planes.restype = ctypes.c_int
_lib.lbm_set_fused_config.argtypes = [_ctx_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
_lib.lbm_set_fused_config.restype = ctypes.c_int
_lib.lbm_get_fused_config.argtypes = [_ctx_p] + [ctypes.POINTER(ctypes.c_int)] * 3
_lib.lbm_get_fused_config.restype = ctypes.c_int
_lib.lbm_create_batch.argtypes = [ctypes.POINTER(LbmParams), ctypes.c_int, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_void_p)]
_lib.lbm_create_batch.restype = ctypes.c_int
_lib.lbm_num_cases.argtypes = [_ctx_p]
_lib.lbm_num_cases.restype = ctypes.c_int
_lib.lbm_batch_init_fields.argtypes = [_ctx_p, ctypes.c_int, _fp, _fp, _fp]
_lib.lbm_batch_init_fields.restype = ctypes.c_int
_lib.lbm_batch_moments.argtypes = [_ctx_p, ctypes.c_int, _fp, _fp, _fp]
_lib.lbm_batch_moments.restype = ctypes.c_int
_lib.lbm_batch_diagnostics.argtypes = [_ctx_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
_lib.lbm_batch_diagnostics.restype = ctypes.c_int
_lib.lbm_batch_get_f.argtypes = [_ctx_p, ctypes.c_int, _fp]
_lib.lbm_batch_get_f.restype = ctypes.c_int
_lib.lbm_batch_set_f.argtypes = [_ctx_p, ctypes.c_int, _fp]
_lib.lbm_batch_set_f.restype = ctypes.c_int
_lib.lbm_set_graphs.argtypes = [_ctx_p, ctypes.c_int]
_lib.lbm_set_graphs.restype = ctypes.c_int
_lib.lbm_batch_footprint.argtypes = [_ctx_p, ctypes.c_int, ctypes.c_int, _fp]
_lib.lbm_batch_footprint.restype = ctypes.c_int
_mlp_p = ctypes.c_void_p
_lib.lbm_mlp_create.argtypes = [ctypes.c_int] * 5 + [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
_lib.lbm_mlp_create.restype = ctypes.c_int
_lib.lbm_mlp_num_params.argtypes = [_mlp_p]
_lib.lbm_mlp_num_params.restype = ctypes.c_size_t
_lib.lbm_mlp_set_params.argtypes = [_mlp_p, _fp]
_lib.lbm_mlp_set_params.restype = ctypes.c_int
_lib.lbm_mlp_get_params.argtypes = [_mlp_p, _fp]
_lib.lbm_mlp_get_params.restype = ctypes.c_int
_lib.lbm_mlp_forward.argtypes = [_mlp_p, _fp, ctypes.c_int, _fp]
_lib.lbm_mlp_forward.restype = ctypes.c_int
_lib.lbm_mlp_loss_grad.argtypes = [_mlp_p, _fp, _fp, ctypes.c_int, _fp, _fp]
_lib.lbm_mlp_loss_grad.restype = ctypes.c_int
_lib.lbm_mlp_train_step.argtypes = [_mlp_p, _fp, _fp, ctypes.c_int, ctypes.c_float, _fp]
_lib.lbm_mlp_train_step.restype = ctypes.c_int
_lib.lbm_mlp_destroy.argtypes = [_mlp_p]
_lib.lbm_mlp_destroy.restype = None
_lib.lbm_mlp_last_error.argtypes = [_mlp_p]
_lib.lbm_mlp_last_error.restype = ctypes.c_char_p
_lib.lbm_gemm_bf16.argtypes = [_fp, ctypes.c_longlong, ctypes.c_longlong, _fp, ctypes.c_longlong,
                               ctypes.c_longlong, _fp, ctypes.c_longlong, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, _fp, ctypes.c_void_p]
_lib.lbm_gemm_bf16.restype = ctypes.c_int
_lib.lbm_default_fused_config.argtypes = [ctypes.POINTER(LbmParams), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]
_lib.lbm_default_fused_config.restype = ctypes.c_int
_lib.lbm_step_noalloc.argtypes = [ctypes.POINTER(LbmParams), _fp, _fp, ctypes.c_void_p]
_lib.lbm_step_noalloc.restype = ctypes.c_int
_lib.lbm_inplace_init.argtypes = [ctypes.POINTER(LbmParams), _fp, _fp, _fp, _fp,
                                  ctypes.c_void_p]
_lib.lbm_inplace_init.restype = ctypes.c_int
_lib.lbm_inplace_set.argtypes = [ctypes.POINTER(LbmParams), _fp, _fp, ctypes.c_void_p]
_lib.lbm_inplace_set.restype = ctypes.c_int
_lib.lbm_step_inplace.argtypes = [ctypes.POINTER(LbmParams), _fp, ctypes.c_int, ctypes.c_int,
                                  _fp, ctypes.c_void_p]
_lib.lbm_step_inplace.restype = ctypes.c_int
_lib.lbm_inplace_read.argtypes = [ctypes.POINTER(LbmParams), _fp, ctypes.c_int, _fp, _fp, _fp,
                                  _fp, ctypes.c_void_p]
_lib.lbm_inplace_read.restype = ctypes.c_int
_lib.lbm_launches_per_step.argtypes = [_ctx_p]
_lib.lbm_launches_per_step.restype = ctypes.c_int
_lib.lbm_destroy.argtypes = [_ctx_p]
_lib.lbm_destroy.restype = None
_lib.lbm_last_error.argtypes = [_ctx_p]
_lib.lbm_last_error.restype = ctypes.c_char_p

EXPORTED = ("lbm_create", "lbm_init_fields", "lbm_step", "lbm_moments",
            "lbm_diagnostics", "lbm_step_diagnostics_async", "lbm_step_monitored", "lbm_sync", "lbm_get_f", "lbm_set_f", "lbm_population_bytes",
            "lbm_get_populations", "lbm_set_populations", "lbm_plane_bytes",
            "lbm_get_planes", "lbm_set_planes",
            "lbm_set_fused_config", "lbm_get_fused_config", "lbm_default_fused_config",
            "lbm_step_noalloc",
            "lbm_inplace_init", "lbm_inplace_set", "lbm_step_inplace", "lbm_inplace_read",
            "lbm_create_batch", "lbm_num_cases", "lbm_batch_init_fields",
            "lbm_batch_moments", "lbm_batch_diagnostics", "lbm_batch_get_f",
            "lbm_batch_set_f", "lbm_batch_footprint", "lbm_set_graphs", "lbm_mlp_create", "lbm_mlp_num_params",
            "lbm_mlp_set_params", "lbm_mlp_get_params", "lbm_mlp_forward",
            "lbm_mlp_loss_grad", "lbm_mlp_train_step", "lbm_mlp_destroy",
            "lbm_mlp_last_error", "lbm_gemm_bf16",
            "lbm_launches_per_step", "lbm_destroy", "lbm_last_error")


def lbm_last_error(ctx) -> str:
    msg = _lib.lbm_last_error(ctx)
    return msg.decode() if msg else ""


def _check(ctx, status):
    if status != LBM_OK:
        raise LbmError(status, lbm_last_error(ctx))


def make_params(nx, ny, nz, *, wall=(0, 0, 0), improved=True, storage="f32",
                kernel="fused", rho_in_R=1.0, rho_in_B=1.0, alpha_R=1.0 / 3.0,
                alpha_B=1.0 / 3.0, tau_R=1.0, tau_B=1.0, tau_e=1.0, tau_q=1.0,
                tau_pi=1.0, A_R=0.0, A_B=0.0, beta=0.7, delta=0.98,
                force=(0.0, 0.0, 0.0), gravity=(0.0, 0.0, 0.0), ref_R=0.0,
                ref_B=0.0, wetting=False, contact_angle_deg=90.0, collision="mrt",
                wall_u=((0.0, 0.0, 0.0), (0.0, 0.0, 0.0)), **_ignored) -> LbmParams:
    p = LbmParams()
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    for a in range(3):
        p.wall[a] = int(wall[a])
        p.force[a] = float(force[a])
        p.gravity[a] = float(gravity[a])
    p.improved = 1 if improved else 0
    p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    p.kernel = {"fused": LBM_KERNEL_FUSED, "two_pass": LBM_KERNEL_TWO_PASS}[kernel] \
        if isinstance(kernel, str) else int(kernel)
    p.wetting = 1 if wetting else 0
    p.contact_angle_deg = float(contact_angle_deg)
    p.collision = COLLISION[collision] if isinstance(collision, str) else int(collision)
    for side in range(2):
        for a in range(3):
            p.wall_u[side][a] = float(wall_u[side][a])
    p.rho_in_R, p.rho_in_B = float(rho_in_R), float(rho_in_B)
    p.alpha_R, p.alpha_B = float(alpha_R), float(alpha_B)
    p.tau_R, p.tau_B = float(tau_R), float(tau_B)
    p.tau_e, p.tau_q, p.tau_pi = float(tau_e), float(tau_q), float(tau_pi)
    p.A_R, p.A_B = float(A_R), float(A_B)
    p.beta, p.delta = float(beta), float(delta)
    p.ref_R, p.ref_B = float(ref_R), float(ref_B)
    return p


def _addr(x):
    """Address of a torch tensor, numpy array or raw integer (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor arguments must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array arguments must be C-contiguous")
        return x.ctypes.data
    return int(x)


def lbm_create(params: LbmParams, stream=None):
    ctx = ctypes.c_void_p()
    s = ctypes.c_void_p(stream) if stream else None
    st = _lib.lbm_create(ctypes.byref(params), s, ctypes.byref(ctx))
    if st != LBM_OK:
        raise LbmError(st, lbm_last_error(None))
    return ctx


def lbm_create_batch(params_list, stream=None):
    arr = (LbmParams * len(params_list))(*params_list)
    ctx = ctypes.c_void_p()
    s = ctypes.c_void_p(stream) if stream else None
    st = _lib.lbm_create_batch(arr, len(params_list), s, ctypes.byref(ctx))
    if st != LBM_OK:
        raise LbmError(st, lbm_last_error(None))
    return ctx


def lbm_num_cases(ctx) -> int:
    return int(_lib.lbm_num_cases(ctx))


def lbm_batch_init_fields(ctx, case, rho_R, rho_B, u):
    _check(ctx, _lib.lbm_batch_init_fields(ctx, int(case), _addr(rho_R), _addr(rho_B),
                                           _addr(u)))


def lbm_batch_moments(ctx, case, rho_R, rho_B, u):
    _check(ctx, _lib.lbm_batch_moments(ctx, int(case), _addr(rho_R), _addr(rho_B),
                                       _addr(u)))


def lbm_batch_diagnostics(ctx, case, raise_unstable=True):
    out = (ctypes.c_double * 16)()
    st = _lib.lbm_batch_diagnostics(ctx, int(case), out)
    if st != LBM_OK and (raise_unstable or st != LBM_ERR_UNSTABLE):
        raise LbmError(st, lbm_last_error(ctx))
    return np.array(out[:], dtype=np.float64)


def lbm_batch_get_f(ctx, case, f):
    _check(ctx, _lib.lbm_batch_get_f(ctx, int(case), _addr(f)))


def lbm_batch_set_f(ctx, case, f):
    _check(ctx, _lib.lbm_batch_set_f(ctx, int(case), _addr(f)))


def lbm_set_graphs(ctx, enable):
    _check(ctx, _lib.lbm_set_graphs(ctx, 1 if enable else 0))


def lbm_init_fields(ctx, rho_R, rho_B, u, solid=None):
    _check(ctx, _lib.lbm_init_fields(ctx, _addr(rho_R), _addr(rho_B), _addr(u),
                                     _addr(solid)))


def lbm_step(ctx, n=1):
    _check(ctx, _lib.lbm_step(ctx, int(n)))


def lbm_moments(ctx, rho_R, rho_B, u):
    _check(ctx, _lib.lbm_moments(ctx, _addr(rho_R), _addr(rho_B), _addr(u)))


def lbm_diagnostics(ctx, raise_unstable=True):
    out = (ctypes.c_double * 16)()
    st = _lib.lbm_diagnostics(ctx, out)
    if st != LBM_OK and (raise_unstable or st != LBM_ERR_UNSTABLE):
        raise LbmError(st, lbm_last_error(ctx))
    return np.array(out[:], dtype=np.float64)


def lbm_step_diagnostics_async(ctx, n, out):
    """Queues n steps, the diagnostics of the state they reach and their
    copy into ``out`` (16 float64: a pinned CPU tensor or a device tensor);
    ``out`` is valid after :func:`lbm_sync`."""
    if isinstance(out, torch.Tensor) and (out.dtype != torch.float64 or out.numel() < 16):
        raise ValueError("out must hold 16 float64 values")
    _check(ctx, _lib.lbm_step_diagnostics_async(ctx, int(n), _addr(out)))


def lbm_step_monitored(ctx, n, out):
    """Queues n steps, step k reporting the diagnostics of the state it
    reads into ``out[k]`` (16 float64 per step: a pinned CPU tensor or a
    device tensor of at least 16 n values); ``out`` is valid after
    :func:`lbm_sync`."""
    if isinstance(out, torch.Tensor) and (out.dtype != torch.float64 or
                                          out.numel() < 16 * int(n)):
        raise ValueError("out must hold 16 n float64 values")
    _check(ctx, _lib.lbm_step_monitored(ctx, int(n), _addr(out)))


def lbm_sync(ctx):
    _check(ctx, _lib.lbm_sync(ctx))


def lbm_get_f(ctx, f):
    _check(ctx, _lib.lbm_get_f(ctx, _addr(f)))


def lbm_set_f(ctx, f):
    _check(ctx, _lib.lbm_set_f(ctx, _addr(f)))


def lbm_population_bytes(ctx) -> int:
    return int(_lib.lbm_population_bytes(ctx))


def lbm_get_populations(ctx, dst):
    _check(ctx, _lib.lbm_get_populations(ctx, _addr(dst)))


def lbm_set_populations(ctx, src):
    _check(ctx, _lib.lbm_set_populations(ctx, _addr(src)))


def lbm_plane_bytes(ctx) -> int:
    return int(_lib.lbm_plane_bytes(ctx))


def lbm_get_planes(ctx, z0, n, dst):
    _check(ctx, _lib.lbm_get_planes(ctx, int(z0), int(n), _addr(dst)))


def lbm_set_planes(ctx, z0, n, src):
    _check(ctx, _lib.lbm_set_planes(ctx, int(z0), int(n), _addr(src)))


def lbm_set_fused_config(ctx, tile_y, zchunk, hold):
    _check(ctx, _lib.lbm_set_fused_config(ctx, int(tile_y), int(zchunk), int(hold)))


def lbm_get_fused_config(ctx):
    v = [ctypes.c_int() for _ in range(3)]
    _check(ctx, _lib.lbm_get_fused_config(ctx, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def lbm_default_fused_config(params: LbmParams, sms=0):
    """(tile_y, zchunk, hold) lbm_create would pick for this single lattice
    on a GPU with `sms` SMs (0: 152); host only, no GPU needed."""
    v = [ctypes.c_int() for _ in range(3)]
    st = _lib.lbm_default_fused_config(ctypes.byref(params), int(sms),
                                       *[ctypes.byref(x) for x in v])
    if st != LBM_OK:
        raise LbmError(st, lbm_last_error(None))
    return tuple(x.value for x in v)


def lbm_step_noalloc(params: LbmParams, f_in, f_out, stream=None):
    """One step on caller-owned device arrays (float32 [2][19][N] each)
    without any device allocation; see include/lbm.h for its limits."""
    s = ctypes.c_void_p(stream) if stream else None
    st = _lib.lbm_step_noalloc(ctypes.byref(params), _addr(f_in), _addr(f_out), s)
    if st != LBM_OK:
        raise LbmError(st, lbm_last_error(None))


def _stream_arg(stream):
    return ctypes.c_void_p(stream) if stream else None


def _inplace_check(st):
    if st != LBM_OK:
        raise LbmError(st, lbm_last_error(None))


def lbm_inplace_init(params: LbmParams, rho_R, rho_B, u, f, stream=None):
    """Equilibrium populations of the fields into f ([2][19][N] values of
    params.storage, device) as an even in-place state; see include/lbm.h."""
    _inplace_check(_lib.lbm_inplace_init(ctypes.byref(params), _addr(rho_R), _addr(rho_B),
                                         _addr(u), _addr(f), _stream_arg(stream)))


def lbm_inplace_set(params: LbmParams, f_in, f, stream=None):
    """An even in-place state f from float32 populations f_in [2][19][N]
    (stored in params.storage's format)."""
    _inplace_check(_lib.lbm_inplace_set(ctypes.byref(params), _addr(f_in), _addr(f),
                                        _stream_arg(stream)))


def lbm_step_inplace(params: LbmParams, f, parity, nsteps, scratch, stream=None):
    """nsteps in-place steps of the state f of the given parity; returns the
    new parity.  scratch: 16 bytes per cell of device memory."""
    _inplace_check(_lib.lbm_step_inplace(ctypes.byref(params), _addr(f), int(parity),
                                         int(nsteps), _addr(scratch), _stream_arg(stream)))
    return (int(parity) + int(nsteps)) & 1


def lbm_inplace_read(params: LbmParams, f, parity, f_out=None, rho_R=None, rho_B=None,
                     u=None, stream=None):
    """f_i^k(x, t) in the even layout and / or the moments of an in-place
    state of either parity."""
    _inplace_check(_lib.lbm_inplace_read(ctypes.byref(params), _addr(f), int(parity),
                                         _addr(f_out), _addr(rho_R), _addr(rho_B), _addr(u),
                                         _stream_arg(stream)))


def _mlp_check(m, st):
    if st != LBM_OK:
        msg = _lib.lbm_mlp_last_error(m)
        raise LbmError(st, msg.decode() if msg else "")


def lbm_mlp_create(n_in, width, depth, n_out, max_batch, stream=None):
    m = ctypes.c_void_p()
    s = ctypes.c_void_p(stream) if stream else None
    _mlp_check(None, _lib.lbm_mlp_create(n_in, width, depth, n_out, max_batch, s,
                                         ctypes.byref(m)))
    return m


def lbm_mlp_num_params(m) -> int:
    return int(_lib.lbm_mlp_num_params(m))


def lbm_mlp_set_params(m, theta):
    _mlp_check(m, _lib.lbm_mlp_set_params(m, _addr(theta)))


def lbm_mlp_get_params(m, theta):
    _mlp_check(m, _lib.lbm_mlp_get_params(m, _addr(theta)))


def lbm_mlp_forward(m, x, batch, y):
    _mlp_check(m, _lib.lbm_mlp_forward(m, _addr(x), int(batch), _addr(y)))


def lbm_mlp_loss_grad(m, x, t, batch, grad=None):
    loss = ctypes.c_float()
    _mlp_check(m, _lib.lbm_mlp_loss_grad(m, _addr(x), _addr(t), int(batch),
                                         ctypes.addressof(loss), _addr(grad)))
    return float(loss.value)


def lbm_mlp_train_step(m, x, t, batch, lr, want_loss=False):
    loss = ctypes.c_float()
    _mlp_check(m, _lib.lbm_mlp_train_step(m, _addr(x), _addr(t), int(batch), float(lr),
                                          ctypes.addressof(loss) if want_loss else None))
    return float(loss.value) if want_loss else None


def lbm_mlp_destroy(m):
    _lib.lbm_mlp_destroy(m)


def lbm_gemm_bf16(A, sa_m, sa_k, B, sb_k, sb_n, C, sc_m, M, N, K, err, stream=None):
    s = ctypes.c_void_p(stream) if stream else None
    st = _lib.lbm_gemm_bf16(_addr(A), sa_m, sa_k, _addr(B), sb_k, sb_n, _addr(C), sc_m,
                            M, N, K, _addr(err), s)
    if st != LBM_OK:
        raise LbmError(st, "lbm_gemm_bf16 failed")


def lbm_launches_per_step(ctx) -> int:
    return int(_lib.lbm_launches_per_step(ctx))


def lbm_destroy(ctx):
    _lib.lbm_destroy(ctx)


class Lattice:
    """One lattice on one device, bound to the current torch stream of that
    device at construction."""

    def __init__(self, params: LbmParams, device=None, stream=None):
        self.device = torch.device(device or "cuda")
        self.params = params
        with torch.cuda.device(self.device):
            self.stream = stream or torch.cuda.current_stream(self.device)
            self.ctx = lbm_create(params, self.stream.cuda_stream)
        self.shape = (params.nz, params.ny, params.nx)
        self.N = params.nx * params.ny * params.nz

    def _t(self, x):
        if isinstance(x, torch.Tensor):
            return x.to(device=self.device, dtype=torch.float32).contiguous()
        return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32,
                               device=self.device)

    def _after_caller(self):
        """Orders this object's stream after the work queued so far on the
        caller's current stream: tensors made there (or memory freed there)
        are only touched by the library once that work is done."""
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def init_fields(self, rho_R, rho_B, u):
        rR, rB, uu = self._t(rho_R), self._t(rho_B), self._t(u)
        self._after_caller()
        lbm_init_fields(self.ctx, rR, rB, uu)
        self._keep = (rR, rB, uu)  # alive until the queued kernel has read them
        self.stream.synchronize()

    def set_f(self, f):
        ft = self._t(f)
        self._after_caller()
        lbm_set_f(self.ctx, ft)
        self.stream.synchronize()

    def get_f(self):
        out = torch.empty((2, 19) + self.shape, dtype=torch.float32, device=self.device)
        self._after_caller()
        lbm_get_f(self.ctx, out)
        self.stream.synchronize()
        return out

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def moments(self):
        rR = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        rB = torch.empty_like(rR)
        u = torch.empty((3,) + self.shape, dtype=torch.float32, device=self.device)
        self._after_caller()
        lbm_moments(self.ctx, rR, rB, u)
        self.stream.synchronize()
        return rR, rB, u

    def diagnostics(self, raise_unstable=True):
        return lbm_diagnostics(self.ctx, raise_unstable)

    def close(self):
        if self.ctx is not None:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class InPlaceLattice:
    """One lattice stepped in place (one population array, AA access
    pattern): 168 bytes of device memory per cell instead of 304 in FP32 (92
    instead of 152 in FP16 / BF16 deviation storage), no limit on the cell
    count beyond memory.  Walls 0 or 1."""

    def __init__(self, params: LbmParams, device=None, stream=None):
        self.device = torch.device(device or "cuda")
        self.params = params
        self.shape = (params.nz, params.ny, params.nx)
        self.N = params.nx * params.ny * params.nz
        with torch.cuda.device(self.device):
            self.stream = stream or torch.cuda.current_stream(self.device)
        dt = {STORAGE["f32"]: torch.float32, STORAGE["f16"]: torch.float16,
              STORAGE["bf16"]: torch.bfloat16}[params.storage]
        self.f = torch.empty((2, 19) + self.shape, dtype=dt, device=self.device)
        self.scratch = torch.empty((self.N, 4), dtype=torch.float32, device=self.device)
        # used on self.stream: the allocator must not reuse the memory while
        # work queued there may still touch it
        self.f.record_stream(self.stream)
        self.scratch.record_stream(self.stream)
        self.parity = 0
        self._after_caller()

    def _t(self, x):
        if isinstance(x, torch.Tensor):
            return x.to(device=self.device, dtype=torch.float32).contiguous()
        return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32,
                               device=self.device)

    def _after_caller(self):
        """Orders this object's stream after the work queued so far on the
        caller's current stream: tensors made there (or memory freed there)
        are only touched by the library once that work is done."""
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def init_fields(self, rho_R, rho_B, u):
        rR, rB, uu = self._t(rho_R), self._t(rho_B), self._t(u)
        self._after_caller()
        lbm_inplace_init(self.params, rR, rB, uu, self.f, self.stream.cuda_stream)
        self.parity = 0
        self.stream.synchronize()

    def set_f(self, f):
        """Sets an even state: f_i^k(x, t) as float32 [2][19][N] (stored in
        the lattice's storage format)."""
        ft = self._t(f).reshape(self.f.shape)
        self._after_caller()
        lbm_inplace_set(self.params, ft, self.f, self.stream.cuda_stream)
        self.parity = 0
        self.stream.synchronize()

    def step(self, n=1):
        self.parity = lbm_step_inplace(self.params, self.f, self.parity, n, self.scratch,
                                       self.stream.cuda_stream)

    def get_f(self):
        out = torch.empty(self.f.shape, dtype=torch.float32, device=self.device)
        self._after_caller()
        lbm_inplace_read(self.params, self.f, self.parity, f_out=out,
                         stream=self.stream.cuda_stream)
        self.stream.synchronize()
        return out

    def moments(self):
        rR = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        rB = torch.empty_like(rR)
        u = torch.empty((3,) + self.shape, dtype=torch.float32, device=self.device)
        self._after_caller()
        lbm_inplace_read(self.params, self.f, self.parity, rho_R=rR, rho_B=rB, u=u,
                         stream=self.stream.cuda_stream)
        self.stream.synchronize()
        return rR, rB, u

    def close(self):
        """Releases the population array and the scratch (after the work
        queued on the lattice's stream)."""
        if self.f is not None:
            self.stream.synchronize()
        self.f = None
        self.scratch = None


class Batch:
    """Many independent lattices on one device, advanced together by
    lbm_step (one kernel launch per step over all cases)."""

    def __init__(self, params_list, device=None, stream=None):
        self.device = torch.device(device or "cuda")
        self.params = list(params_list)
        with torch.cuda.device(self.device):
            self.stream = stream or torch.cuda.current_stream(self.device)
            self.ctx = lbm_create_batch(self.params, self.stream.cuda_stream)
        self.shapes = [(p.nz, p.ny, p.nx) for p in self.params]

    def _t(self, x):
        if isinstance(x, torch.Tensor):
            return x.to(device=self.device, dtype=torch.float32).contiguous()
        return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32,
                               device=self.device)

    def _after_caller(self):
        """Orders this object's stream after the work queued so far on the
        caller's current stream: tensors made there (or memory freed there)
        are only touched by the library once that work is done."""
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def init_fields(self, case, rho_R, rho_B, u):
        rR, rB, uu = self._t(rho_R), self._t(rho_B), self._t(u)
        self._after_caller()
        lbm_batch_init_fields(self.ctx, case, rR, rB, uu)
        self.stream.synchronize()

    def set_f(self, case, f):
        ft = self._t(f)
        self._after_caller()
        lbm_batch_set_f(self.ctx, case, ft)
        self.stream.synchronize()

    def get_f(self, case):
        out = torch.empty((2, 19) + self.shapes[case], dtype=torch.float32,
                          device=self.device)
        self._after_caller()
        lbm_batch_get_f(self.ctx, case, out)
        self.stream.synchronize()
        return out

    def moments(self, case):
        shape = self.shapes[case]
        rR = torch.empty(shape, dtype=torch.float32, device=self.device)
        rB = torch.empty_like(rR)
        u = torch.empty((3,) + shape, dtype=torch.float32, device=self.device)
        self._after_caller()
        lbm_batch_moments(self.ctx, case, rR, rB, u)
        self.stream.synchronize()
        return rR, rB, u

    def diagnostics(self, case, raise_unstable=True):
        return lbm_batch_diagnostics(self.ctx, case, raise_unstable)

    def footprint(self, axis=2, index=0):
        """Red-dominated cell count of one plane, per case (int64 array)."""
        out = np.zeros(len(self.params), dtype=np.int64)
        _check(self.ctx, _lib.lbm_batch_footprint(self.ctx, int(axis), int(index),
                                                  out.ctypes.data))
        return out

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def close(self):
        if self.ctx is not None:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
