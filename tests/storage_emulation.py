"""The 16-bit deviation storage of the GPU as a rounding applied to FP64
oracle states (test infrastructure): each population is stored as its
deviation from the FP32 offset ref_k phi_i^k, formed in FP32 and rounded to
FP16 or BF16 (nearest even), and read back as the widened value plus the
offset."""
import numpy as np


def rest_weights(alpha):
    """phi_i^k of the rest state (Eq. 5 at u = 0): alpha on the rest
    population, (1 - alpha) / 12 on the axes, (1 - alpha) / 24 on the
    diagonals (directions 1-6 and 7-18 of the oracle's order)."""
    w = np.empty(19)
    w[0] = alpha
    w[1:7] = (1.0 - alpha) / 12.0
    w[7:] = (1.0 - alpha) / 24.0
    return w


def offsets(pd, ref_R, ref_B):
    """FP32 offsets [colour][direction]."""
    return np.stack([(ref_R * rest_weights(pd["alpha_R"])).astype(np.float32),
                     (ref_B * rest_weights(pd["alpha_B"])).astype(np.float32)])


def to_bf16(x32):
    b = x32.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def stored(f, storage, off):
    """The populations (2, 19, ...) as the GPU holds them."""
    out = np.empty_like(f)
    for k in range(2):
        o = off[k].reshape((19,) + (1,) * (f.ndim - 2))
        d = f[k].astype(np.float32) - o
        r = d.astype(np.float16).astype(np.float32) if storage == "f16" else to_bf16(d)
        out[k] = (r + o).astype(np.float64)
    return out
