"""lbm_default_fused_config: the launch configuration lbm_create picks,
computed on the host.

Pinned to the configurations live contexts reported (lbm_get_fused_config)
on a GB300 (152 SMs) for the same lattices; the seam form's z chunk is
checked against a naive CTA-by-CTA simulation of the list schedule it
models (one CTA per SM, CTAs handed out in launch order -- tile columns
fastest, then z chunks -- to the SM that falls free first, each costing its
planes + 3 plane-times), over many lattice shapes and SM counts."""
import heapq

import pytest

from paper_1904_03618_gb300 import lbm


def _droplet(n, **kw):
    d = dict(nx=n, ny=n, nz=n, wall=(0, 0, 0), rho_in_R=10.0, rho_in_B=1.0,
             alpha_R=0.97, alpha_B=0.7, A_R=0.01125, A_B=0.01125)
    d.update(kw)
    return d


@pytest.mark.parametrize("kw,want", [
    (_droplet(128), (12, 24, 7)),
    (_droplet(160), (12, 46, 7)),
    (_droplet(192), (12, 39, 7)),
    (_droplet(256), (12, 48, 7)),
    (_droplet(256, nz=1024, wall=(0, 0, 1)), (12, 48, 7)),   # Rayleigh-Taylor lattice
    (_droplet(128, storage="f16"), (15, 37, 7)),    # the 16-bit seam form, two stages
    (_droplet(128, wall=(1, 1, 0)), (15, 12, 7)),
])
def test_matches_the_configurations_live_contexts_reported(kw, want):
    d = dict(kw)
    nx, ny, nz = d.pop("nx"), d.pop("ny"), d.pop("nz")
    p = lbm.make_params(nx, ny, nz, **d)
    assert lbm.lbm_default_fused_config(p, 152) == want
    assert lbm.lbm_default_fused_config(p, 0) == want        # 0 means 152


def _span(cols, nz, zc, sms, overhead=3.0):
    heap = [0.0] * sms
    for k in range((nz + zc - 1) // zc):
        planes = min(zc, nz - k * zc)
        for _ in range(cols):
            t = heapq.heappop(heap)
            heapq.heappush(heap, t + planes + overhead)
    return max(heap)


@pytest.mark.parametrize("nx,ny,nz,sms", [
    (128, 128, 128, 152), (160, 160, 160, 152), (96, 64, 200, 152), (256, 40, 77, 152),
    (64, 64, 64, 152), (128, 128, 128, 132), (34, 15, 9, 152), (192, 96, 300, 80),
    (512, 512, 64, 152), (40, 30, 500, 16),
])
def test_seam_chunk_is_the_shortest_list_schedule(nx, ny, nz, sms):
    p = lbm.make_params(nx, ny, nz)
    tile_y, zchunk, hold = lbm.lbm_default_fused_config(p, sms)
    assert (tile_y, hold) == (12, 7)
    cols = ((nx + 31) // 32) * ((ny + 9) // 10)
    spans = {zc: _span(cols, nz, zc, sms) for zc in range(6, 49)}
    best = min(spans.values())
    want = max(zc for zc, s in spans.items() if s <= best + 1e-9)   # ties: the longer chunk
    assert zchunk == min(want, nz)


def test_forms_outside_the_seam_rules():
    # BGK and the two-pass kernel keep the shared-memory hold form
    assert lbm.lbm_default_fused_config(lbm.make_params(64, 64, 64, collision="bgk"))[::2] == (8, 2)
    assert lbm.lbm_default_fused_config(lbm.make_params(64, 64, 64, kernel="two_pass"))[::2] == (8, 2)
    # too narrow for the 34-wide seam tile
    assert lbm.lbm_default_fused_config(lbm.make_params(32, 64, 64))[0] != 12
    # odd nx: the x seam is not a 16-byte TMA coordinate
    assert lbm.lbm_default_fused_config(lbm.make_params(65, 64, 64))[::2] == (8, 2)
    for n in (1, 3, 5):                                    # the chunk never exceeds nz
        assert lbm.lbm_default_fused_config(lbm.make_params(64, 64, n))[1] <= n
    with pytest.raises(lbm.LbmError):
        lbm.lbm_default_fused_config(lbm.make_params(64, 64, 64), -1)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_default_fused_config(lbm.make_params(64, 64, 64, tau_R=0.2))


@pytest.mark.gpu
@pytest.mark.parametrize("kw", [
    _droplet(128), _droplet(160), _droplet(64, nz=200), _droplet(256, nz=1024, wall=(0, 0, 1)),
    _droplet(128, storage="f16"), _droplet(128, storage="bf16"), _droplet(128, wall=(1, 1, 0)),
    _droplet(96, wall=(1, 1, 1)), _droplet(64, collision="bgk"), _droplet(64, kernel="two_pass"),
])
def test_query_equals_the_live_context(kw):
    torch = pytest.importorskip("torch")
    d = dict(kw)
    nx, ny, nz = d.pop("nx"), d.pop("ny"), d.pop("nz")
    p = lbm.make_params(nx, ny, nz, **d)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    lat = lbm.Lattice(p, device=torch.device("cuda:0"))
    try:
        live = lbm.lbm_get_fused_config(lat.ctx)
    finally:
        lat.close()
    assert lbm.lbm_default_fused_config(p, sms) == live


# lbm_test_gemm_plan: the surrogate GEMM's launch plan for K <= 256, worked
# out by hand from the rule (TMA form for K-contiguous A with a 16-byte
# multiple row stride, a 16-byte aligned base, M >= 128 and K >= 32; column
# block halved while 2 * row tiles * blocks <= SMs and the halves keep 16
# columns, and in the TMA form until it is <= 128; CTAs per block = SMs /
# blocks, at most the row tiles).
# (M, N, K, sa_m, sa_k, aligned, sms) -> (form, columns, blocks, CTAs per block)
GEMM_PLANS = [
    ((65536, 256, 256, 256, 1, 1, 152), (1, 128, 2, 76)),       # forward H W
    ((65536, 256, 256, 256, 1, 1, 148), (1, 128, 2, 74)),
    ((65536, 256, 5, 5, 1, 1, 152), (0, 256, 1, 152)),          # input layer: 20-byte rows
    ((65536, 256, 256, 1, 65536, 1, 152), (0, 256, 1, 152)),    # A stored K x M
    ((65536, 256, 256, 256, 1, 0, 152), (0, 256, 1, 152)),      # A not 16-byte aligned
    ((300, 200, 130, 130, 1, 1, 152), (0, 32, 7, 3)),           # row stride 130 floats
    ((100, 64, 64, 64, 1, 1, 152), (0, 16, 4, 1)),              # less than one row tile
    ((256, 256, 256, 256, 1, 1, 152), (1, 16, 16, 2)),          # a batch-256 training layer
    ((40001, 200, 252, 252, 1, 1, 152), (1, 112, 2, 76)),       # ragged M, N and K
    # K > 256: the register form split into slices of 256 K (columns, slices,
    # CTAs per slice = SMs / slices, at most the row tiles)
    ((256, 256, 65536, 1, 256, 1, 152), (2, 256, 256, 1)),      # weight gradient H^T dZ
    ((257, 256, 1000, 1000, 1, 1, 152), (2, 256, 4, 3)),
    ((300, 200, 300, 300, 1, 1, 152), (2, 208, 2, 3)),
    ((4096, 64, 512, 512, 1, 1, 152), (2, 64, 2, 32)),
    ((16, 16, 65535 * 256 + 1, 1, 16, 1, 152), (3, 0, 0, 0)),   # too many slices
]


@pytest.mark.parametrize("args,want", GEMM_PLANS)
def test_gemm_launch_plan(args, want):
    import ctypes
    L = lbm._lib
    L.lbm_test_gemm_plan.argtypes = [ctypes.c_int] * 3 + [ctypes.c_longlong] * 2 + \
        [ctypes.c_int] * 2 + [ctypes.POINTER(ctypes.c_int)]
    L.lbm_test_gemm_plan.restype = ctypes.c_int
    out = (ctypes.c_int * 4)()
    assert L.lbm_test_gemm_plan(*args, out) == lbm.LBM_OK
    assert tuple(out) == want
    form, bn, nt, gx = want
    M, N, K = args[0], args[1], args[2]
    if form == 3:
        return
    assert bn % 16 == 0 and (bn <= 128 if form == 1 else bn <= 256)
    if form == 2:                                       # nt: the K slices
        assert (nt - 1) * 256 < K <= nt * 256 and bn >= N
        assert gx == max(1, min(args[6] // nt, (M + 127) // 128))
        return
    assert (nt - 1) * bn < N <= nt * bn                 # every column in one block
    assert nt * gx <= args[6] and gx <= (M + 127) // 128


def test_gemm_launch_plan_rejects_bad_arguments():
    import ctypes
    L = lbm._lib
    L.lbm_test_gemm_plan.argtypes = [ctypes.c_int] * 3 + [ctypes.c_longlong] * 2 + \
        [ctypes.c_int] * 2 + [ctypes.POINTER(ctypes.c_int)]
    L.lbm_test_gemm_plan.restype = ctypes.c_int
    out = (ctypes.c_int * 4)()
    for M, N, K, sms in [(0, 16, 16, 152), (16, 0, 16, 152), (16, 257, 16, 152),
                         (16, 16, 0, 152), (16, 16, 16, 0)]:
        assert L.lbm_test_gemm_plan(M, N, K, K, 1, 1, sms, out) == lbm.LBM_ERR_ARG
    assert L.lbm_test_gemm_plan(16, 16, 16, 16, 1, 1, 152, None) == lbm.LBM_ERR_ARG
