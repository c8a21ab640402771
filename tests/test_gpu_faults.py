"""Failure detection without a GPU fault.

  * Bounded device waits: a test shortens the give-up limit of the step
    kernels' waits for their tensor copies (and of the surrogate GEMM's waits
    for its tensor-core commits) to 1 ns through lbm_test_set_wait_limits;
    the waits give up, the kernels drain their own copies (or MMAs) at the
    full limit and leave, and the host call reports LBM_ERR_TIMEOUT.  The
    context stays usable: once its state is set anew it steps exactly as a
    fresh one.  Nothing traps, faults or hangs: every wait still ends.
  * Allocation failure: lbm_test_fail_allocation makes the n-th allocation
    of the library fail as cudaMalloc does when memory runs out; every
    failing creation returns LBM_ERR_OOM and leaves no allocation behind
    (live-allocation count and the device's free memory unchanged), and a
    lazily allocated staging buffer that fails leaves the context usable.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1904_03618_gb300 import lbm, workloads as wl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
L = lbm._lib
L.lbm_test_set_wait_limits.argtypes = [ctypes.c_ulonglong, ctypes.c_ulonglong]
L.lbm_test_set_wait_limits.restype = ctypes.c_int
L.lbm_test_fail_allocation.argtypes = [ctypes.c_int]
L.lbm_test_fail_allocation.restype = None
L.lbm_test_live_allocations.argtypes = []
L.lbm_test_live_allocations.restype = ctypes.c_longlong


def _params(nx, ny, nz, storage="f32", wall=(0, 0, 0)):
    return lbm.make_params(nx, ny, nz, storage=storage, wall=wall, rho_in_R=3.0,
                           rho_in_B=1.0, alpha_R=0.9, alpha_B=0.7, tau_R=1.0, tau_B=0.8,
                           A_R=0.01, A_B=0.01, beta=0.7)


def _fields(nx, ny, nz):
    return wl.droplet(nx, ny, nz, 6.0, 3.0, 1.0, velocity=(0.02, 0.0, 0.01), noise=1e-3,
                      seed=3)


def _diag_status(ctx):
    out = (ctypes.c_double * 16)()
    return L.lbm_diagnostics(ctx, out), out[14]


def _step_until_timeout(ctx, tries=6):
    """Steps with the 1 ns limit until a step reports a give-up."""
    assert L.lbm_test_set_wait_limits(1, 0) == lbm.LBM_OK
    try:
        for _ in range(tries):
            lbm.lbm_step(ctx, 1)
            st, word = _diag_status(ctx)
            if st == lbm.LBM_ERR_TIMEOUT:
                return word
    finally:
        assert L.lbm_test_set_wait_limits(0, 0) == lbm.LBM_OK
    return None


@pytest.mark.parametrize("shape,storage,wall", [
    ((64, 40, 36), "f32", (0, 0, 0)),    # seam form, two stages
    ((64, 40, 36), "f32", (0, 0, 1)),    # seam form, walls in z
    ((64, 40, 36), "f16", (0, 0, 0)),    # 16-bit TMA form
])
def test_stage_wait_give_up_is_reported_and_the_context_recovers(shape, storage, wall):
    nx, ny, nz = shape
    p = _params(nx, ny, nz, storage, wall)
    if storage != "f32":
        p.ref_R, p.ref_B = 0.0, 1.0
    rR, rB, u = _fields(nx, ny, nz)
    lat = lbm.Lattice(p, device=DEV, stream=torch.cuda.Stream(DEV))
    ref = lbm.Lattice(p, device=DEV, stream=torch.cuda.Stream(DEV))
    try:
        assert lbm.lbm_get_fused_config(lat.ctx)[2] in (7, 8)   # a TMA form runs
        lat.init_fields(rR, rB, u)
        lat.step(2)
        assert _diag_status(lat.ctx)[0] == lbm.LBM_OK
        word = _step_until_timeout(lat.ctx)
        assert word == 1.0                      # a stage wait gave up
        assert "bounded wait" in lbm.lbm_last_error(lat.ctx)
        # the report stays until the state is set anew ...
        lat.step(1)
        assert _diag_status(lat.ctx)[0] == lbm.LBM_ERR_TIMEOUT
        # ... after which the context steps exactly as a fresh one
        lat.init_fields(rR, rB, u)
        ref.init_fields(rR, rB, u)
        lat.step(3)
        ref.step(3)
        assert _diag_status(lat.ctx)[0] == lbm.LBM_OK
        assert torch.equal(lat.get_f(), ref.get_f())
    finally:
        lat.close()
        ref.close()


def test_batch_stage_wait_give_up_is_reported():
    plist = [_params(32, 32, 32), _params(48, 48, 48)]
    b = lbm.Batch(plist, device=DEV, stream=torch.cuda.Stream(DEV))
    try:
        assert lbm.lbm_get_fused_config(b.ctx)[2] in (7, 8)
        for k, p in enumerate(plist):
            b.init_fields(k, *_fields(p.nx, p.ny, p.nz))
        b.step(2)
        out = (ctypes.c_double * 16)()
        assert L.lbm_batch_diagnostics(b.ctx, 1, out) == lbm.LBM_OK
        assert L.lbm_test_set_wait_limits(1, 0) == lbm.LBM_OK
        try:
            got = False
            for _ in range(6):
                b.step(1)
                if L.lbm_batch_diagnostics(b.ctx, 0, out) == lbm.LBM_ERR_TIMEOUT:
                    got = True
                    break
        finally:
            assert L.lbm_test_set_wait_limits(0, 0) == lbm.LBM_OK
        assert got and out[14] == 1.0
    finally:
        b.close()


def test_tensor_core_wait_give_up_is_reported_and_the_network_recovers():
    torch.manual_seed(0)
    s = torch.cuda.Stream(DEV)
    m = lbm.lbm_mlp_create(5, 256, 4, 16, 8192, s.cuda_stream)
    try:
        n = lbm.lbm_mlp_num_params(m)
        theta = (torch.randn(n) * 0.05).float()
        lbm.lbm_mlp_set_params(m, theta.numpy())
        x = torch.randn(8192, 5, device=DEV)
        y0 = np.zeros((8192, 16), dtype=np.float32)
        lbm.lbm_mlp_forward(m, x, 8192, y0)
        assert L.lbm_test_set_wait_limits(0, 1) == lbm.LBM_OK
        status = None
        try:
            for _ in range(6):
                y = np.zeros_like(y0)
                try:
                    lbm.lbm_mlp_forward(m, x, 8192, y)
                except lbm.LbmError as e:
                    status = e.status
                    break
        finally:
            assert L.lbm_test_set_wait_limits(0, 0) == lbm.LBM_OK
        assert status == lbm.LBM_ERR_TIMEOUT
        # the record stays until the parameters are set anew
        with pytest.raises(lbm.LbmError):
            lbm.lbm_mlp_forward(m, x, 8192, np.zeros_like(y0))
        lbm.lbm_mlp_set_params(m, theta.numpy())
        y1 = np.zeros_like(y0)
        lbm.lbm_mlp_forward(m, x, 8192, y1)
        assert np.array_equal(y0, y1)
    finally:
        lbm.lbm_mlp_destroy(m)


def _create(p_list):
    ctx = ctypes.c_void_p()
    if len(p_list) == 1:
        st = L.lbm_create(ctypes.byref(p_list[0]), None, ctypes.byref(ctx))
    else:
        arr = (lbm.LbmParams * len(p_list))(*p_list)
        st = L.lbm_create_batch(arr, len(p_list), None, ctypes.byref(ctx))
    return st, ctx


@pytest.mark.parametrize("kind", ["single", "two_pass", "batch"])
def test_every_failed_allocation_of_create_reports_oom_and_leaks_nothing(kind):
    torch.cuda.synchronize()
    if kind == "single":
        plist = [_params(64, 40, 36)]
    elif kind == "two_pass":
        plist = [lbm.make_params(20, 12, 9, kernel="two_pass")]
    else:
        plist = [_params(32, 32, 32), _params(48, 32, 16)]
    base = L.lbm_test_live_allocations()
    st, ctx = _create(plist)
    assert st == lbm.LBM_OK
    made = L.lbm_test_live_allocations() - base
    lbm.lbm_destroy(ctx)
    assert L.lbm_test_live_allocations() == base
    assert made >= 6
    free0 = torch.cuda.mem_get_info(DEV)[0]
    ooms = 0
    for n in range(1, made + 1):
        L.lbm_test_fail_allocation(n)
        st, ctx = _create(plist)
        L.lbm_test_fail_allocation(0)
        if st == lbm.LBM_OK:
            # an optional allocation (one of a batch's six tensor-map
            # tables) degraded the launch form instead
            assert kind == "batch"
            lbm.lbm_destroy(ctx)
        else:
            assert st == lbm.LBM_ERR_OOM
            assert "cudaMalloc" in lbm.lbm_last_error(None)
            ooms += 1
        assert L.lbm_test_live_allocations() == base
    assert ooms >= made - (6 if kind == "batch" else 0)
    assert torch.cuda.mem_get_info(DEV)[0] == free0


def test_failed_staging_allocation_leaves_the_context_usable():
    nx, ny, nz = 40, 36, 20
    p = _params(nx, ny, nz)
    rR, rB, u = (np.ascontiguousarray(a, dtype=np.float32) for a in _fields(nx, ny, nz))
    ctx = lbm.lbm_create(p)
    try:
        live = L.lbm_test_live_allocations()
        L.lbm_test_fail_allocation(1)       # the staging buffer for host fields
        try:
            with pytest.raises(lbm.LbmError) as ei:
                lbm.lbm_init_fields(ctx, rR, rB, u)
        finally:
            L.lbm_test_fail_allocation(0)
        assert ei.value.status == lbm.LBM_ERR_OOM
        assert L.lbm_test_live_allocations() == live
        lbm.lbm_init_fields(ctx, rR, rB, u)  # now it allocates and runs
        lbm.lbm_step(ctx, 2)
        assert lbm.lbm_diagnostics(ctx)[12] == 2
    finally:
        lbm.lbm_destroy(ctx)


def test_failed_network_creation_reports_oom_and_leaks_nothing():
    base = L.lbm_test_live_allocations()
    for n in range(1, 11):
        L.lbm_test_fail_allocation(n)
        try:
            with pytest.raises(lbm.LbmError) as ei:
                lbm.lbm_mlp_create(5, 64, 2, 8, 256)
        finally:
            L.lbm_test_fail_allocation(0)
        assert ei.value.status == lbm.LBM_ERR_OOM
        assert L.lbm_test_live_allocations() == base
    m = lbm.lbm_mlp_create(5, 64, 2, 8, 256)
    assert L.lbm_test_live_allocations() == base + 10
    lbm.lbm_mlp_destroy(m)
    assert L.lbm_test_live_allocations() == base
