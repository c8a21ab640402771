"""Tensor-core surrogate network: the tcgen05 GEMM against an FP64 matrix
product of the same BF16-rounded operands, and the network's loss, gradient
and Adam step against the FP64 reference in ``oracle.mlp``."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import mlp as ref
from paper_1904_03618_gb300 import lbm

pytestmark = pytest.mark.gpu


def _bf16(a: np.ndarray) -> np.ndarray:
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).bfloat16().double().numpy()


def _gemm(A, B, transpose_a=False, transpose_b=False):
    """C = A @ B through lbm_gemm_bf16; A (M x K), B (K x N) as numpy arrays,
    passed with the requested storage order."""
    M, K = A.shape
    N = B.shape[1]
    if transpose_a:      # stored K x M: A(m, k) = At[k * M + m]
        Ad = torch.from_numpy(np.ascontiguousarray(A.T, dtype=np.float32)).cuda()
        sa_m, sa_k = 1, M
    else:
        Ad = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).cuda()
        sa_m, sa_k = K, 1
    if transpose_b:      # stored N x K: B(k, n) = Bt[n * K + k]
        Bd = torch.from_numpy(np.ascontiguousarray(B.T, dtype=np.float32)).cuda()
        sb_k, sb_n = 1, K
    else:
        Bd = torch.from_numpy(np.ascontiguousarray(B, dtype=np.float32)).cuda()
        sb_k, sb_n = N, 1
    C = torch.full((M, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    lbm.lbm_gemm_bf16(Ad, sa_m, sa_k, Bd, sb_k, sb_n, C, N, M, N, K, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return C.cpu().double().numpy()


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (128, 16, 64), (129, 17, 65), (300, 200, 130),
                                   (257, 256, 1000), (5, 256, 7), (1000, 64, 16),
                                   # several row tiles per persistent CTA: both
                                   # accumulators and every ring stage reused
                                   (40000, 256, 256), (40003, 16, 5), (20000, 100, 200),
                                   # the TMA-fed form (A K-contiguous, rows of a
                                   # 16-byte multiple): K ends inside a 32-k box,
                                   # M inside a row tile, column blocks < 128
                                   (1000, 48, 40), (333, 96, 100), (40001, 200, 252)])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_gemm_matches_fp64_product_of_bf16_operands(M, N, K, ta, tb):
    rng = np.random.default_rng(M * 7919 + N * 31 + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    C = _gemm(A, B, ta, tb)
    Ar, Br = _bf16(A), _bf16(B)
    exact = Ar @ Br
    # BF16 x BF16 products are exact in FP32, so any FP32 summation order
    # stays within the textbook bound K u sum|a||b| (u = 2^-24); 2x slack
    bound = max(K, 16) * 2.0 ** -23 * (np.abs(Ar) @ np.abs(Br)) + 1e-30
    assert np.all(np.isfinite(C))
    assert np.all(np.abs(C - exact) <= bound), float(np.max(np.abs(C - exact) / bound))


def test_gemm_rejects_bad_shapes():
    x = torch.zeros(16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for (M, N, K) in [(0, 1, 1), (1, 0, 1), (1, 257, 1), (1, 1, 0)]:
        with pytest.raises(lbm.LbmError):
            lbm.lbm_gemm_bf16(x, 1, 1, x, 1, 1, x, 1, M, N, K, err)


def _xavier(rng, n_in, width, depth, n_out):
    parts = []
    for a, b in ref.layer_shapes(n_in, width, depth, n_out):
        parts.append(rng.uniform(-1, 1, a * b) * np.sqrt(6.0 / (a + b)))
        parts.append(rng.uniform(-0.1, 0.1, b))
    return np.concatenate(parts)


def _layers(vec, n_in, width, depth, n_out):
    return [np.concatenate([W.ravel(), b]) for W, b in ref.unpack(vec, n_in, width, depth, n_out)]


@pytest.mark.parametrize("n_in,width,depth,n_out,batch",
                         [(5, 64, 3, 16, 300), (3, 256, 2, 8, 129), (7, 40, 0, 5, 50),
                          (5, 128, 4, 16, 1)])
def test_loss_and_gradient_match_oracle(n_in, width, depth, n_out, batch):
    rng = np.random.default_rng(n_in * 100 + width + depth)
    theta = _xavier(rng, n_in, width, depth, n_out)
    x = rng.uniform(-1, 1, (batch, n_in))
    t = rng.uniform(-1, 1, (batch, n_out))
    m = lbm.lbm_mlp_create(n_in, width, depth, n_out, max(batch, 64))
    try:
        P = lbm.lbm_mlp_num_params(m)
        assert P == ref.num_params(n_in, width, depth, n_out)
        th = np.ascontiguousarray(theta, dtype=np.float32)
        lbm.lbm_mlp_set_params(m, th)
        back = np.zeros(P, dtype=np.float32)
        lbm.lbm_mlp_get_params(m, back)
        assert np.array_equal(back, th)
        xd = torch.from_numpy(x.astype(np.float32)).cuda()
        td = torch.from_numpy(t.astype(np.float32)).cuda()
        y = np.zeros((batch, n_out), dtype=np.float32)
        lbm.lbm_mlp_forward(m, xd, batch, y)
        torch.cuda.synchronize()
        grad = np.zeros(P, dtype=np.float32)
        loss = lbm.lbm_mlp_loss_grad(m, xd, td, batch, grad)
    finally:
        lbm.lbm_mlp_destroy(m)
    theta32 = th.astype(np.float64)
    y_ref, _ = ref.forward(theta32, x.astype(np.float32).astype(np.float64), n_in, width, depth,
                           n_out)
    loss_ref, g_ref = ref.loss_and_grad(theta32, x.astype(np.float32).astype(np.float64),
                                        t.astype(np.float32).astype(np.float64), n_in, width,
                                        depth, n_out)
    # BF16 operands (relative rounding 2^-9) through a few layers
    scale = np.sqrt(np.mean(y_ref ** 2)) + 1e-12
    assert np.max(np.abs(y - y_ref)) <= 2e-2 * scale
    assert abs(loss - loss_ref) <= 2e-2 * loss_ref
    for gl, rl in zip(_layers(grad.astype(np.float64), n_in, width, depth, n_out),
                      _layers(g_ref, n_in, width, depth, n_out)):
        assert np.linalg.norm(gl - rl) <= 3e-2 * np.linalg.norm(rl) + 1e-7


def test_adam_step_matches_oracle():
    n_in, width, depth, n_out, batch = 4, 32, 2, 6, 96
    rng = np.random.default_rng(5)
    theta = _xavier(rng, n_in, width, depth, n_out).astype(np.float32)
    x = rng.uniform(-1, 1, (batch, n_in)).astype(np.float32)
    t = rng.uniform(-1, 1, (batch, n_out)).astype(np.float32)
    m = lbm.lbm_mlp_create(n_in, width, depth, n_out, batch)
    try:
        P = lbm.lbm_mlp_num_params(m)
        lbm.lbm_mlp_set_params(m, theta)
        xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
        g = np.zeros(P, dtype=np.float32)
        lbm.lbm_mlp_loss_grad(m, xd, td, batch, g)
        lr = 1e-3
        lbm.lbm_mlp_train_step(m, xd, td, batch, lr)
        after = np.zeros(P, dtype=np.float32)
        lbm.lbm_mlp_get_params(m, after)
    finally:
        lbm.lbm_mlp_destroy(m)
    # the device's own gradient through the reference Adam update
    want, _, _ = ref.adam_step(theta.astype(np.float64), g.astype(np.float64), np.zeros(P),
                               np.zeros(P), 1, lr)
    assert np.max(np.abs(after - want)) <= 1e-6 + 1e-5 * np.abs(want).max()
    # first Adam step moves every parameter with a non-negligible gradient by ~lr
    big = np.abs(g) > 1e-4
    assert np.allclose(np.abs(after - theta)[big], lr, rtol=2e-2)


def test_training_reduces_loss():
    n_in, width, depth, n_out, batch = 3, 64, 2, 4, 512
    rng = np.random.default_rng(11)
    x = rng.uniform(-1, 1, (batch, n_in)).astype(np.float32)
    t = np.stack([np.sin(2 * x[:, 0]) * x[:, 1], np.cos(x.sum(1)), x[:, 2] ** 2,
                  np.tanh(3 * x[:, 0] - x[:, 1])], axis=1).astype(np.float32)
    m = lbm.lbm_mlp_create(n_in, width, depth, n_out, batch)
    try:
        lbm.lbm_mlp_set_params(m, _xavier(rng, n_in, width, depth, n_out).astype(np.float32))
        xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
        first = lbm.lbm_mlp_loss_grad(m, xd, td, batch)
        for _ in range(1500):
            lbm.lbm_mlp_train_step(m, xd, td, batch, 3e-3)
        last = lbm.lbm_mlp_loss_grad(m, xd, td, batch)
    finally:
        lbm.lbm_mlp_destroy(m)
    assert last < first / 20, (first, last)


def test_batch_limits_and_errors():
    m = lbm.lbm_mlp_create(2, 8, 1, 2, 16)
    try:
        x = torch.zeros(64, device="cuda")
        y = np.zeros(64, dtype=np.float32)
        with pytest.raises(lbm.LbmError):
            lbm.lbm_mlp_forward(m, x, 17, y)
        with pytest.raises(lbm.LbmError):
            lbm.lbm_mlp_forward(m, x, 0, y)
    finally:
        lbm.lbm_mlp_destroy(m)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_mlp_create(2, 300, 1, 2, 16)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_mlp_create(0, 8, 1, 2, 16)
