"""Tensor-core building blocks (tcgen05 TF32 MMA from swizzled shared memory into
tensor memory, and the no-swizzle sliding-row operand form of the tensor-core belt)
against a host product, through the C ABI."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1211_3556_b300 as sk
    return sk, sk.Context(0), torch


def _run(sk, ctx, torch, A, B, passes):
    a = torch.from_numpy(np.ascontiguousarray(A, np.float32)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(B, np.float32)).cuda()
    d = torch.full((A.shape[0], B.shape[0]), float("nan"), device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = sk.lib()
    rc = L.sk_selftest_tc_gemm(ctx._h, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                               ctypes.c_void_p(d.data_ptr()), B.shape[0], A.shape[1], passes, st)
    assert rc == 0, L.sk_last_error()
    torch.cuda.synchronize()
    assert L.sk_get_status(ctx._h, st) == 0
    return d.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n,k", [(64, 64), (16, 32), (128, 96)])
def test_tf32_mma_exact_on_small_integers(env, n, k):
    sk, ctx, torch = env
    rng = np.random.default_rng(n + k)
    A = rng.integers(-8, 9, size=(128, k)).astype(np.float32)
    B = rng.integers(-8, 9, size=(n, k)).astype(np.float32)
    D = _run(sk, ctx, torch, A, B, 1)
    assert np.array_equal(D, A.astype(np.float64) @ B.T.astype(np.float64))


def test_3xtf32_accuracy(env):
    sk, ctx, torch = env
    rng = np.random.default_rng(3)
    A = rng.standard_normal((128, 64)).astype(np.float32)
    B = rng.standard_normal((64, 64)).astype(np.float32)
    want = A.astype(np.float64) @ B.T.astype(np.float64)
    D3 = _run(sk, ctx, torch, A, B, 3)
    D1 = _run(sk, ctx, torch, A, B, 1)
    scale = np.abs(A).astype(np.float64) @ np.abs(B).T.astype(np.float64)
    assert np.max(np.abs(D3 - want) / scale) < 2e-6          # 3xTF32 ~ FP32 accuracy
    assert np.max(np.abs(D1 - want) / scale) > 1e-5          # plain TF32 is visibly coarser


def _run_sliding(sk, ctx, torch, A, x, n, off):
    a = torch.from_numpy(np.ascontiguousarray(A, np.float32)).cuda()
    xv = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    d = torch.full((128, n), float("nan"), device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = sk.lib()
    rc = L.sk_selftest_tc_sliding(ctx._h, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(xv.data_ptr()),
                                  ctypes.c_void_p(d.data_ptr()), n, A.shape[1], off, st)
    assert rc == 0, L.sk_last_error()
    torch.cuda.synchronize()
    assert L.sk_get_status(ctx._h, st) == 0
    return d.cpu().numpy().astype(np.float64)


def _sliding_ref(A, x, n, off):
    K = A.shape[1]
    B = np.stack([x[8 * s + off: 8 * s + off + K] for s in range(n)]).astype(np.float64)
    return A.astype(np.float64) @ B.T


@pytest.mark.parametrize("n,k,off", [(256, 40, 0), (256, 40, 4), (16, 8, 4), (128, 64, 0), (64, 24, 4)])
def test_sliding_rows_exact_on_small_integers(env, n, k, off):
    sk, ctx, torch = env
    rng = np.random.default_rng(7 * n + k + off)
    A = rng.integers(-8, 9, size=(128, k)).astype(np.float32)
    x = rng.integers(-8, 9, size=8 * (n + k // 8 + 2)).astype(np.float32)
    D = _run_sliding(sk, ctx, torch, A, x, n, off)
    assert np.array_equal(D, _sliding_ref(A, x, n, off))


def test_sliding_rows_3xtf32_accuracy(env):
    sk, ctx, torch = env
    rng = np.random.default_rng(11)
    n, k = 256, 48
    A = rng.standard_normal((128, k)).astype(np.float32)
    x = rng.standard_normal(8 * (n + k // 8 + 2)).astype(np.float32)
    for off in (0, 4):
        D = _run_sliding(sk, ctx, torch, A, x, n, off)
        want = _sliding_ref(A, x, n, off)
        scale = _sliding_ref(np.abs(A), np.abs(x), n, off)
        assert np.max(np.abs(D - want) / scale) < 2e-6


def _run_sliding_bf16(sk, ctx, torch, A, x, n):
    a = torch.from_numpy(np.ascontiguousarray(A, np.float32)).cuda()
    xv = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    d = torch.full((128, n), float("nan"), device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = sk.lib()
    rc = L.sk_selftest_tc_sliding_bf16(ctx._h, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(xv.data_ptr()),
                                       ctypes.c_void_p(d.data_ptr()), n, A.shape[1], st)
    assert rc == 0, L.sk_last_error()
    torch.cuda.synchronize()
    assert L.sk_get_status(ctx._h, st) == 0
    return d.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n,k", [(256, 32), (16, 16), (128, 64), (64, 48)])
def test_sliding_rows_bf16_exact_on_small_integers(env, n, k):
    sk, ctx, torch = env
    rng = np.random.default_rng(9 * n + k)
    A = rng.integers(-8, 9, size=(128, k)).astype(np.float32)
    x = rng.integers(-8, 9, size=8 * (n + k // 8)).astype(np.float32)
    D = _run_sliding_bf16(sk, ctx, torch, A, x, n)
    assert np.array_equal(D, _sliding_ref(A, x, n, 0))


def test_sliding_rows_bf16x3_accuracy(env):
    # BF16x3 keeps about 16 significant bits of each operand: ~1e-5 per product, far
    # coarser than 3xTF32 (the reason it is not the accuracy-bound form)
    sk, ctx, torch = env
    rng = np.random.default_rng(12)
    n, k = 256, 48
    A = rng.standard_normal((128, k)).astype(np.float32)
    x = rng.standard_normal(8 * (n + k // 8)).astype(np.float32)
    D = _run_sliding_bf16(sk, ctx, torch, A, x, n)
    want = _sliding_ref(A, x, n, 0)
    scale = _sliding_ref(np.abs(A), np.abs(x), n, 0)
    err = np.max(np.abs(D - want) / scale)
    assert 2e-6 < err < 1e-4
