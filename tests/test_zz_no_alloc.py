"""The allocation-free table gradient, called through the C ABI.

sk_grad_table_noalloc serves callers that cannot let the library allocate
device memory (their memory belongs to their own allocator or budget, or a
cudaMalloc would stall a latency-critical loop): it keeps its FP64
accumulator in a fixed array inside the library instead of the context
workspace.  Two calls in a row must each match sk_grad_table, so the second
call must not see what the first left in the shared array.  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-5          # the table-gradient tolerance of the parity tests (relative to the largest bin)


def test_noalloc_grad_matches_workspace_grad_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1211_3556_b300 as sk
    import oracle as O
    from inputs import gaussian_beam, white_noise_maps

    L = sk.lib()
    ctx = sk.Context(0)
    nside, tc, nt = 32, 0.12, 512
    V = O.tabulate_real_kernel(gaussian_beam(10.0 * 60.0 * tc / 3.0, 96), 24, 96, tc, nt)
    g = sk.Geometry(ctx, nside)
    k = sk.Kernel(g, V, tc)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = []
    for seed in (1, 2):
        x = torch.from_numpy(white_noise_maps(nside, 3, 10 + seed)).cuda()
        gy = torch.from_numpy(white_noise_maps(nside, 3, 20 + seed)).cuda()
        ref = torch.empty(nt, dtype=torch.float32, device="cuda")
        got = torch.full((nt,), float("nan"), dtype=torch.float32, device="cuda")
        stride = x.stride(0)
        rc = L.sk_grad_table(ctx._h, k._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(gy.data_ptr()),
                             3, stride, ctypes.c_void_p(ref.data_ptr()), stream)
        assert rc == 0, L.sk_last_error()
        rc = L.sk_grad_table_noalloc(ctx._h, k._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(gy.data_ptr()),
                                     3, stride, ctypes.c_void_p(got.data_ptr()), stream)
        assert rc == 0, L.sk_last_error()
        torch.cuda.synchronize()
        assert L.sk_get_status(ctx._h, stream) == 0
        r = ref.cpu().numpy().astype(np.float64)
        o = got.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(o))
        assert np.abs(o - r).max() <= TOL * np.abs(r).max()
        outs.append(o)
    assert not np.allclose(outs[0], outs[1])        # the two calls saw different inputs
