"""sph_conv (torch.autograd.Function over the C ABI): the map and table gradients of a
quadratic loss against the FP64 oracle, and a whole training step (table update,
forward, backward) captured in a CUDA graph -- possible only because no call of the
step synchronises with the host -- replayed after the table changed in place.

Operator: the real-space convolution of Sec. 2, Eq. 1 with the tabulated kernel of
Sec. 3; dL/dx = A^T dL/dy (A is symmetric: the same gather), dL/dV_n by the binned
scatter-add of the interpolation weights.  Bars: rms 1e-6 for maps, 1e-5 of the
largest table-gradient bin.
"""
import math

import numpy as np
import pytest

import oracle as O
from inputs import gaussian_beam, white_noise_maps

pytestmark = pytest.mark.gpu

NSIDE, TC, NT = 32, 0.12, 512


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1211_3556_b300 as sk
    ctx = sk.Context(0)
    V1 = O.tabulate_real_kernel(gaussian_beam(9.0 * 60.0 * TC / math.pi, 96), 24, 96, TC, NT)
    V2 = O.tabulate_real_kernel(gaussian_beam(10.0 * 60.0 * TC / math.pi, 96), 24, 96, TC, NT)
    k = sk.Kernel(sk.Geometry(ctx, NSIDE), V1, TC)
    x = white_noise_maps(NSIDE, 2, 41)
    t = white_noise_maps(NSIDE, 2, 42) * np.float32(0.1)
    yield dict(sk=sk, ctx=ctx, k=k, V1=V1, V2=V2, x=x, t=t)
    torch.cuda.synchronize()


def _oracle_grads(V, x, t):
    """y, dL/dx, dL/dV for L = sum (y - t)^2 by the oracle (FP64)."""
    y = np.stack([O.conv_window(NSIDE, V, TC, 0, x[b].astype(np.float64)) for b in range(len(x))])
    r = 2.0 * (y - t.astype(np.float64))
    gx = np.stack([O.conv_window(NSIDE, V, TC, 0, r[b]) for b in range(len(x))])
    gV = sum(O.grad_table(NSIDE, NT, TC, 0, x[b].astype(np.float64), r[b]) for b in range(len(x)))
    return y, gx, gV


def _rms(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_gradients_of_a_quadratic_loss_match_the_oracle(env):
    import torch
    sk = env["sk"]
    xt = torch.from_numpy(env["x"]).cuda().requires_grad_(True)
    tt = torch.from_numpy(env["t"]).cuda()
    table = torch.tensor(env["V2"], dtype=torch.float64, device="cuda", requires_grad=True)
    y = sk.sph_conv(xt, table, env["k"])
    loss = ((y - tt) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    env["ctx"].status()
    yo, gxo, gVo = _oracle_grads(env["V2"], env["x"], env["t"])
    assert _rms(y.detach().cpu().numpy(), yo) <= 1e-6
    assert _rms(xt.grad.cpu().numpy(), gxo) <= 1e-6
    g = table.grad.cpu().numpy()
    assert np.abs(g - gVo).max() <= 1e-5 * np.abs(gVo).max()
    # the oracle's table gradient is itself a central difference of the FP64 loss
    rng = np.random.default_rng(43)
    for n in rng.choice(NT - 1, 4, replace=False):
        h = 1e-6 * np.abs(env["V2"]).max()
        Vp, Vm = env["V2"].copy(), env["V2"].copy()
        Vp[n] += h
        Vm[n] -= h
        lp = sum(float(np.sum((O.conv_window(NSIDE, Vp, TC, 0, env["x"][b].astype(np.float64)) - env["t"][b]) ** 2))
                 for b in range(2))
        lm = sum(float(np.sum((O.conv_window(NSIDE, Vm, TC, 0, env["x"][b].astype(np.float64)) - env["t"][b]) ** 2))
                 for b in range(2))
        assert abs((lp - lm) / (2 * h) - g[n]) <= 1e-5 * np.abs(gVo).max()


def test_training_step_captures_in_a_cuda_graph(env):
    import torch
    sk = env["sk"]
    k = env["k"]
    xs = torch.from_numpy(env["x"]).cuda().requires_grad_(True)
    ts = torch.from_numpy(env["t"]).cuda()
    table = torch.tensor(env["V1"], dtype=torch.float64, device="cuda", requires_grad=True)

    def step():
        y = sk.sph_conv(xs, table, k)
        ((y - ts) ** 2).sum().backward()
        return y

    # warm-up on a side stream (workspaces, the update flag and autograd state exist afterwards)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(2):
            xs.grad = None
            table.grad = None
            step()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    xs.grad = None
    table.grad = None
    with torch.cuda.graph(graph):
        y_static = step()
    for V in (env["V2"], env["V1"]):
        with torch.no_grad():
            table.copy_(torch.from_numpy(V))         # in place: the graph reads the new values
            xs.grad.zero_()
            table.grad.zero_()
        graph.replay()
        torch.cuda.synchronize()
        env["ctx"].status()
        yo, gxo, gVo = _oracle_grads(V, env["x"], env["t"])
        assert _rms(y_static.detach().cpu().numpy(), yo) <= 1e-6
        assert _rms(xs.grad.cpu().numpy(), gxo) <= 1e-6
        assert np.abs(table.grad.cpu().numpy() - gVo).max() <= 1e-5 * np.abs(gVo).max()
