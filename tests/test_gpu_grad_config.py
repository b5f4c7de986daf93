"""Gradients at the differentiation workload's full size, through the C ABI.

Workload: 16 FP32 white-noise maps at Nside 1024 (12.6 M pixels each), Gaussian
beam FWHM 10' split at l_cut 512 (l_max 2048), theta_cut 30', 4096 uniform
nodes; loss L = sum_{b,o} (y_bo - t_bo)^2 with y = A x and the target t = A' x of
the kernel perturbed to FWHM 10.5', computed by the FP64 oracle and stored as
FP32 (the convolution is Sec. 2, Eq. 1 with the tabulated kernel of Sec. 3).

* The table gradient against the oracle's, element by element over all 4096
  nodes, for dL/dy non-zero on 2000 random outputs per map (the oracle visits
  only those outputs, so the check costs seconds at this size).
* FP64 central differences through the oracle (entries drawn with seed 402,
  uniform without replacement):
  - 64 map entries on the full loss: x_bi changes only the outputs within
    theta_cut of pixel i, so L(x + h e_bi) - L(x - h e_bi) is the difference of
    the loss restricted to those outputs, which the oracle recomputes;
  - 64 table nodes on the loss restricted to the 2000 sampled outputs per map
    (the full loss would take the oracle about 5e10 pair evaluations per loss
    value); the GPU gradient is then the table gradient of that loss.
  h = 1e-6 relative to the perturbed quantity's scale (unit-variance maps:
  h = 1e-6; the table: h = 1e-6 max|V|).  The loss is quadratic, so central
  differences equal the gradient up to FP64 rounding, which this h keeps
  below 1e-9 of the gradients.  The differences of squares are summed as
  (L+ - L-) = sum (y+ - y-)(y+ + y- - 2t), the same value without cancelling
  two large sums.
Bar: max |g_gpu - g_ref| <= 1e-5 max |g_ref| over the checked entries.
"""
import math

import numpy as np
import pytest

import oracle as O
from inputs import WORKLOADS, gaussian_beam, sample_indices, white_noise_maps

pytestmark = pytest.mark.gpu

GRAD_BOUND = 1e-5
N_SAMPLED = 2000
FD_SEED = 402
FD_COUNT = 64
TARGET_FWHM = 10.5


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1211_3556_b300 as sk
    ctx = sk.Context(0)
    grp = WORKLOADS["n1024x16_grad"].groups[0]
    ks = grp.kernel
    nside, B = grp.nside, grp.batch
    V = O.tabulate_real_kernel(ks.beam(), ks.lcut, ks.lmax, ks.theta_cut, ks.n_nodes, ks.layout)
    Vt = O.tabulate_real_kernel(gaussian_beam(TARGET_FWHM, ks.lmax), ks.lcut, ks.lmax, ks.theta_cut,
                                ks.n_nodes, ks.layout)
    k = sk.Kernel(sk.Geometry(ctx, nside), V, ks.theta_cut, ks.layout)
    x = white_noise_maps(nside, B, grp.seed)
    xt = torch.from_numpy(x).cuda()
    y = sk.convolve(k, xt)
    torch.cuda.synchronize()
    ctx.status()
    d = dict(sk=sk, ctx=ctx, ks=ks, nside=nside, B=B, V=V, Vt=Vt, k=k, x=x, xt=xt, y=y,
             npix=x.shape[1])
    yield d
    torch.cuda.synchronize()


def test_table_gradient_full_size_elementwise(setup):
    import torch
    s = setup
    sk, ks, nside, B, npix = s["sk"], s["ks"], s["nside"], s["B"], s["npix"]
    rng = np.random.default_rng(4001)
    gy = np.zeros_like(s["x"])
    for b in range(B):
        outs = sample_indices(npix, N_SAMPLED, 4100 + b)
        gy[b, outs] = rng.standard_normal(len(outs)).astype(np.float32)
    gt = sk.grad_table(s["k"], s["xt"], torch.from_numpy(gy).cuda())
    torch.cuda.synchronize()
    s["ctx"].status()
    go = np.zeros(ks.n_nodes)
    for b in range(B):
        go += O.grad_table(nside, ks.n_nodes, ks.theta_cut, ks.layout, s["x"][b].astype(np.float64),
                           gy[b].astype(np.float64))
    got = gt.cpu().numpy().astype(np.float64)
    assert np.count_nonzero(go) > 0.9 * ks.n_nodes       # the sampled outputs reach most nodes
    assert np.abs(got - go).max() <= GRAD_BOUND * np.abs(go).max()


def _entries():
    rng = np.random.default_rng(FD_SEED)
    grp = WORKLOADS["n1024x16_grad"].groups[0]
    npix = 12 * grp.nside * grp.nside
    flat = rng.choice(grp.batch * npix, FD_COUNT, replace=False)
    nodes = rng.choice(grp.kernel.n_nodes, FD_COUNT, replace=False)
    return flat // npix, flat % npix, np.sort(nodes)


def test_map_gradient_central_differences(setup):
    import torch
    s = setup
    sk, ks, nside, B, npix = s["sk"], s["ks"], s["nside"], s["B"], s["npix"]
    maps, pix, _ = _entries()
    # outputs whose loss terms x_bi reaches: within theta_cut of pixel i (a superset
    # by 1e-9 rad; outputs beyond the cut keep their value and cancel exactly)
    vec = O.all_vecs(nside)
    cosc = math.cos(ks.theta_cut + 1e-9)
    near = [np.nonzero(vec @ vec[i] >= cosc)[0] for i in pix]
    del vec
    # target on those outputs (FP64 oracle, stored FP32)
    t = [O.conv_window(nside, s["Vt"], ks.theta_cut, ks.layout, s["x"][b].astype(np.float64), nb)
         .astype(np.float32) for b, nb in zip(maps, near)]
    # GPU: dL/dx = A^T 2 (y - t); only the outputs near the checked entries matter for them
    y = s["y"].cpu().numpy()
    gy = np.zeros_like(s["x"])
    for b, nb, tb in zip(maps, near, t):
        gy[b, nb] = 2.0 * (y[b, nb].astype(np.float64) - tb)
    gx = sk.convolve_adjoint(s["k"], torch.from_numpy(gy).cuda())
    torch.cuda.synchronize()
    s["ctx"].status()
    g_gpu = gx.cpu().numpy()[maps, pix].astype(np.float64)
    # oracle central differences of the full loss (only the outputs near i change)
    h = 1e-6
    g_fd = np.empty(FD_COUNT)
    for e, (b, i, nb) in enumerate(zip(maps, pix, near)):
        tb = t[e].astype(np.float64)
        xp = s["x"][b].astype(np.float64)
        xm = xp.copy()
        xp[i] += h
        xm[i] -= h
        yp = O.conv_window(nside, s["V"], ks.theta_cut, ks.layout, xp, nb)
        ym = O.conv_window(nside, s["V"], ks.theta_cut, ks.layout, xm, nb)
        g_fd[e] = float(np.sum((yp - ym) * (yp + ym - 2.0 * tb))) / (2.0 * h)
    assert np.abs(g_fd).max() > 0
    assert np.abs(g_gpu - g_fd).max() <= GRAD_BOUND * np.abs(g_fd).max()


def test_table_gradient_central_differences(setup):
    import torch
    s = setup
    sk, ks, nside, B, npix = s["sk"], s["ks"], s["nside"], s["B"], s["npix"]
    _, _, nodes = _entries()
    outs = [sample_indices(npix, N_SAMPLED, 4200 + b) for b in range(B)]
    xs = [s["x"][b].astype(np.float64) for b in range(B)]
    t = [O.conv_window(nside, s["Vt"], ks.theta_cut, ks.layout, xs[b], outs[b]).astype(np.float32)
         .astype(np.float64) for b in range(B)]
    # GPU: the table gradient of the loss on the sampled outputs
    y = s["y"].cpu().numpy()
    gy = np.zeros_like(s["x"])
    for b in range(B):
        gy[b, outs[b]] = 2.0 * (y[b, outs[b]].astype(np.float64) - t[b])
    gt = sk.grad_table(s["k"], s["xt"], torch.from_numpy(gy).cuda())
    torch.cuda.synchronize()
    s["ctx"].status()
    g_gpu = gt.cpu().numpy()[nodes].astype(np.float64)
    # oracle central differences in the node values
    h = 1e-6 * np.abs(s["V"]).max()
    g_fd = np.zeros(FD_COUNT)
    for e, n in enumerate(nodes):
        Vp = s["V"].copy()
        Vm = s["V"].copy()
        Vp[n] += h
        Vm[n] -= h
        acc = 0.0
        for b in range(B):
            yp = O.conv_window(nside, Vp, ks.theta_cut, ks.layout, xs[b], outs[b])
            ym = O.conv_window(nside, Vm, ks.theta_cut, ks.layout, xs[b], outs[b])
            acc += float(np.sum((yp - ym) * (yp + ym - 2.0 * t[b])))
        g_fd[e] = acc / (2.0 * h)
    assert np.abs(g_fd).max() > 0
    assert np.abs(g_gpu - g_fd).max() <= GRAD_BOUND * np.abs(g_fd).max()
