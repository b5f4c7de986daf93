"""CUDA path against the FP64 oracle, through the C ABI (via the thin binding).

Bar: rms relative error <= 1e-6 against the oracle on the same FP32 input
promoted to FP64 and the same FP64 table (error budget: FP32 chord, asin
series and table coordinate, each ~1e-7 relative; FP32 accumulation over a few
hundred terms).  Integer results (ring tables, pair counts) are bit-exact.
Inputs are seeded and synthetic (white-noise maps, Gaussian-beam kernels split
at l_cut, point sources).
"""
import math

import numpy as np
import pytest

import oracle as O
from inputs import (ARCMIN, WORKLOADS, add_point_sources, gaussian_beam, sample_indices,
                    white_noise_maps)

pytestmark = pytest.mark.gpu

RMS_BOUND = 1e-6


@pytest.fixture(scope="module")
def sk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1211_3556_b300 as sk
    sk._ctx = sk.Context(0)
    yield sk
    torch.cuda.synchronize()


def rms_rel(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_conv(sk, kern, x, path=0):
    import torch
    xt = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    y = sk.convolve(kern, xt, path=path)
    torch.cuda.synchronize()
    sk._ctx.status()
    return y.cpu().numpy().astype(np.float64)


def oracle_table(nside, fwhm, lmax, lcut, tc, nt, layout=0):
    return O.tabulate_real_kernel(gaussian_beam(fwhm, lmax), lcut, lmax, tc, nt, layout)


# ------------------------------------------------------------------ geometry

@pytest.mark.parametrize("nside", [1, 2, 16, 64, 2048])
def test_ring_tables_match_oracle(sk, nside):
    g = sk.Geometry(sk._ctx, nside)
    n, st, s, z, sn = g.rings()
    for r in range(1, 4 * nside, max(1, (4 * nside) // 97)):
        on, ost, os_, oz, osn = O.ring_info(nside, r)
        assert (n[r - 1], st[r - 1], s[r - 1]) == (on, ost, os_)
        assert z[r - 1] == pytest.approx(oz, abs=2e-16)
        assert sn[r - 1] == pytest.approx(osn, abs=2e-16)


# ------------------------------------------------------------------ tabulation

@pytest.mark.parametrize("layout", [0, 1])
def test_legendre_tabulation_matches_oracle(sk, layout):
    g = sk.Geometry(sk._ctx, 64)
    b = gaussian_beam(60.0, 192)
    tc = 180 * ARCMIN
    v_gpu = sk.Kernel.tabulate(g, b, 97, 192, 4096, tc, layout)
    v_or = O.tabulate_real_kernel(b, 96, 192, tc, 4096, layout)
    assert np.abs(v_gpu - v_or).max() <= 1e-11 * np.abs(v_or).max()


def test_legendre_tabulation_high_l(sk):
    g = sk.Geometry(sk._ctx, 64)
    b = gaussian_beam(7.1, 4096)
    tc = 20 * ARCMIN
    v_gpu = sk.Kernel.tabulate(g, b, 1025, 4096, 512, tc, 0)
    v_or = O.tabulate_real_kernel(b, 1024, 4096, tc, 512, 0)
    assert np.abs(v_gpu - v_or).max() <= 1e-9 * np.abs(v_or).max()


# ------------------------------------------------------------------ pair counts

@pytest.mark.parametrize("nside,tc", [(4, 0.9), (8, 0.3), (16, 0.15), (64, 180 * ARCMIN), (32, 2.5)])
def test_pair_count_exact(sk, nside, tc):
    g = sk.Geometry(sk._ctx, nside)
    k = sk.Kernel(g, np.ones(16), tc)
    assert k.count_pairs() == O.count_pairs(nside, tc)


# ------------------------------------------------------------------ forward parity

CASES = [
    # nside, theta_cut, n_nodes, layout, path
    (8, 0.35, 256, 0, 0), (8, 0.35, 256, 0, 1),
    (16, 0.2, 512, 1, 0), (16, 1.2, 512, 0, 0),      # wide cut: whole-ring windows, no belt
    (32, 0.08, 1024, 0, 0), (32, 0.08, 1024, 1, 1),
    (64, 180 * ARCMIN, 4096, 0, 0), (64, 180 * ARCMIN, 4096, 0, 1),
    (128, 0.03, 2048, 0, 0), (128, 0.03, 2048, 1, 0),
    (256, 0.02, 4096, 0, 0),
]


@pytest.mark.parametrize("nside,tc,nt,layout,path", CASES)
def test_forward_matches_oracle(sk, nside, tc, nt, layout, path):
    lmax = 3 * nside
    V = oracle_table(nside, 2.5 * tc / 3 / ARCMIN, lmax, lmax // 4, tc, nt, layout)
    g = sk.Geometry(sk._ctx, nside)
    k = sk.Kernel(g, V, tc, layout)
    x = white_noise_maps(nside, 1, 1000 + nside)
    y = gpu_conv(sk, k, x, path)[0]
    yo = O.conv_window(nside, V, tc, layout, x[0].astype(np.float64))
    assert rms_rel(y, yo) <= RMS_BOUND
    assert np.abs(y - yo).max() <= 1e-5 * np.abs(yo).max()


# The smallest pixelisations and the widest cut the ABI accepts (theta_cut = pi: every
# window is a whole ring and every pixel reaches the whole map, its antipode included).
# The table is any smooth function, tapered to 0 at theta_cut (reading: the cut is
# closed and the table vanishes there, so FP32/FP64 inclusion at the edge agrees).
TINY_CASES = [
    # nside, theta_cut, path
    (1, math.pi, 0), (1, math.pi, 1), (1, 1.3, 0),
    (2, math.pi, 0), (2, math.pi, 1), (2, 0.8, 0),
    (4, math.pi, 0), (4, math.pi, 1), (4, 0.45, 0),
    (8, math.pi, 0), (8, math.pi, 1),
    # every output sums all 3072 / 12288 pixels: the blocked summation of wide windows
    (16, math.pi, 0), (32, math.pi, 0),
]


@pytest.mark.parametrize("nside,tc,path", TINY_CASES)
def test_forward_tiny_and_whole_sphere(sk, nside, tc, path):
    nt = 512
    th = O.node_thetas(nt, tc, 0)
    V = (1.0 + 0.5 * np.cos(3.0 * th) - 0.2 * th) * O.taper(th, tc)
    g = sk.Geometry(sk._ctx, nside)
    k = sk.Kernel(g, V, tc)
    x = white_noise_maps(nside, 2, 1100 + nside)
    y = gpu_conv(sk, k, x, path)
    for b in range(2):
        yo = O.conv_brute(nside, V, tc, 0, x[b].astype(np.float64))
        assert rms_rel(y[b], yo) <= RMS_BOUND, (b, rms_rel(y[b], yo))
        assert np.abs(y[b] - yo).max() <= 1e-5 * np.abs(yo).max()


def test_config_n64_full_map(sk):
    wl = WORKLOADS["n64_plain"].groups[0]
    ks = wl.kernel
    V = O.tabulate_real_kernel(ks.beam(), ks.lcut, ks.lmax, ks.theta_cut, ks.n_nodes, ks.layout)
    g = sk.Geometry(sk._ctx, wl.nside)
    k = sk.Kernel(g, V, ks.theta_cut, ks.layout)
    x = white_noise_maps(wl.nside, 1, wl.seed)
    y = gpu_conv(sk, k, x)[0]
    yo = O.conv_window(wl.nside, V, ks.theta_cut, ks.layout, x[0].astype(np.float64))
    assert rms_rel(y, yo) <= RMS_BOUND


def _special_pixels(nside):
    """Pole rings, the first pixel of rings (phi = 0 wrap), the z = +-2/3 rings, the equator."""
    N = nside
    rings = [1, 2, N - 1, N, N + 1, 2 * N - 1, 2 * N, 3 * N, 3 * N + 1, 4 * N - 2, 4 * N - 1]
    pix = []
    for r in rings:
        n, st, *_ = O.ring_info(N, r)
        pix += [st, st + n - 1, st + n // 4, st + n // 2 - 1]
    return np.unique(np.array(pix, dtype=np.int64))


@pytest.mark.parametrize("nside,tc", [(32, 0.12), (128, 0.04)])
def test_delta_maps_at_special_pixels(sk, nside, tc):
    V = oracle_table(nside, 2.5 * tc / 3 / ARCMIN, 3 * nside, nside, tc, 1024)
    g = sk.Geometry(sk._ctx, nside)
    k = sk.Kernel(g, V, tc)
    pix = _special_pixels(nside)
    x = np.zeros((len(pix), 12 * nside * nside), np.float32)
    x[np.arange(len(pix)), pix] = 1.0
    y = gpu_conv(sk, k, x)
    for b, p in enumerate(pix):
        yo = O.conv_window(nside, V, tc, 0, x[b].astype(np.float64))
        assert rms_rel(y[b], yo) <= RMS_BOUND, (p, rms_rel(y[b], yo))


def test_config_n2048_sampled_outputs(sk):
    wl = WORKLOADS["n2048_plain"]
    grp = wl.groups[0]
    ks = grp.kernel
    V = O.tabulate_real_kernel(ks.beam(), ks.lcut, ks.lmax, ks.theta_cut, ks.n_nodes, ks.layout)
    g = sk.Geometry(sk._ctx, grp.nside)
    k = sk.Kernel(g, V, ks.theta_cut, ks.layout)
    x = white_noise_maps(grp.nside, 1, grp.seed)
    add_point_sources(x, *wl.sources[0])
    y = gpu_conv(sk, k, x)[0]
    outs = np.concatenate([sample_indices(x.shape[1], 20000, 203), _special_pixels(grp.nside)])
    yo = O.conv_window(grp.nside, V, ks.theta_cut, ks.layout, x[0].astype(np.float64), outs)
    assert rms_rel(y[outs], yo) <= RMS_BOUND


@pytest.mark.parametrize("form", ["fp32", "tensor"])
def test_config_n8192_sampled_outputs(sk, form):
    # the largest workload (Nside 8192, 16384 nodes, 3.2 GB per map) in bench.py's
    # launch configuration, on sampled outputs, with each belt form
    grp = WORKLOADS["n8192_plain"].groups[0]
    ks = grp.kernel
    V = O.tabulate_real_kernel(ks.beam(), ks.lcut, ks.lmax, ks.theta_cut, ks.n_nodes, ks.layout)
    g = sk.Geometry(sk._ctx, grp.nside)
    k = sk.Kernel(g, V, ks.theta_cut, ks.layout)
    if form == "tensor":
        assert k.config()["tensor_form_available"]
        k.set_belt_form(sk.BELT_TENSOR)
    x = white_noise_maps(grp.nside, 1, grp.seed)
    y = gpu_conv(sk, k, x)[0]
    outs = np.concatenate([sample_indices(x.shape[1], 5000, 503), _special_pixels(grp.nside)])
    yo = O.conv_window(grp.nside, V, ks.theta_cut, ks.layout, x[0].astype(np.float64), outs)
    assert rms_rel(y[outs], yo) <= RMS_BOUND


@pytest.mark.parametrize("form", ["fp32", "tensor"])
def test_config_mixed_batch_sampled_outputs(sk, form):
    # the uneven batch (8 x Nside 256, 8 x 512, 4 x 1024, 2 x 2048, four kernels) in one
    # convolve_jobs call, every map checked on sampled outputs, with each belt form
    import torch
    wl = WORKLOADS["mixed_batch"]
    jobs, keep = [], []
    for grp in wl.groups:
        ks = grp.kernel
        V = O.tabulate_real_kernel(ks.beam(), ks.lcut, ks.lmax, ks.theta_cut, ks.n_nodes, ks.layout)
        g = sk.Geometry(sk._ctx, grp.nside)
        k = sk.Kernel(g, V, ks.theta_cut, ks.layout)
        if form == "tensor":
            assert k.config()["tensor_form_available"]
            k.set_belt_form(sk.BELT_TENSOR)
        x = white_noise_maps(grp.nside, grp.batch, grp.seed)
        xt = torch.from_numpy(x).cuda()
        yt = torch.empty_like(xt)
        jobs.append((k, xt, yt))
        keep.append((grp, V, x, g))
    sk.convolve_jobs(sk._ctx, jobs)
    torch.cuda.synchronize()
    sk._ctx.status()
    for (grp, V, x, g), (k, xt, yt) in zip(keep, jobs):
        ks = grp.kernel
        y = yt.cpu().numpy()
        for b in range(grp.batch):
            outs = sample_indices(x.shape[1], 1500, 610 + b)
            yo = O.conv_window(grp.nside, V, ks.theta_cut, ks.layout, x[b].astype(np.float64), outs)
            assert rms_rel(y[b, outs], yo) <= RMS_BOUND


def test_config_grad_full_size_euler_identity(sk):
    # y is linear in the node values, so for L = <gy, y> with gy held fixed,
    # sum_n V_n dL/dV_n = <gy, y>; with gy = y the right side is |y|^2 (no
    # cancellation), and a node shift or a lost term moves the left side by ~1e-3
    import torch
    grp = WORKLOADS["n1024x16_grad"].groups[0]
    ks = grp.kernel
    V = O.tabulate_real_kernel(ks.beam(), ks.lcut, ks.lmax, ks.theta_cut, ks.n_nodes, ks.layout)
    g = sk.Geometry(sk._ctx, grp.nside)
    k = sk.Kernel(g, V, ks.theta_cut, ks.layout)
    x = torch.from_numpy(white_noise_maps(grp.nside, grp.batch, grp.seed)).cuda()
    y = sk.convolve(k, x)
    gt = sk.grad_table(k, x, y)
    torch.cuda.synchronize()
    lhs = float(np.dot(V, gt.cpu().numpy().astype(np.float64)))
    rhs = float((y.double() * y.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * rhs


# ------------------------------------------------------------------ batch, adjoint

def test_batch_equals_single_maps(sk):
    nside, tc = 128, 0.03
    V = oracle_table(nside, 2.5 * tc / 3 / ARCMIN, 384, 96, tc, 2048)
    g = sk.Geometry(sk._ctx, nside)
    k = sk.Kernel(g, V, tc)
    x = white_noise_maps(nside, 5, 77)
    yb = gpu_conv(sk, k, x)
    for b in range(5):
        assert np.array_equal(yb[b], gpu_conv(sk, k, x[b:b + 1])[0])


@pytest.mark.parametrize("nside,tc,batch", [(8, 0.6, 1), (64, 180 * ARCMIN, 1), (128, 0.05, 3), (512, 0.012, 2)])
def test_host_buffer_path_equals_device_path(sk, nside, tc, batch):
    # sk_convolve_host moves the maps in ring bands and sums each band once its
    # inputs are there: same kernels, same per-output order, so bit-identical results
    import torch
    V = oracle_table(nside, tc / ARCMIN / 3.0, 2 * nside, nside // 2, tc, 1024)
    g = sk.Geometry(sk._ctx, nside)
    k = sk.Kernel(g, V, tc)
    npix = 12 * nside * nside
    x = white_noise_maps(nside, batch, 900 + nside)
    y_dev = gpu_conv(sk, k, x)
    y_host = sk.convolve_host(k, x)
    assert np.array_equal(y_host.reshape(batch, npix), y_dev.reshape(batch, npix).astype(np.float32))
    xp = torch.from_numpy(x).pin_memory()
    yp = torch.empty_like(xp).pin_memory()
    sk.convolve_host(k, xp.numpy(), yp.numpy())
    assert np.array_equal(yp.numpy(), y_host.reshape(batch, npix))


def test_adjoint_dot_product(sk):
    import torch
    nside, tc = 64, 0.06
    V = oracle_table(nside, 2.5 * tc / 3 / ARCMIN, 192, 48, tc, 1024)
    g = sk.Geometry(sk._ctx, nside)
    k = sk.Kernel(g, V, tc)
    x = torch.from_numpy(white_noise_maps(nside, 1, 5)).cuda()
    yb = torch.from_numpy(white_noise_maps(nside, 1, 6)).cuda()
    Ax = sk.convolve(k, x)
    ATy = sk.convolve_adjoint(k, yb)
    lhs = float((Ax.double() * yb.double()).sum())
    rhs = float((x.double() * ATy.double()).sum())
    assert abs(lhs - rhs) <= 1e-6 * float((Ax.double().abs() * yb.double().abs()).sum())


# ------------------------------------------------------------------ table gradient

@pytest.mark.parametrize("nside,tc,layout,nt", [(16, 0.25, 0, 64), (32, 0.1, 1, 64), (32, 0.12, 0, 512),
                                                 (64, 0.05, 0, 4096), (256, 0.02, 0, 4096)])
def test_grad_table_matches_oracle(sk, nside, tc, layout, nt):
    import torch
    V = oracle_table(nside, 2.5 * tc / 3 / ARCMIN, 3 * nside, nside, tc, nt, layout)
    g = sk.Geometry(sk._ctx, nside)
    k = sk.Kernel(g, V, tc, layout)
    x = white_noise_maps(nside, 2, 21)
    gy = white_noise_maps(nside, 2, 22)
    gt = sk.grad_table(k, torch.from_numpy(x).cuda(), torch.from_numpy(gy).cuda())
    torch.cuda.synchronize()
    go = sum(O.grad_table(nside, nt, tc, layout, x[b].astype(np.float64), gy[b].astype(np.float64))
             for b in range(2))
    got = gt.cpu().numpy().astype(np.float64)
    assert np.abs(got - go).max() <= 1e-5 * np.abs(go).max()


@pytest.mark.parametrize("nside,tc,layout,nt", [(32, 0.1, 1, 64), (32, 0.12, 0, 512), (64, 0.05, 0, 4096)])
def test_grad_table_many_maps_matches_oracle(sk, nside, tc, layout, nt):
    """Nine maps: the cap gradient's later passes over the maps (four per pass, the last one
    partial) take the node interval and fraction of each pair from the first pass's cache."""
    import torch
    V = oracle_table(nside, 2.5 * tc / 3 / ARCMIN, 3 * nside, nside, tc, nt, layout)
    g = sk.Geometry(sk._ctx, nside)
    k = sk.Kernel(g, V, tc, layout)
    x = white_noise_maps(nside, 9, 23)
    gy = white_noise_maps(nside, 9, 24)
    gt = sk.grad_table(k, torch.from_numpy(x).cuda(), torch.from_numpy(gy).cuda())
    torch.cuda.synchronize()
    go = sum(O.grad_table(nside, nt, tc, layout, x[b].astype(np.float64), gy[b].astype(np.float64))
             for b in range(9))
    got = gt.cpu().numpy().astype(np.float64)
    assert np.abs(got - go).max() <= 1e-5 * np.abs(go).max()
    # the same bins from one map at a time (no cache: one pass each)
    one = sum(sk.grad_table(k, torch.from_numpy(x[b:b + 1]).cuda(), torch.from_numpy(gy[b:b + 1]).cuda())
              .cpu().numpy().astype(np.float64) for b in range(9))
    assert np.abs(got - one).max() <= 1e-6 * np.abs(go).max()


# ------------------------------------------------------------------ jobs and graphs

def _mixed_jobs(sk):
    import torch
    jobs, refs = [], []
    for nside, tc, batch, seed in [(32, 0.1, 3, 31), (64, 0.05, 2, 32), (128, 0.03, 1, 33)]:
        V = oracle_table(nside, 2.5 * tc / 3 / ARCMIN, 3 * nside, nside, tc, 1024)
        g = sk.Geometry(sk._ctx, nside)
        k = sk.Kernel(g, V, tc)
        x = torch.from_numpy(white_noise_maps(nside, batch, seed)).cuda()
        y = torch.zeros_like(x)
        jobs.append((k, x, y))
        refs.append(sk.convolve(k, x))
    return jobs, refs


def test_jobs_equal_single_calls(sk):
    import torch
    jobs, refs = _mixed_jobs(sk)
    sk.convolve_jobs(sk._ctx, jobs)
    torch.cuda.synchronize()
    for (k, x, y), r in zip(jobs, refs):
        assert torch.equal(y, r)


def test_graph_replay_equals_eager(sk):
    import torch
    jobs, refs = _mixed_jobs(sk)
    gr = sk.Graph(sk._ctx, jobs)
    for _ in range(2):
        for (_, _, y) in jobs:
            y.zero_()
        gr.launch()
        torch.cuda.synchronize()
        for (k, x, y), r in zip(jobs, refs):
            assert torch.equal(y, r)
    gr.close()


def test_graph_with_side_stream_cap_launches_equals_eager(sk):
    # an operator whose cap rings fall into several strip classes (wide windows, blocked
    # summation): its stored-weight cap launches run side by side, the smaller ones forked
    # onto the context's side stream and joined back -- inside a captured graph too
    import torch
    nside, tc, nt = 64, 0.6, 1024
    th = O.node_thetas(nt, tc, 0)
    V = (1.0 + 0.5 * np.cos(3.0 * th) - 0.2 * th) * O.taper(th, tc)
    k = sk.Kernel(sk.Geometry(sk._ctx, nside), V, tc)
    assert k.config()["cap_weights"] == "stored"
    x = torch.from_numpy(white_noise_maps(nside, 2, 1201)).cuda()
    sk._ctx.profile(True)
    sk._ctx.profile_read()
    ref = sk.convolve(k, x)
    torch.cuda.synchronize()
    prof = sk._ctx.profile_read()
    sk._ctx.profile(False)
    assert prof["conv_capw"][1] >= 2
    y = torch.zeros_like(x)
    gr = sk.Graph(sk._ctx, [(k, x, y)])
    for _ in range(2):
        y.zero_()
        gr.launch()
        torch.cuda.synchronize()
        assert torch.equal(y, ref)
    gr.close()
    sk._ctx.status()
    for b in range(2):
        outs = sample_indices(x.shape[1], 400, 1210 + b)
        yo = O.conv_window(nside, V, tc, 0, x[b].cpu().numpy().astype(np.float64), outs)
        assert rms_rel(ref[b].cpu().numpy()[outs], yo) <= RMS_BOUND


# ------------------------------------------------------------------ errors

def test_handles_released_after_their_context(sk):
    # a context released before the handles made with it, as a garbage collector may order
    # it: their release uses only their own device, not the freed context
    import torch
    nside, tc = 32, 0.1
    V = oracle_table(nside, 2.5 * tc / 3 / ARCMIN, 3 * nside, nside, tc, 512)
    ctx = sk.Context(0)
    g = sk.Geometry(ctx, nside)
    k = sk.Kernel(g, V, tc)
    ctx.close()
    k.close()
    g.close()
    torch.cuda.synchronize()
    x = torch.from_numpy(white_noise_maps(nside, 1, 5)).cuda()
    y = sk.convolve(sk.Kernel(sk.Geometry(sk._ctx, nside), V, tc), x)
    torch.cuda.synchronize()
    sk._ctx.status()
    yo = O.conv_window(nside, V, tc, 0, x[0].cpu().numpy().astype(np.float64))
    assert rms_rel(y[0].cpu().numpy(), yo) <= RMS_BOUND


def test_workspace_limit_fails_cleanly_and_the_context_survives(sk):
    # out-of-memory emulated by a capped workspace: the call fails with SK_ENOMEM before
    # launching anything, nothing is written, and the same context then runs the call
    import torch
    nside, tc = 256, 0.02
    V = oracle_table(nside, 2.5 * tc / 3 / ARCMIN, 3 * nside, nside, tc, 1024)
    ctx = sk.Context(0)
    k = sk.Kernel(sk.Geometry(ctx, nside), V, tc)
    x = torch.from_numpy(white_noise_maps(nside, 2, 1301)).cuda()
    y = torch.full_like(x, 7.0)
    ctx.set_workspace_limit(64 << 10)
    with pytest.raises(sk.SkError) as ei:
        sk.convolve(k, x, out=y)
    assert ei.value.code == sk.SK_ENOMEM
    torch.cuda.synchronize()
    assert bool((y == 7.0).all())
    ctx.status()
    ctx.set_workspace_limit(0)
    sk.convolve(k, x, out=y)
    torch.cuda.synchronize()
    ctx.status()
    assert torch.equal(y, sk.convolve(sk.Kernel(sk.Geometry(sk._ctx, nside), V, tc), x))


def test_argument_errors(sk):
    import torch
    g = sk.Geometry(sk._ctx, 16)
    with pytest.raises(sk.SkError):
        sk.Geometry(sk._ctx, 24)
    with pytest.raises(sk.SkError):
        sk.Kernel(g, np.ones(1), 0.1)
    with pytest.raises(sk.SkError):
        sk.Kernel(g, np.ones(8), -0.1)
    k = sk.Kernel(g, np.ones(8), 0.1)
    x = torch.zeros(1, 12 * 16 * 16, device="cuda")
    with pytest.raises(sk.SkError):
        sk.convolve(k, x, out=x)                          # aliasing
    big = torch.zeros(1, 12 * 16 * 16 + 4, device="cuda")
    with pytest.raises(sk.SkError):
        sk.convolve(k, big[:, 1:1 + 12 * 16 * 16])        # misaligned map pointer
    sk._ctx.status()


# ------------------------------------------------------------------ failure reporting, tuning

def test_bounded_wait_reports_timeout_and_context_survives(sk):
    import torch
    sk._ctx.status()
    sk._ctx.selftest_wait_timeout(0.05)
    with pytest.raises(sk.SkError) as ei:
        sk._ctx.status()
    assert ei.value.code == sk.SK_ETIMEOUT
    sk._ctx.status()                                   # the word was cleared
    nside, tc = 32, 0.1
    V = oracle_table(nside, 2.5 * tc / 3 / ARCMIN, 96, 24, tc, 256)
    k = sk.Kernel(sk.Geometry(sk._ctx, nside), V, tc)
    x = white_noise_maps(nside, 1, 3)
    y = gpu_conv(sk, k, x)[0]                          # the context is still usable
    assert rms_rel(y, O.conv_window(nside, V, tc, 0, x[0].astype(np.float64))) <= RMS_BOUND


def test_belt_tile_widths_give_identical_results_and_autotune(sk, tmp_path):
    import torch
    nside, tc = 256, 0.02
    V = oracle_table(nside, 2.5 * tc / 3 / ARCMIN, 768, 192, tc, 2048)
    k = sk.Kernel(sk.Geometry(sk._ctx, nside), V, tc)
    x = torch.from_numpy(white_noise_maps(nside, 2, 9)).cuda()
    ref = None
    for p in (5, 7, 9, 11, 13, 15, 17):
        k.set_tiles(belt_p=p)
        assert k.tiles()[0] == p
        y = sk.convolve(k, x)
        torch.cuda.synchronize()
        if ref is None:
            ref = y.clone()
        else:
            assert torch.equal(y, ref)                 # same summation order for every tile width
    cache = str(tmp_path / "tune.txt")
    p1 = k.autotune(x, cache_path=cache)
    c1 = k.config()
    p2 = k.autotune(x, cache_path=cache)               # second call is served by the cache
    assert p1 == p2 and p1 in (5, 7, 9, 11, 13, 15, 17) and k.config() == c1
    assert torch.equal(sk.convolve(k, x, path=sk.PATH_FP32), ref)
    # whichever form the tuner kept, PATH_AUTO runs it and meets the bound
    yo = O.conv_window(nside, V, tc, 0, x[1].cpu().numpy().astype(np.float64))
    assert rms_rel(sk.convolve(k, x)[1].cpu().numpy(), yo) <= RMS_BOUND
    sk._ctx.status()


# ------------------------------------------------------------------ batched tensor-core form

@pytest.mark.parametrize("nside,tc,batch,layout", [(32, 0.08, 40, 0), (64, 0.05, 33, 1), (128, 0.03, 32, 0),
                                                   (256, 0.02, 5, 0)])
def test_tensor_path_matches_oracle(sk, nside, tc, batch, layout):
    V = oracle_table(nside, 2.5 * tc / 3 / ARCMIN, 3 * nside, nside, tc, 1024, layout)
    k = sk.Kernel(sk.Geometry(sk._ctx, nside), V, tc, layout)
    x = white_noise_maps(nside, batch, 700 + nside)
    y = gpu_conv(sk, k, x, path=sk.PATH_TENSOR)
    yf = gpu_conv(sk, k, x, path=sk.PATH_FP32)
    for b in sorted({0, batch // 2, batch - 1}):
        yo = O.conv_window(nside, V, tc, layout, x[b].astype(np.float64))
        assert rms_rel(y[b], yo) <= RMS_BOUND, (b, rms_rel(y[b], yo))
    assert rms_rel(y, yf) <= RMS_BOUND


def test_tensor_path_n1024_batch_sampled(sk):
    grp = WORKLOADS["n1024x64_batched"].groups[0]
    ks = grp.kernel
    V = O.tabulate_real_kernel(ks.beam(), ks.lcut, ks.lmax, ks.theta_cut, ks.n_nodes, ks.layout)
    k = sk.Kernel(sk.Geometry(sk._ctx, grp.nside), V, ks.theta_cut, ks.layout)
    x = white_noise_maps(grp.nside, 64, grp.seed)
    y = gpu_conv(sk, k, x, path=sk.PATH_TENSOR)
    outs = sample_indices(x.shape[1], 3000, 303)
    for b in (0, 31, 32, 63):
        yo = O.conv_window(grp.nside, V, ks.theta_cut, ks.layout, x[b].astype(np.float64), outs)
        assert rms_rel(y[b][outs], yo) <= RMS_BOUND


# ------------------------------------------------------------------ stored cap weights

@pytest.mark.parametrize("nside,tc,nt,layout,batch", [
    (8, math.pi, 512, 0, 1), (16, 1.2, 512, 0, 1), (16, 0.2, 512, 1, 2), (32, 0.08, 1024, 0, 1),
    (64, 180 * ARCMIN, 4096, 0, 2), (128, 0.03, 2048, 1, 1), (256, 0.02, 16384, 0, 1), (512, 0.0262, 4096, 0, 3)])
def test_stored_cap_weights_equal_evaluated(sk, nside, tc, nt, layout, batch):
    # the stored weights are the evaluating kernel's FP32 weights, summed in the same
    # order per output (extra terms of the wider union windows have weight 0): the two
    # forms agree bit for bit, and both match the oracle
    import torch
    th = O.node_thetas(nt, tc, layout)
    V = (1.0 + 0.5 * np.cos(3.0 * th) - 0.2 * th) * O.taper(th, tc)
    k = sk.Kernel(sk.Geometry(sk._ctx, nside), V, tc, layout)
    assert k.cap_weight_bytes() > 0
    x = white_noise_maps(nside, batch, 1300 + nside)
    y_stored = gpu_conv(sk, k, x)
    k.set_cap_weights(False)
    assert k.cap_weight_bytes() == 0
    y_eval = gpu_conv(sk, k, x)
    assert np.array_equal(y_stored, y_eval)
    k.set_cap_weights(True)
    assert k.cap_weight_bytes() > 0
    assert np.array_equal(gpu_conv(sk, k, x), y_stored)
    yo = O.conv_window(nside, V, tc, layout, x[0].astype(np.float64))
    assert rms_rel(y_stored[0], yo) <= RMS_BOUND


def test_stored_cap_weights_follow_table_updates(sk):
    nside, tc, nt = 64, 0.06, 1024
    V1 = oracle_table(nside, 2.5 * tc / 3 / ARCMIN, 192, 48, tc, nt)
    V2 = oracle_table(nside, 3.0 * tc / 3 / ARCMIN, 192, 48, tc, nt)
    k = sk.Kernel(sk.Geometry(sk._ctx, nside), V1, tc)
    x = white_noise_maps(nside, 1, 77)
    k.update_values(V2)
    y = gpu_conv(sk, k, x)[0]
    assert rms_rel(y, O.conv_window(nside, V2, tc, 0, x[0].astype(np.float64))) <= RMS_BOUND


def test_pair_counts_by_launch_add_up(sk):
    for nside, tc in [(16, 1.2), (64, 0.05), (256, 0.02)]:
        k = sk.Kernel(sk.Geometry(sk._ctx, nside), np.ones(64), tc)
        by_launch = k.count_pairs_by_launch()
        by_path = k.count_pairs_by_path()
        assert sum(by_launch) == k.count_pairs() == sum(by_path)
        assert by_launch[0] == by_path[0] and by_launch[1] + by_launch[2] == by_path[1]
        assert by_launch[3] == by_path[2]


# ------------------------------------------------------------------ non-finite inputs

@pytest.mark.parametrize("path", [0, 2, 3])
def test_non_finite_input_stays_local(sk, path):
    # The sums multiply some pixels just outside an output's window by an exact zero (the
    # union windows of the caps and of the FP32 belt's ring pairs, the tensor belt's
    # 16-ring tiles), so a NaN input reaches a few outputs beyond its cut -- but no output
    # farther than theta_cut plus 20 pixel sizes, and every other output is bit-identical
    # to the run without it
    import torch
    nside, tc = 128, 0.03
    V = oracle_table(nside, 2.5 * tc / 3 / ARCMIN, 384, 96, tc, 2048)
    k = sk.Kernel(sk.Geometry(sk._ctx, nside), V, tc)
    x = white_noise_maps(nside, 1, 1601)
    vec = O.all_vecs(nside)
    reach = math.cos(tc + 20.0 * math.sqrt(4.0 * math.pi / x.shape[1]))
    for p in (5, 12 * nside * nside // 2 + 7, 12 * nside * nside - 3):     # cap, belt, south cap
        xn = x.copy()
        xn[0, p] = np.nan
        y = gpu_conv(sk, k, x, path)
        yn = gpu_conv(sk, k, xn, path)
        far = vec @ vec[p] < reach
        assert np.isnan(yn[0, p])
        assert np.array_equal(yn[0, far], y[0, far])
