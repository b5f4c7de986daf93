"""Ring-pair Fourier form of the belt (wide theta_cut) against the FP64 oracle.

The equatorial-zone rings go through their Fourier modes (Y_o(m) = sum_i W_oi(m)
X_i(m)); the other rings through the direct paths.  Bar: rms relative error <= 1e-6
against the oracle on the same FP32 input and FP64 table (FP32 FFTs of ~1e3 points
and FP32 mode sums over ~40 ring offsets add ~1e-7), and the same bar against the
direct sums.  Inputs: white-noise maps, Gaussian beams split at l_cut.
"""
import numpy as np
import pytest

import oracle as O
from inputs import ARCMIN, gaussian_beam, white_noise_maps

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


def build(sk, nside, fwhm, tc_arcmin, lmax, lcut, nt, layout=0):
    tc = tc_arcmin * ARCMIN
    V = O.tabulate_real_kernel(gaussian_beam(fwhm, lmax), lcut, lmax, tc, nt, layout)
    g = sk.Geometry(sk._ctx, nside)
    k = sk.Kernel(g, V, tc, layout)
    return g, k, V, tc


# (nside, FWHM', theta_cut', lmax, lcut, nodes, layout): windows of ~10-17 rings each side
CASES = [
    (32, 240.0, 720.0, 64, 16, 4096, 0),
    (64, 120.0, 600.0, 128, 32, 4096, 0),
    (64, 120.0, 600.0, 128, 32, 4096, 1),
]


@pytest.mark.parametrize("case", CASES)
def test_fourier_matches_oracle_and_direct(sk, case):
    import torch
    nside, fwhm, tcm, lmax, lcut, nt, layout = case
    g, k, V, tc = build(sk, nside, fwhm, tcm, lmax, lcut, nt, layout)
    f = sk.FourierBelt(k)
    info = f.info()
    assert info["rings"] > 0 and info["H"] >= 5
    x = white_noise_maps(nside, 2, 901 + nside)
    xt = torch.from_numpy(x).cuda()
    y = f.apply(xt)
    torch.cuda.synchronize()
    sk._ctx.status()
    yf = y.cpu().numpy().astype(np.float64)
    yd = sk.convolve(k, xt).cpu().numpy().astype(np.float64)
    for b in range(2):
        ref = O.conv_window(nside, V, tc, layout, x[b].astype(np.float64))
        assert rms_rel(yf[b], ref) <= RMS_BOUND
        # the Fourier rings themselves, against the oracle
        n, st, s, z, sn = g.rings()
        r0, r1 = info["first_ring"], info["first_ring"] + info["rings"]
        sl = slice(int(st[r0]), int(st[r1 - 1] + n[r1 - 1]))
        assert rms_rel(yf[b, sl], ref[sl]) <= RMS_BOUND
    assert rms_rel(yf, yd) <= RMS_BOUND


def test_fourier_batch_stride_and_per_map_identity(sk):
    import torch
    g, k, V, tc = build(sk, 32, 240.0, 720.0, 64, 16, 4096)
    f = sk.FourierBelt(k)
    npix = g.npix
    x = white_noise_maps(32, 3, 911)
    stride = npix + 12
    buf = torch.zeros(3, stride, device="cuda")
    buf[:, :npix] = torch.from_numpy(x).cuda()
    out = torch.full((3, stride), 7.0, device="cuda")
    f.apply(buf[:, :npix], out=out[:, :npix])
    torch.cuda.synchronize()
    sk._ctx.status()
    yb = out.cpu().numpy()
    assert np.all(yb[:, npix:] == 7.0)                 # padding untouched
    for b in range(3):
        y1 = f.apply(torch.from_numpy(x[b:b + 1]).cuda()).cpu().numpy()
        assert np.array_equal(yb[b, :npix], y1[0])      # same FFTs and sums per map


def test_fourier_without_zone_rings_is_the_direct_operator(sk):
    # Nside 16 with theta_cut 80 deg: no output ring has its whole window in the zone
    import torch
    g, k, V, tc = build(sk, 16, 1200.0, 4800.0, 32, 8, 2048)
    f = sk.FourierBelt(k)
    assert f.info()["rings"] == 0 and f.info()["bytes"] == 0
    x = white_noise_maps(16, 1, 921)
    y = f.apply(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    ref = O.conv_window(16, V, tc, 0, x[0].astype(np.float64))
    assert rms_rel(y[0], ref) <= RMS_BOUND


def test_fourier_argument_errors(sk):
    import torch
    g, k, V, tc = build(sk, 32, 240.0, 720.0, 64, 16, 4096)
    f = sk.FourierBelt(k)
    x = torch.zeros(1, g.npix, device="cuda")
    with pytest.raises(sk.SkError):
        f.apply(x, out=x)                               # aliasing
    with pytest.raises(ValueError):
        f.apply(torch.zeros(1, g.npix - 4, device="cuda"))


def test_wide_workload_sampled_outputs(sk):
    # the 300' workload at Nside 1024: zone rings (Fourier form) and the other rings (the
    # direct sums, summing each input ring apart over the ~2.4e4 neighbours of a pixel at
    # this cut) on sampled outputs against the oracle
    import torch
    from inputs import WORKLOADS, make_maps, sample_indices
    grp = WORKLOADS["n1024_wide"].groups[0]
    ks = grp.kernel
    V = O.tabulate_real_kernel(ks.beam(), ks.lcut, ks.lmax, ks.theta_cut, ks.n_nodes, ks.layout)
    g = sk.Geometry(sk._ctx, grp.nside)
    k = sk.Kernel(g, V, ks.theta_cut, ks.layout)
    f = sk.FourierBelt(k)
    info = f.info()
    assert info["rings"] > 1000
    x = make_maps(grp)
    y = f.apply(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)[0]
    sk._ctx.status()
    n, st, s, z, sn = g.rings()
    r0, r1 = info["first_ring"], info["first_ring"] + info["rings"]
    p0, p1 = int(st[r0]), int(st[r1 - 1] + n[r1 - 1])
    zone = p0 + sample_indices(p1 - p0, 600, 602)
    other = sample_indices(g.npix, 1200, 603)
    other = other[(other < p0) | (other >= p1)][:400]
    xs = x[0].astype(np.float64)
    assert rms_rel(y[zone], O.conv_window(grp.nside, V, ks.theta_cut, 0, xs, outs=zone)) <= RMS_BOUND
    assert rms_rel(y[other], O.conv_window(grp.nside, V, ks.theta_cut, 0, xs, outs=other)) <= RMS_BOUND


def test_table1_point_sampled_outputs(sk):
    # Sec. 4, Table 1's optimum split for a 7' beam at Planck resolution (l_cut 1158,
    # theta_cut 390', Nside 2048): the real-space part by the ring-pair Fourier zone and the
    # direct sums elsewhere, on sampled outputs against the oracle
    import torch
    from inputs import WORKLOADS, make_maps, sample_indices
    grp = WORKLOADS["n2048_table1"].groups[0]
    ks = grp.kernel
    g = sk.Geometry(sk._ctx, grp.nside)
    k, V = sk.Kernel.from_legendre(g, ks.beam(), ks.lcut + 1, ks.lmax, ks.n_nodes, ks.theta_cut, ks.layout)
    f = sk.FourierBelt(k)
    x = make_maps(grp)
    y = f.apply(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)[0]
    sk._ctx.status()
    del f
    outs = sample_indices(g.npix, 240, 803)
    yo = O.conv_window(grp.nside, np.asarray(V, np.float64), ks.theta_cut, ks.layout, x[0].astype(np.float64), outs)
    assert rms_rel(y[outs], yo) <= RMS_BOUND
