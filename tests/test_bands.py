"""Ring-band decomposition of one map on the device (sk_convolve_rings).

Each band of output rings is computed from an input that holds the map on the band's
halo (the rings within theta_cut, Sec. 2) and zeros -- or unrelated finite values --
elsewhere, as a rank would hold it after the halo all-gather.  The stitched bands are
bit-identical to the full operator (the same work items, the same sums), and the full
operator matches the FP64 oracle at rms <= 1e-6.  The ranks run one after the other on
one device: no band waits on another.
"""
import numpy as np
import pytest

import oracle as O
from inputs import ARCMIN, gaussian_beam, white_noise_maps

pytestmark = pytest.mark.gpu


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


# (nside, FWHM', theta_cut', lmax, lcut, nodes, world, batch)
CASES = [
    (64, 240.0, 360.0, 128, 32, 2048, 3, 1),
    (256, 40.0, 60.0, 512, 128, 4096, 5, 2),
    (128, 60.0, 120.0, 256, 64, 4096, 16, 1),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("outside", ["zeros", "noise"])
def test_bands_stitch_to_the_full_operator(sk, case, outside):
    import torch
    from paper_1211_3556_b300.bands import ring_bands
    nside, fwhm, tcm, lmax, lcut, nt, world, batch = case
    tc = tcm * ARCMIN
    V = O.tabulate_real_kernel(gaussian_beam(fwhm, lmax), lcut, lmax, tc, nt, 0)
    g = sk.Geometry(sk._ctx, nside)
    k = sk.Kernel(g, V, tc, 0)
    x = white_noise_maps(nside, batch, 1300 + nside)
    xt = torch.from_numpy(x).cuda()
    y_full = sk.convolve(k, xt).cpu().numpy()
    stitched = np.full_like(y_full, np.nan)
    rng = np.random.default_rng(nside)
    for b in ring_bands(nside, tc, world):
        lo, hi = b.out_rings
        if hi == lo:
            continue
        if outside == "zeros":
            xm = np.zeros_like(x)
        else:
            xm = (1e3 * rng.standard_normal(x.shape)).astype(np.float32)
        p0, p1 = b.in_pix
        xm[:, p0:p1] = x[:, p0:p1]
        y = sk.convolve_rings(k, torch.from_numpy(xm).cuda(), lo, hi).cpu().numpy()
        q0, q1 = b.out_pix
        stitched[:, q0:q1] = y[:, q0:q1]
    sk._ctx.status()
    assert np.array_equal(stitched, y_full)
    for m in range(batch):
        outs = np.arange(0, g.npix, max(1, g.npix // 3000), dtype=np.int64)
        ref = O.conv_window(nside, V, tc, 0, x[m].astype(np.float64), outs=outs)
        assert rms_rel(stitched[m, outs], ref) <= 1e-6


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("form", ["fp32", "tensor"])
def test_symmetric_bands_stitch_to_the_full_operator(sk, case, form):
    # bands of a northern range and its mirror (convolve_rings_sym), from inputs that hold the
    # halo and noise elsewhere: stitched, bit-identical to the full operator -- with the belt
    # on the CUDA cores or on the tensor cores (the subset's ring groups only)
    import torch
    from paper_1211_3556_b300.bands import symmetric_bands
    nside, fwhm, tcm, lmax, lcut, nt, world, batch = case
    tc = tcm * ARCMIN
    V = O.tabulate_real_kernel(gaussian_beam(fwhm, lmax), lcut, lmax, tc, nt, 0)
    g = sk.Geometry(sk._ctx, nside)
    k = sk.Kernel(g, V, tc, 0)
    if form == "tensor":
        if not k.config()["tensor_form_available"]:
            pytest.skip("windows too wide for the tensor form")
        k.set_belt_form(sk.BELT_TENSOR)
    x = white_noise_maps(nside, batch, 1350 + nside)
    y_full = sk.convolve(k, torch.from_numpy(x).cuda()).cpu().numpy()
    stitched = np.full_like(y_full, np.nan)
    rng = np.random.default_rng(nside + 1)
    for b in symmetric_bands(nside, tc, world):
        lo, hi = b.north
        if hi == lo:
            continue
        xm = (1e3 * rng.standard_normal(x.shape)).astype(np.float32)
        for p0, p1 in b.in_pix:
            xm[:, p0:p1] = x[:, p0:p1]
        y = sk.convolve_rings_sym(k, torch.from_numpy(xm).cuda(), lo, hi).cpu().numpy()
        for q0, q1 in b.out_pix:
            assert np.all(np.isnan(stitched[:, q0:q1]))
            stitched[:, q0:q1] = y[:, q0:q1]
    sk._ctx.status()
    assert np.array_equal(stitched, y_full)


def test_convolve_rings_ranges(sk):
    import torch
    tc = 360.0 * ARCMIN
    V = O.tabulate_real_kernel(gaussian_beam(240.0, 128), 32, 128, tc, 2048, 0)
    g = sk.Geometry(sk._ctx, 64)
    k = sk.Kernel(g, V, tc, 0)
    x = torch.from_numpy(white_noise_maps(64, 1, 1400)).cuda()
    nr = 4 * 64 - 1
    y_full = sk.convolve(k, x).cpu().numpy()
    # the whole ring range is the full operator; single rings (a polar cap ring, a belt
    # ring, the equator) agree with it on the ring
    assert np.array_equal(sk.convolve_rings(k, x, 0, nr).cpu().numpy(), y_full)
    n, st, s, z, sn = g.rings()
    for r in (0, 5, 70, 2 * 64 - 1, nr - 1):
        out = torch.full_like(x, 3.0)
        sk.convolve_rings(k, x, r, r + 1, out=out)
        a, b = int(st[r]), int(st[r] + n[r])
        assert np.array_equal(out.cpu().numpy()[0, a:b], y_full[0, a:b])
    # an empty range writes nothing
    out = torch.full_like(x, 3.0)
    sk.convolve_rings(k, x, 10, 10, out=out)
    assert bool((out == 3.0).all())
    for lo, hi in ((-1, 4), (0, nr + 1), (9, 8)):
        with pytest.raises(sk.SkError):
            sk.convolve_rings(k, x, lo, hi)


def test_convolve_rings_sym_ranges(sk):
    import torch
    tc = 360.0 * ARCMIN
    V = O.tabulate_real_kernel(gaussian_beam(240.0, 128), 32, 128, tc, 2048, 0)
    g = sk.Geometry(sk._ctx, 64)
    k = sk.Kernel(g, V, tc, 0)
    x = torch.from_numpy(white_noise_maps(64, 1, 1401)).cuda()
    nr = 4 * 64 - 1
    y_full = sk.convolve(k, x).cpu().numpy()
    n, st, s, z, sn = g.rings()
    # the northern half with the equator and its mirror is the whole map
    assert np.array_equal(sk.convolve_rings_sym(k, x, 0, 2 * 64).cpu().numpy(), y_full)
    # a range that crosses the equator overlaps its mirror; single rings with their mirrors
    for lo, hi in ((100, 160), (0, 1), (40, 41), (127, 128)):
        out = torch.full_like(x, 3.0)
        sk.convolve_rings_sym(k, x, lo, hi, out=out)
        o = out.cpu().numpy()[0]
        for a, b in ((lo, hi), (nr - hi, nr - lo)):
            p, q = int(st[a]), int(st[b - 1] + n[b - 1])
            assert np.array_equal(o[p:q], y_full[0, p:q])
    out = torch.full_like(x, 3.0)
    sk.convolve_rings_sym(k, x, 7, 7, out=out)
    assert bool((out == 3.0).all())
    for lo, hi in ((-1, 4), (0, nr + 1), (9, 8)):
        with pytest.raises(sk.SkError):
            sk.convolve_rings_sym(k, x, lo, hi)
