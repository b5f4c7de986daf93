"""Harmonic half of the split (Sec. 2, Eq. 1) on the GPU against the FP64 oracle.

The oracle's `sht_convolve` is the plain pixel-sum transform with real
orthonormal harmonics (pinned in test_oracle_pins by the addition theorem).
The GPU transform works in FP32 (ring DFTs, Legendre sums over up to 2 Nside
rings with an FP32 table of lambda_lm): its error is a few FP32 roundings per
accumulated term, ~1e-7..1e-6 relative in rms; the bar here is 1e-5.
"""
import math

import numpy as np
import pytest

import oracle as O
from inputs import ARCMIN, gaussian_beam, white_noise_maps

pytestmark = pytest.mark.gpu

HARM_BOUND = 1e-5


@pytest.fixture(scope="module")
def sk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1211_3556_b300 as sk
    sk._hctx = sk.Context(0)
    yield sk
    torch.cuda.synchronize()


def rms_rel(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_harm(sk, nside, kl, lmax, x, accumulate_into=None):
    import torch
    g = sk.Geometry(sk._hctx, nside)
    h = sk.Harmonic(sk._hctx, g, kl, lmax)
    xt = torch.from_numpy(np.ascontiguousarray(np.atleast_2d(x), np.float32)).cuda()
    if accumulate_into is None:
        y = h.apply(xt)
    else:
        y = torch.from_numpy(np.ascontiguousarray(accumulate_into, np.float32)).cuda()
        h.apply(xt, out=y, accumulate=True)
    torch.cuda.synchronize()
    sk._hctx.status()
    return y.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("nside,lmax", [(2, 3), (4, 7), (8, 12), (16, 31), (32, 40)])
def test_harmonic_matches_oracle_sht(sk, nside, lmax):
    rng = np.random.default_rng(700 + nside)
    kl = rng.uniform(0.2, 1.0, lmax + 1)
    x = white_noise_maps(nside, 1, 710 + nside)[0]
    y = run_harm(sk, nside, kl, lmax, x)[0]
    ref = O.sht_convolve(nside, x.astype(np.float64), kl, lmax)
    assert rms_rel(y, ref) <= HARM_BOUND


def test_harmonic_single_multipole(sk):
    # K^_l = 1 at one l only: the output is the projection of x on that multipole
    nside, lmax = 16, 20
    for ell in (0, 1, 7, 20):
        kl = np.zeros(lmax + 1); kl[ell] = 1.0
        x = white_noise_maps(nside, 1, 720 + ell)[0]
        y = run_harm(sk, nside, kl, lmax, x)[0]
        ref = O.sht_convolve(nside, x.astype(np.float64), kl, lmax)
        assert rms_rel(y, ref) <= HARM_BOUND


def test_harmonic_batch_stride_and_accumulate(sk):
    import torch
    nside, lmax, batch = 8, 15, 3
    npix = 12 * nside * nside
    stride = npix + 4
    kl = np.linspace(1.0, 0.1, lmax + 1)
    xs = white_noise_maps(nside, batch, 730)
    base = white_noise_maps(nside, batch, 731)
    g = sk.Geometry(sk._hctx, nside)
    h = sk.Harmonic(sk._hctx, g, kl, lmax)
    xt = torch.zeros(batch, stride, dtype=torch.float32, device="cuda")
    yt = torch.zeros(batch, stride, dtype=torch.float32, device="cuda")
    xt[:, :npix] = torch.from_numpy(xs).cuda()
    yt[:, :npix] = torch.from_numpy(base).cuda()
    h.apply(xt, out=yt, accumulate=True)
    torch.cuda.synchronize()
    y = yt[:, :npix].cpu().numpy().astype(np.float64)
    for b in range(batch):
        ref = base[b].astype(np.float64) + O.sht_convolve(nside, xs[b].astype(np.float64), kl, lmax)
        assert rms_rel(y[b], ref) <= HARM_BOUND
    assert float(yt[:, npix:].abs().max()) == 0.0      # padding untouched


def test_split_assembly_matches_oracle(sk):
    # The whole split of Eq. 1 for a Gaussian beam: real-space part (tabulated,
    # tapered) + harmonic part K^_l = b_l - R_l, both sides from the same tables.
    import torch
    nside, fwhm, nt = 32, 278.0, 2048
    tc = 3.0 * fwhm * ARCMIN
    lmax, lcut = 64, 32
    bl = gaussian_beam(fwhm, lmax)
    V = O.tabulate_real_kernel(bl, lcut, lmax, tc, nt, 0)
    R = O.kernel_response(V, tc, 0, lmax)
    kh = O.harmonic_part(bl, R, lcut)
    x = white_noise_maps(nside, 1, 740)[0]
    g = sk.Geometry(sk._hctx, nside)
    k = sk.Kernel(g, V, tc)
    h = sk.Harmonic(sk._hctx, g, kh, lcut)
    xt = torch.from_numpy(x).cuda()
    y = sk.split_convolve(k, h, xt)
    torch.cuda.synchronize()
    y = y.cpu().numpy().astype(np.float64)
    xd = x.astype(np.float64)
    ref = O.conv_window(nside, V, tc, 0, xd) + O.sht_convolve(nside, xd, kh, lcut)
    assert rms_rel(y, ref) <= HARM_BOUND
    # the split's own error against the full band-limited convolution is of the size
    # Eq. 2 predicts (sigma_rms from K~_l = K^_l + R_l, within its factor alpha = 5)
    full = O.sht_convolve(nside, xd, bl, lmax)
    err = rms_rel(ref, full)
    est = O.relative_error_estimate(bl, kh + R[: lmax + 1]) / 5.0
    assert est / 5.0 <= err <= est * 5.0


@pytest.mark.parametrize("layout", [0, 1])
def test_kernel_response_matches_oracle(sk, layout):
    # R_l of the real-space part: both sides FP64 Gauss-Legendre on every node interval
    nside, fwhm, nt, lmax, lcut = 64, 60.0, 1024, 192, 96
    tc = 180.0 * ARCMIN
    bl = gaussian_beam(fwhm, lmax)
    V = O.tabulate_real_kernel(bl, lcut, lmax, tc, nt, layout)
    g = sk.Geometry(sk._hctx, nside)
    k = sk.Kernel(g, V, tc, layout)
    R = sk.kernel_response(k, lmax)
    Ro = O.kernel_response(V, tc, layout, lmax)
    assert float(np.max(np.abs(R - Ro))) <= 1e-12 * float(np.max(np.abs(Ro)))


def test_harmonic_argument_errors(sk):
    import torch
    g1 = sk.Geometry(sk._hctx, 1)
    with pytest.raises(sk.SkError):
        sk.Harmonic(sk._hctx, g1, np.ones(2), 1)          # nside below 2
    g = sk.Geometry(sk._hctx, 4)
    with pytest.raises(sk.SkError):
        sk.Harmonic(sk._hctx, g, np.ones(9), 8)           # lmax > 2 nside - 1
    h = sk.Harmonic(sk._hctx, g, np.ones(8), 7)
    x = torch.zeros(192, dtype=torch.float32, device="cuda")
    with pytest.raises(sk.SkError):
        h.apply(x, out=x)                                  # aliasing
    assert h.table_bytes() == 4 * (8 * 9 // 2) * 8


# ------------------------------------------------ least-squares real-space part

@pytest.mark.parametrize("fwhm,tcf,lcut,lfit,nb", [(60.0, 3.0, 96, 384, 129), (7.1, 2.8, 1024, 4096, 257)])
def test_fit_matches_oracle(sk, fwhm, tcf, lcut, lfit, nb):
    # Cholesky of the normal equations (library) vs lstsq (oracle) on the same
    # objective: the same Eq. 2 residual, and tables with the same response above l_cut
    tc = tcf * fwhm * ARCMIN
    kl = gaussian_beam(fwhm, lfit)
    nt = 4 * (nb - 1) + 1
    V, sig = sk.fit_real_kernel(sk._hctx, kl, lcut, tc, n_basis=nb, nt_out=nt, lfit=lfit)
    Vo, sigo = O.fit_real_kernel(kl, lcut, lfit, tc, nb, nt)
    assert abs(sig - sigo) <= 1e-3 * sigo + 1e-12
    R = O.kernel_response(V, tc, 0, lfit)
    Ro = O.kernel_response(Vo, tc, 0, lfit)
    ell = np.arange(lcut + 1, lfit + 1)
    w = 2 * ell + 1
    den = math.sqrt(np.sum((2 * np.arange(lfit + 1) + 1) * kl ** 2))
    assert math.sqrt(np.sum(w * (R[lcut + 1:] - Ro[lcut + 1:]) ** 2)) <= 1e-6 * den


def test_fit_planted_response(sk):
    nb, tc, lcut, lfit = 33, 0.3, 10, 120
    M = O.hat_response_matrix(nb, tc, 0, lfit)
    kl = M @ (10.0 * np.sin(np.linspace(0.0, 3.0, nb - 1)))
    V, sig = sk.fit_real_kernel(sk._hctx, kl, lcut, tc, n_basis=nb, nt_out=nb, lfit=lfit)
    assert sig < 1e-6


def test_plan_split_picks_the_fastest_feasible_candidate(sk):
    nside = 32
    g = sk.Geometry(sk._hctx, nside)
    kl = gaussian_beam(300.0, 4 * nside)
    best, rows = sk.plan_split(sk._hctx, g, kl, 1e-2, [16, 24], [600.0 * ARCMIN, 900.0 * ARCMIN],
                               n_basis=65, reps=2)
    assert len(rows) == 4
    ok = [r for r in rows if r["sigma"] <= 1e-2]
    assert ok and best is not None
    assert best["ms_total"] == min(r["ms_total"] for r in ok)
    for r in rows:
        assert r["ms_real"] > 0 and r["ms_harmonic"] > 0


# ------------------------------------------------------------------ larger maps, spectra

@pytest.mark.parametrize("nside,lmax", [(128, 200), (256, 383)])
def test_harmonic_matches_ring_oracle_above_nside_32(sk, nside, lmax):
    # the oracle's ring-by-ring FP64 transform (the pixel-sum transform rewritten with ring
    # FFTs, pinned to the brute-force one on the CPU): y = synthesis(K^_l analysis(x))
    kl = np.exp(-np.arange(lmax + 1) / (0.4 * lmax)) * (1.0 + 0.3 * np.cos(np.arange(lmax + 1) / 7.0))
    x = white_noise_maps(nside, 1, 730 + nside)[0]
    y = run_harm(sk, nside, kl, lmax, x)[0]
    a = O.sht_analysis_rings(nside, x.astype(np.float64), lmax)
    ref = O.sht_synthesis_rings(nside, a, lmax, kl)
    assert rms_rel(y, ref) <= HARM_BOUND


def test_harmonic_at_the_split_workloads_nside(sk):
    # Nside 2048, the split workload's geometry -- 2047 cap rings through chirp-z transforms
    # in several FFT-length classes, the 4097 zone rings through 8192-point FFTs, the lambda
    # table's row starts -- at a band limit the oracle's FP64 ring transform finishes in
    # seconds (the workload's l_cut of 1024 would take it minutes)
    nside, lmax = 2048, 160
    kl = np.exp(-np.arange(lmax + 1) / (0.4 * lmax)) * (1.0 + 0.3 * np.cos(np.arange(lmax + 1) / 5.0))
    x = white_noise_maps(nside, 1, 740)[0]
    y = run_harm(sk, nside, kl, lmax, x)[0]
    a = O.sht_analysis_rings(nside, x.astype(np.float64), lmax)
    ref = O.sht_synthesis_rings(nside, a, lmax, kl)
    assert rms_rel(y, ref) <= HARM_BOUND


@pytest.mark.parametrize("nside,lmax", [(32, 63), (128, 255)])
def test_power_spectrum_matches_oracle(sk, nside, lmax):
    import torch
    g = sk.Geometry(sk._hctx, nside)
    h = sk.Harmonic(sk._hctx, g, np.ones(lmax + 1), lmax)
    x = white_noise_maps(nside, 2, 740 + nside)
    cl = h.spectrum(torch.from_numpy(x).cuda()).cpu().numpy()
    torch.cuda.synchronize()
    sk._hctx.status()
    for b in range(2):
        ref = O.power_spectrum(O.sht_analysis_rings(nside, x[b].astype(np.float64), lmax), lmax)
        assert np.abs(cl[b] - ref).max() <= 1e-5 * ref.max()
        assert np.abs(cl[b] / ref - 1.0).max() <= 1e-4       # every l: white noise keeps C_l ~ 1
