"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Each test ties one oracle function to something other than itself, so that a
plausible mistake (dropped term, wrong sign or index, transposed operand) fails
at least one of them:

* HEALPix RING geometry (the pixelisation of Sec. 2): golden base-pixel centres
  and ring tables written from the closed forms of Gorski et al. 2005,
  counting identities, mirror symmetry, sum of unit vectors.
* Legendre operator P_{l theta} (Eq. 1): P_l(1) = 1, P_l(-1) = (-1)^l, the
  generating function, Gauss-Legendre orthogonality and the K_l round trip.
* Kernel response R_l (Eq. 1 applied to the truncated real-space kernel):
  the closed form for a constant kernel on a cap.
* Pair sums: brute force vs windowed, closed-form angles between base pixels
  (delta maps), symmetry of the operator, a constant map against the cap area,
  spherical harmonics as eigenfunctions (Funk-Hecke), linearity.
* SHT: the addition theorem against the Bonnet recurrence; harmonic-space
  convolution against the all-pairs sum of its real-space kernel.
* Gradient: central differences of a quadratic loss (exact up to rounding).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from inputs import gaussian_beam, white_noise_maps

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ARCMIN = math.pi / 10800.0


def _load(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(t) for t in line.split()])
    return np.array(rows)


# ----------------------------------------------------------------- geometry

def test_base_pixel_centres_golden():
    g = _load("healpix_nside1_centres.txt")
    for p, zn, zd, phi_pi in g:
        th, ph = O.pix2ang(1, int(p))
        assert math.cos(th) == pytest.approx(zn / zd, abs=1e-15)
        assert ph == pytest.approx(phi_pi * math.pi, abs=1e-15)


def test_nside2_ring_table_golden():
    g = _load("healpix_nside2_rings.txt")
    for r, n, st, zn, zd, phi0 in g:
        n_, st_, s_, z_, sn_ = O.ring_info(2, int(r))
        assert (n_, st_) == (int(n), int(st))
        assert z_ == pytest.approx(zn / zd, abs=1e-15)
        th, ph = O.pix2ang(2, st_)
        assert ph == pytest.approx(phi0 * math.pi, abs=1e-15)
        assert sn_ == pytest.approx(math.sqrt(1 - (zn / zd) ** 2), abs=1e-15)


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 64, 1024])
def test_ring_counts_and_mirror(nside):
    N = nside
    assert O.npix(N) == 12 * N * N
    total, prev_end = 0, 0
    for r in range(1, 4 * N):
        n, st, s, z, sn = O.ring_info(N, r)
        assert st == prev_end                    # rings tile the pixel range
        prev_end = st + n
        total += n
        n2, st2, s2, z2, sn2 = O.ring_info(N, 4 * N - r)
        assert n2 == n and s2 == s and z2 == -z and sn2 == sn  # N/S mirror
        assert st % 4 == 0 and n % 4 == 0
    assert total == 12 * N * N


@pytest.mark.parametrize("nside", [1, 2, 8, 32])
def test_unit_vectors(nside):
    v = O.all_vecs(nside)
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-15)
    assert np.abs(v.sum(axis=0)).max() < 1e-12           # centres are symmetric
    # pixel -> (ring, j) -> pixel round trip
    for p in [0, 1, O.npix(nside) // 2, O.npix(nside) - 1]:
        r, j = O.pix2ring(nside, p)
        n, st, *_ = O.ring_info(nside, r)
        assert st + j == p and 0 <= j < n


# ----------------------------------------------------------------- Legendre

def test_legendre_endpoints_and_generating_function():
    lmax = 300
    P = O.legendre_P(lmax, np.array([1.0, -1.0]))
    assert np.allclose(P[:, 0], 1.0, atol=1e-13)
    assert np.allclose(P[:, 1], (-1.0) ** np.arange(lmax + 1), atol=1e-13)
    # sum_l t^l P_l(x) = (1 - 2xt + t^2)^(-1/2): with coef_l = 4 pi t^l / (2l+1)
    t = 0.5
    coef = 4 * math.pi * t ** np.arange(lmax + 1) / (2 * np.arange(lmax + 1) + 1)
    th = np.linspace(0.0, math.pi, 37)
    got = O.legendre_series(coef, 0, lmax, th)
    want = 1.0 / np.sqrt(1 - 2 * np.cos(th) * t + t * t)
    assert np.allclose(got, want, rtol=1e-13, atol=0)


def test_legendre_orthogonality_gauss():
    lmax = 64
    x, w = np.polynomial.legendre.leggauss(lmax + 1)
    P = O.legendre_P(lmax, x)
    G = (P * w) @ P.T
    want = np.diag(2.0 / (2 * np.arange(lmax + 1) + 1))
    assert np.abs(G - want).max() < 1e-13


def test_legendre_round_trip_of_kernel():
    """2 pi int K(theta) P_l(cos theta) sin theta dtheta = K_l for the full series."""
    lmax = 96
    k_ell = gaussian_beam(60.0, lmax)
    x, w = np.polynomial.legendre.leggauss(lmax + 2)
    K = O.legendre_series(k_ell, 0, lmax, np.arccos(x))
    P = O.legendre_P(lmax, x)
    back = 2 * math.pi * (P * w) @ K
    assert np.allclose(back, k_ell, rtol=0, atol=1e-13 * np.abs(K).sum() / len(K) * lmax)


def test_small_angle_limit_is_gaussian_beam():
    """For a wide-band Gaussian beam the series approaches the flat-sky Gaussian
    exp(-theta^2 / 2 sigma^2) / (2 pi sigma^2) near theta = 0."""
    fwhm = 60.0
    lmax = 2000
    k_ell = gaussian_beam(fwhm, lmax)
    sig = fwhm * ARCMIN / math.sqrt(8 * math.log(2))
    th = np.array([0.0, 0.5 * sig, sig])
    got = O.legendre_series(k_ell, 0, lmax, th)
    want = np.exp(-th ** 2 / (2 * sig * sig)) / (2 * math.pi * sig * sig)
    assert np.allclose(got, want, rtol=2e-3)


def test_nodes_and_coordinates():
    tc = 0.01
    for layout, nt in [(0, 17), (1, 32), (1, 33)]:
        th = O.node_thetas(nt, tc, layout)
        assert th[0] == 0.0 and th[-1] == pytest.approx(tc, rel=1e-15)
        assert np.all(np.diff(th) > 0)
        L = O.lib()
        for k, t in enumerate(th):
            assert L.or_node_coord(t, nt, tc, layout) == pytest.approx(k, abs=1e-9)
        if layout == 1:
            M = nt // 2
            assert th[M] == pytest.approx(tc / 16, rel=1e-14)   # half the nodes in 1/16


def test_klin_interpolates_linearly_and_cuts():
    tc = 0.02
    for layout in (0, 1):
        th = O.node_thetas(64, tc, layout)
        V = 3.0 * th - 1.0                       # linear: interpolation is exact
        q = np.linspace(0, tc, 101)
        assert np.allclose(O.klin(V, tc, layout, q), 3.0 * q - 1.0, atol=1e-14)
        assert O.klin(V, tc, layout, [tc * (1 + 1e-12)])[0] == 0.0


# ----------------------------------------------------------------- response / split

def test_response_of_constant_kernel_closed_form():
    """R_l of K_lin = 1 on [0, theta_cut] is 2 pi (P_{l-1}(c) - P_{l+1}(c)) / (2l+1),
    c = cos theta_cut ((2l+1) P_l = P'_{l+1} - P'_{l-1}); R_0 = 2 pi (1 - c)."""
    tc = 0.3
    lmax = 40
    V = np.ones(33)
    R = O.kernel_response(V, tc, 0, lmax)
    c = math.cos(tc)
    P = O.legendre_P(lmax + 1, np.array([c]))[:, 0]
    want = np.empty(lmax + 1)
    want[0] = 2 * math.pi * (1 - c)
    for l in range(1, lmax + 1):
        want[l] = 2 * math.pi * (P[l - 1] - P[l + 1]) / (2 * l + 1)
    assert np.allclose(R, want, rtol=0, atol=1e-13)


def test_split_reproduces_kernel_below_lcut():
    """K~_l = K^_l + P_{l theta} K^_theta equals K_l exactly for l <= l_cut (Eq. 1)."""
    lmax, lcut, tc = 192, 96, 180 * ARCMIN
    b = gaussian_beam(60.0, lmax)
    V = O.tabulate_real_kernel(b, lcut, lmax, tc, 1024)
    R = O.kernel_response(V, tc, 0, lmax)
    kh = O.harmonic_part(b, R, lcut)
    assert np.allclose((kh + R)[: lcut + 1], b[: lcut + 1], rtol=0, atol=1e-15)
    assert np.all(kh[lcut + 1:] == 0)
    # the tabulated real-space kernel vanishes at theta_cut (tapered)
    assert V[-1] == 0.0


def test_tabulation_l_range_and_taper_against_scipy():
    """The tabulated real-space part at nodes that fall on the taper's closed-form
    points: with 21 uniform nodes, theta_18 = 0.9 theta_cut (taper 1), theta_19 =
    0.95 theta_cut (taper (1 + cos(pi/2)) / 2 = 1/2) and theta_20 = theta_cut (0).
    The series sum_{l = l_cut + 1}^{l_max} (2l+1)/(4 pi) b_l P_l(cos theta) is
    evaluated independently with scipy's Legendre polynomials; starting the sum at
    l_cut (one term too many) or a different taper moves these values."""
    from scipy.special import eval_legendre
    lmax, lcut, tc = 64, 16, 0.5
    b = gaussian_beam(120.0, lmax)
    V = O.tabulate_real_kernel(b, lcut, lmax, tc, 21)
    th = tc * np.arange(21) / 20.0
    ell = np.arange(lcut + 1, lmax + 1)
    series = np.array([np.sum((2 * ell + 1) / (4 * math.pi) * b[ell] * eval_legendre(ell, math.cos(t)))
                       for t in th])
    w = np.ones(21)
    w[19], w[20] = 0.5, 0.0
    assert np.allclose(V, series * w, rtol=1e-12, atol=1e-12 * np.abs(series).max())
    # the l_cut term alone is far above that tolerance (the pin sees an off-by-one)
    extra = (2 * lcut + 1) / (4 * math.pi) * b[lcut] * eval_legendre(lcut, np.cos(th[:19]))
    assert np.abs(extra).max() > 1e-3 * np.abs(series).max()
    # the taper's shape between its closed-form points: (1 + cos(pi u)) / 2, u = (theta - 0.9 tc) / (0.1 tc)
    u = np.array([0.0, 0.25, 0.5, 0.75, 1.0])
    tq = (0.9 + 0.1 * u) * tc
    assert np.allclose(O.taper(tq, tc), [1.0, (1 + math.sqrt(0.5)) / 2, 0.5, (1 - math.sqrt(0.5)) / 2, 0.0],
                       rtol=0, atol=1e-15)


def test_whole_sphere_high_pass_response_is_the_beam_above_lcut():
    """With theta_cut = pi and no taper, the real-space part is the whole l > l_cut
    series, so by orthogonality of the P_l its response is b_l for l_cut < l <= l_max
    and 0 for l <= l_cut (and above l_max), up to the quadrature error of the
    piecewise-linear table (16384 nodes: below 1e-4 of the largest b_l here).  An
    l range that starts at l_cut or stops before l_max fails the first check."""
    lmax, lcut = 40, 12
    b = gaussian_beam(300.0, lmax)
    V = O.tabulate_real_kernel(b, lcut, lmax, math.pi, 16384, taper_start=1.0)
    R = O.kernel_response(V, math.pi, 0, lmax + 8)
    tol = 1e-4 * b.max()
    assert np.abs(R[lcut + 1: lmax + 1] - b[lcut + 1:]).max() <= tol
    assert np.abs(R[: lcut + 1]).max() <= tol
    assert np.abs(R[lmax + 1:]).max() <= tol
    assert b[lcut] > 100 * tol and b[lmax] > 100 * tol       # both ends of the range are visible


def test_relative_error_estimate_definition():
    k = np.ones(11)
    assert O.relative_error_estimate(k, k) == 0.0
    # K~ = K (1 + eps) everywhere: sigma = alpha * eps
    assert O.relative_error_estimate(k, 1.001 * k, alpha=5.0) == pytest.approx(0.005, rel=1e-12)


# ----------------------------------------------------------------- pair sums

@pytest.mark.parametrize("nside,tc_deg,layout", [(2, 50.0, 0), (4, 40.0, 1), (4, 120.0, 0),
                                                 (8, 15.0, 0), (8, 179.0, 1), (16, 6.0, 1)])
def test_brute_equals_window(nside, tc_deg, layout):
    tc = math.radians(tc_deg)
    nt = 256
    rng = np.random.default_rng(7)
    V = rng.standard_normal(nt)
    x = rng.standard_normal(O.npix(nside))
    yb = O.conv_brute(nside, V, tc, layout, x)
    yw = O.conv_window(nside, V, tc, layout, x)
    assert np.allclose(yw, yb, rtol=0, atol=1e-13 * np.abs(yb).max())
    outs = np.array([0, 3, O.npix(nside) // 2, O.npix(nside) - 1])
    assert np.allclose(O.conv_window(nside, V, tc, layout, x, outs), yb[outs], rtol=0,
                       atol=1e-13 * np.abs(yb).max())


def test_delta_maps_closed_form_angles():
    """Nside 1, K_lin(theta) = theta (linear table): a delta at pixel i gives
    y_o = dOmega * gamma_oi, with gamma between base-pixel centres in closed form:
    cos gamma(0,1) = 4/9, cos gamma(0,4) = sqrt(10)/6, cos gamma(0,2) = -1/9,
    cos gamma(0,8) = -4/9 + 5/9 * cos(0) = 1/9."""
    tc = math.pi
    th = O.node_thetas(16, tc, 0)
    V = th.copy()
    dOm = 4 * math.pi / 12
    cases = {1: math.acos(4 / 9), 4: math.acos(math.sqrt(10) / 6), 2: math.acos(-1 / 9),
             8: math.acos(1 / 9), 0: 0.0}
    for i, g in cases.items():
        x = np.zeros(12); x[i] = 1.0
        y = O.conv_brute(1, V, tc, 0, x)
        assert y[0] == pytest.approx(dOm * g, rel=1e-13, abs=1e-15)


def test_delta_map_cut_excludes_far_pixels():
    tc = math.acos(4 / 9) - 1e-9          # just below gamma(0,1)
    V = np.ones(8)
    x = np.zeros(12); x[1] = 1.0
    y = O.conv_window(1, V, tc, 0, x)
    assert y[0] == 0.0 and y[1] == pytest.approx(4 * math.pi / 12)


@pytest.mark.parametrize("nside,tc", [(8, 0.4), (16, 0.15), (32, 0.08)])
def test_operator_symmetry(nside, tc):
    rng = np.random.default_rng(3)
    V = rng.standard_normal(64)
    a = rng.standard_normal(O.npix(nside)); b = rng.standard_normal(O.npix(nside))
    Aa = O.conv_window(nside, V, tc, 0, a)
    Ab = O.conv_window(nside, V, tc, 0, b)
    assert abs(Aa @ b - a @ Ab) <= 1e-13 * np.abs(Aa).sum() * np.abs(b).max()


def test_linearity():
    rng = np.random.default_rng(4)
    V = rng.standard_normal(64)
    a = rng.standard_normal(O.npix(8)); b = rng.standard_normal(O.npix(8))
    y = O.conv_window(8, V, 0.3, 1, 2.0 * a - 3.0 * b)
    assert np.allclose(y, 2.0 * O.conv_window(8, V, 0.3, 1, a) - 3.0 * O.conv_window(8, V, 0.3, 1, b),
                       atol=1e-12)


def test_constant_map_converges_to_cap_area():
    """A constant kernel and map give dOmega * (#pixels in the cap) ~ 2 pi (1 - cos tc),
    with an error that falls as Nside grows."""
    tc = 0.2
    V = np.ones(8)
    want = 2 * math.pi * (1 - math.cos(tc))
    errs = []
    for nside in (16, 32, 64):
        y = O.conv_window(nside, V, tc, 0, np.ones(O.npix(nside)))
        errs.append(np.sqrt(np.mean((y / want - 1) ** 2)))
    assert errs[2] < errs[1] < errs[0] and errs[2] < 0.02


def test_spherical_harmonics_are_eigenfunctions():
    """Funk-Hecke: A Y_lm ~ R_l Y_lm with R_l the kernel response; the pixel
    quadrature error falls as Nside grows."""
    tc = 0.5
    th_n = O.node_thetas(512, tc, 0)
    V = np.cos(3.0 * th_n) * (1 - th_n / tc)
    lmax = 6
    R = O.kernel_response(V, tc, 0, lmax)
    errs = []
    for nside in (8, 16, 32):
        th, ph = O.pixel_angles(nside)
        Y = O.real_ylm(lmax, th, ph)
        idx = 0
        e = []
        for l in range(lmax + 1):
            for m in range(-l, l + 1):
                y = O.conv_window(nside, V, tc, 0, Y[idx])
                e.append(np.linalg.norm(y - R[l] * Y[idx]) / np.linalg.norm(R[0] * Y[idx]))
                idx += 1
        errs.append(max(e))
    assert errs[2] < errs[1] < errs[0] and errs[2] < 0.05


def test_pair_count_matches_cap_area():
    nside, tc = 32, 0.12
    c = O.count_pairs(nside, tc)
    want = O.npix(nside) * 2 * math.pi * (1 - math.cos(tc)) / (4 * math.pi / O.npix(nside))
    assert abs(c / want - 1) < 0.03          # pixel-counting error at ~4 px radius
    outs = np.arange(0, O.npix(nside), 97)
    per = [O.count_pairs(nside, tc, [o]) for o in outs[:5]]
    assert O.count_pairs(nside, tc, outs[:5]) == sum(per)


# ----------------------------------------------------------------- SHT

def test_addition_theorem():
    """sum_m Y_lm(p) Y_lm(p') = (2l+1)/(4 pi) P_l(p . p') (real harmonics)."""
    lmax = 12
    rng = np.random.default_rng(9)
    th = np.arccos(rng.uniform(-1, 1, 6)); ph = rng.uniform(0, 2 * math.pi, 6)
    Y = O.real_ylm(lmax, th, ph)
    v = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    P = O.legendre_P(lmax, np.clip(v @ v.T, -1, 1))
    idx = 0
    for l in range(lmax + 1):
        blk = Y[idx: idx + 2 * l + 1]
        assert np.allclose(blk.T @ blk, (2 * l + 1) / (4 * math.pi) * P[l], atol=1e-12)
        idx += 2 * l + 1


def test_sht_convolution_equals_real_space_sum_of_its_kernel():
    nside, lmax = 4, 10
    k_ell = gaussian_beam(600.0, lmax)
    x = white_noise_maps(nside, 1, 5)[0].astype(np.float64)
    y_sht = O.sht_convolve(nside, x, k_ell, lmax)
    y_rs = O.conv_function_brute(nside, lambda g: O.legendre_series(k_ell, 0, lmax, g), math.pi, x)
    assert np.allclose(y_sht, y_rs, atol=1e-12 * np.abs(y_rs).max())


# ----------------------------------------------------------------- gradient

@pytest.mark.parametrize("nside", [4, 8, 16])
def test_ring_transform_equals_the_pixel_sum_transform(nside):
    """The ring-by-ring transform (ring FFTs times lambda_lm, for larger maps) is the
    brute-force pixel-sum transform of real_ylm (itself pinned by the addition theorem)
    rewritten: same a_lm (as spectra), same synthesis, and the power spectrum of a map
    made of one real harmonic is that harmonic's l alone (up to the pixel quadrature)."""
    lmax = 2 * nside
    x = white_noise_maps(nside, 1, 300 + nside)[0].astype(np.float64)
    a = O.sht_analysis_rings(nside, x, lmax)
    th, ph = O.pixel_angles(nside)
    Y = O.real_ylm(lmax, th, ph)
    ar = (4 * math.pi / O.npix(nside)) * (Y @ x)
    C_brute = np.array([np.sum(ar[l * l:(l + 1) ** 2] ** 2) / (2 * l + 1) for l in range(lmax + 1)])
    assert np.allclose(O.power_spectrum(a, lmax), C_brute, rtol=1e-12, atol=1e-14 * C_brute.max())
    kl = np.linspace(1.0, 0.1, lmax + 1)
    kr = np.concatenate([np.full(2 * l + 1, kl[l]) for l in range(lmax + 1)])
    y_brute = Y.T @ (kr * ar)
    y_ring = O.sht_synthesis_rings(nside, a, lmax, kl)
    assert np.abs(y_ring - y_brute).max() <= 1e-12 * np.abs(y_brute).max()
    # a single harmonic l = nside / 2: the spectrum peaks there
    l0 = nside // 2
    a1 = O.sht_analysis_rings(nside, Y[l0 * l0 + l0], lmax)
    C1 = O.power_spectrum(a1, lmax)
    assert np.argmax(C1) == l0 and C1[l0] > 0.9 / (2 * l0 + 1)


def test_table_gradient_equals_central_differences():
    nside, tc, nt = 8, 0.35, 24
    rng = np.random.default_rng(11)
    for layout in (0, 1):
        V = rng.standard_normal(nt)
        x = rng.standard_normal(O.npix(nside))
        t = rng.standard_normal(O.npix(nside))

        def loss(Vv):
            return np.sum((O.conv_window(nside, Vv, tc, layout, x) - t) ** 2)

        y = O.conv_window(nside, V, tc, layout, x)
        g = O.grad_table(nside, nt, tc, layout, x, 2 * (y - t))
        h = 1e-3
        for n in range(nt):
            e = np.zeros(nt); e[n] = h
            fd = (loss(V + e) - loss(V - e)) / (2 * h)   # quadratic: exact up to rounding
            assert fd == pytest.approx(g[n], rel=1e-8, abs=1e-9 * np.abs(g).max())


# ---------------------------------------------------------------- least-squares split

def _trunc_on_basis(k_ell, lcut, lfit, tc, n_basis):
    # the high-pass-and-truncate kernel (reading of Sec. 3) sampled on the basis nodes
    th = np.linspace(0.0, tc, n_basis)
    v = O.legendre_series(k_ell, lcut + 1, lfit, th) * O.taper(th, tc, 0.9)
    v[-1] = 0.0
    return v


def test_fit_recovers_a_planted_response():
    # K_l made from a kernel of the basis: the fit reproduces it above l_cut
    nb, tc, lcut, lfit = 33, 0.3, 10, 120
    M = O.hat_response_matrix(nb, tc, 0, lfit)
    c_true = 10.0 * np.sin(np.linspace(0.0, 3.0, nb - 1))
    kl = M @ c_true
    V, sig = O.fit_real_kernel(kl, lcut, lfit, tc, nb, nb)
    assert sig < 1e-6
    R = O.kernel_response(V, tc, 0, lfit)
    assert np.max(np.abs(R[lcut + 1:] - kl[lcut + 1:])) < 1e-5 * np.max(np.abs(kl))


def test_fit_reported_sigma_matches_independent_response():
    # sigma from the fit's own response matrix equals the one recomputed from the
    # output table by kernel_response (a separate quadrature over the fine nodes)
    tc, lcut, lfit, nb = 180.0 * ARCMIN, 96, 384, 129
    kl = gaussian_beam(60.0, lfit)
    V, sig = O.fit_real_kernel(kl, lcut, lfit, tc, nb, 8 * (nb - 1) + 1)
    R = O.kernel_response(V, tc, 0, lfit)
    ell = np.arange(lfit + 1)
    num = np.sum((2 * ell[lcut + 1:] + 1) * (R[lcut + 1:] - kl[lcut + 1:]) ** 2)
    den = np.sum((2 * ell + 1) * kl ** 2)
    assert abs(math.sqrt(num / den) - sig) <= 1e-6 * sig + 1e-12


@pytest.mark.parametrize("fwhm,tcf,lcut,lfit", [(60.0, 3.0, 96, 384), (7.1, 2.8, 1024, 4096)])
def test_fit_beats_truncation(fwhm, tcf, lcut, lfit):
    # the least-squares kernel minimises Eq. 2's residual over the basis, so it is
    # no worse than the truncated high-pass kernel on the same nodes
    tc, nb = tcf * fwhm * ARCMIN, 129
    kl = gaussian_beam(fwhm, lfit)
    V, sig = O.fit_real_kernel(kl, lcut, lfit, tc, nb, nb)
    vt = _trunc_on_basis(kl, lcut, lfit, tc, nb)
    Rt = O.hat_response_matrix(nb, tc, 0, lfit) @ vt[:-1]
    ell = np.arange(lfit + 1)
    num = np.sum((2 * ell[lcut + 1:] + 1) * (Rt[lcut + 1:] - kl[lcut + 1:]) ** 2)
    sig_t = math.sqrt(num / np.sum((2 * ell + 1) * kl ** 2))
    assert sig <= sig_t
