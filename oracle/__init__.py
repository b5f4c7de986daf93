"""FP64 CPU oracle for the real-space spherical convolution (test infrastructure).

TEST INFRASTRUCTURE ONLY: the product never imports this package.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use
it.  It shares no code with the CUDA path.

Contents, each following a passage of the paper (Sutter, Wandelt & Elsner,
"Accelerating convolutions on the sphere with hybrid GPU/CPU kernel
splitting"):

* pair sums (C, ``skoracle.c``): the real-space convolution of a HEALPix RING
  map with a tabulated radial kernel, brute force and windowed -- Sec. 2, Eq. 1
  (the real-space part K^_theta), Sec. 3 (tabulated, linearly interpolated
  kernel with optional node bias);
* ``legendre_series``: K(theta) = sum_l (2l+1)/(4 pi) K_l P_l(cos theta), the
  Legendre transform operator P_{l theta} of Eq. 1;
* ``tabulate_real_kernel``: the real-space part of the split of a kernel K_l
  (Eq. 1): the l > l_cut high-pass series, truncated at theta_cut with a taper,
  sampled at the nodes;
* ``kernel_response``: R_l = 2 pi int_0^theta_cut K_lin(theta) P_l(cos theta)
  sin theta dtheta, i.e. P_{l theta} K^_theta of Eq. 1, and ``harmonic_part``:
  K^_l = K_l - R_l for l <= l_cut (so K~_l = K^_l + R_l reproduces K_l there);
* ``real_ylm`` / ``sht_convolve``: a plain spherical-harmonic transform for the
  harmonic part (the role the paper gives to the CPU SHT, Sec. 2), brute force;
  ``sht_analysis_rings`` / ``sht_synthesis_rings`` / ``power_spectrum``: the same
  pixel-sum transform written ring by ring (for larger maps), and the power spectrum
  the paper extracts from convolved maps (Sec. 3, the spectra of its error figures);
* ``relative_error_estimate``: the fractional rms estimate of Eq. 2;
* ``hat_response_matrix`` / ``fit_real_kernel``: the real-space part as a
  least-squares fit (Sec. 3: K^_theta is fit so that its harmonic transform
  matches K_l above l_cut), a piecewise-linear kernel on [0, theta_cut] that
  vanishes at theta_cut, by ``numpy.linalg.lstsq`` on the plain objective;
* gradients: the table gradient in C and a finite-difference helper;
* ``resample_nearest``: a map re-oriented by a rotation (Sec. 4: a partial-sky
  field moved onto the polar cap), nearest pixel centre by brute force.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "skoracle.c")
_LIB = os.path.join(_HERE, "libskoracle.so")
_lock = threading.Lock()
_lib = None

LAYOUT_UNIFORM = 0
LAYOUT_BIASED = 1


def build(force: bool = False) -> str:
    """Compile skoracle.c into oracle/libskoracle.so with gcc (OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i64, dbl, cint = ctypes.c_int64, ctypes.c_double, ctypes.c_int
            P = ctypes.c_void_p
            L.or_npix.restype = i64; L.or_npix.argtypes = [i64]
            L.or_ring_info.argtypes = [i64, i64, P, P, P, P, P]
            L.or_pix2ang.argtypes = [i64, i64, P, P]
            L.or_pix2vec.argtypes = [i64, i64, P]
            L.or_all_vecs.argtypes = [i64, P]
            L.or_pix2ring.argtypes = [i64, i64, P, P]
            L.or_node_theta.restype = dbl; L.or_node_theta.argtypes = [i64, i64, dbl, cint]
            L.or_node_coord.restype = dbl; L.or_node_coord.argtypes = [dbl, i64, dbl, cint]
            L.or_klin.restype = dbl; L.or_klin.argtypes = [P, i64, dbl, cint, dbl]
            L.or_conv_brute.argtypes = [i64, P, i64, dbl, cint, P, P, cint]
            L.or_conv_window.argtypes = [i64, P, i64, dbl, cint, P, P, i64, P, cint]
            L.or_count_pairs.restype = i64
            L.or_count_pairs.argtypes = [i64, dbl, P, i64, cint]
            L.or_grad_table.argtypes = [i64, i64, dbl, cint, P, P, P, cint]
            L.or_num_threads.restype = cint
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# HEALPix geometry (Gorski et al. 2005; the paper's pixelisation, Sec. 2)
# --------------------------------------------------------------------------

def npix(nside: int) -> int:
    return int(lib().or_npix(nside))


def ring_info(nside: int, r: int):
    """(n_pixels, first_pixel, shift s, z, sin theta) of ring r (1-based)."""
    n = ctypes.c_int64(); st = ctypes.c_int64(); s = ctypes.c_int()
    z = ctypes.c_double(); sn = ctypes.c_double()
    lib().or_ring_info(nside, r, ctypes.byref(n), ctypes.byref(st), ctypes.byref(s),
                       ctypes.byref(z), ctypes.byref(sn))
    return n.value, st.value, s.value, z.value, sn.value


def pix2ang(nside: int, p: int):
    th = ctypes.c_double(); ph = ctypes.c_double()
    lib().or_pix2ang(nside, p, ctypes.byref(th), ctypes.byref(ph))
    return th.value, ph.value


def pix2ring(nside: int, p: int):
    r = ctypes.c_int64(); j = ctypes.c_int64()
    lib().or_pix2ring(nside, p, ctypes.byref(r), ctypes.byref(j))
    return r.value, j.value


def all_vecs(nside: int) -> np.ndarray:
    v = np.empty((npix(nside), 3), dtype=np.float64)
    lib().or_all_vecs(nside, _p(v))
    return v


# --------------------------------------------------------------------------
# Tabulated kernel nodes (Sec. 3)
# --------------------------------------------------------------------------

def node_thetas(nt: int, theta_cut: float, layout: int = LAYOUT_UNIFORM) -> np.ndarray:
    L = lib()
    return np.array([L.or_node_theta(k, nt, theta_cut, layout) for k in range(nt)])


def klin(V: np.ndarray, theta_cut: float, layout: int, theta) -> np.ndarray:
    """K_lin at the given angles (0 beyond theta_cut)."""
    V = _f64(V)
    L = lib()
    th = np.atleast_1d(np.asarray(theta, dtype=np.float64))
    return np.array([L.or_klin(_p(V), len(V), theta_cut, layout, float(t)) for t in th])


# --------------------------------------------------------------------------
# Legendre transform operator P_{l theta} (Eq. 1) and the split
# --------------------------------------------------------------------------

def legendre_P(lmax: int, x: np.ndarray) -> np.ndarray:
    """P_l(x) for l = 0..lmax by the Bonnet recurrence, shape [lmax+1, len(x)]."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty((lmax + 1,) + x.shape)
    out[0] = 1.0
    if lmax >= 1:
        out[1] = x
    for l in range(1, lmax):
        out[l + 1] = ((2 * l + 1) * x * out[l] - l * out[l - 1]) / (l + 1)
    return out


def legendre_series(coef: np.ndarray, lmin: int, lmax: int, theta) -> np.ndarray:
    """sum_{l=lmin}^{lmax} (2l+1)/(4 pi) coef_l P_l(cos theta), Bonnet recurrence."""
    theta = np.asarray(theta, dtype=np.float64)
    x = np.cos(theta)
    p0 = np.ones_like(x)
    p1 = x.copy()
    acc = np.zeros_like(x)
    for l in range(0, lmax + 1):
        if l == 0:
            pl = p0
        elif l == 1:
            pl = p1
        else:
            p2 = ((2 * l - 1) * x * p1 - (l - 1) * p0) / l
            p0, p1 = p1, p2
            pl = p2
        if l >= lmin:
            acc += (2 * l + 1) / (4.0 * math.pi) * coef[l] * pl
    return acc


def taper(theta, theta_cut: float, start: float = 0.9) -> np.ndarray:
    """1 below start*theta_cut, then a raised cosine down to exactly 0 at theta_cut."""
    theta = np.asarray(theta, dtype=np.float64)
    if start >= 1.0:
        return np.ones_like(theta)
    t0 = start * theta_cut
    w = np.ones_like(theta)
    m = theta > t0
    w[m] = 0.5 * (1.0 + np.cos(math.pi * (theta[m] - t0) / (theta_cut - t0)))
    w[theta >= theta_cut] = 0.0
    return w


def tabulate_real_kernel(k_ell: np.ndarray, lcut: int, lmax: int, theta_cut: float,
                         nt: int, layout: int = LAYOUT_UNIFORM,
                         taper_start: float = 0.9) -> np.ndarray:
    """Node values of the real-space part K^_theta (Eq. 1): the l > l_cut part of
    the Legendre series of K_l, truncated at theta_cut with a taper, FP64."""
    th = node_thetas(nt, theta_cut, layout)
    return legendre_series(k_ell, lcut + 1, lmax, th) * taper(th, theta_cut, taper_start)


def kernel_response(V: np.ndarray, theta_cut: float, layout: int, lmax: int,
                    npts: int = 8) -> np.ndarray:
    """R_l = 2 pi int_0^theta_cut K_lin(theta) P_l(cos theta) sin(theta) dtheta,
    l = 0..lmax: Gauss-Legendre with npts points on every node interval (K_lin is
    linear there)."""
    V = _f64(V)
    nt = len(V)
    th = node_thetas(nt, theta_cut, layout)
    g, w = np.polynomial.legendre.leggauss(npts)
    a, b = th[:-1, None], th[1:, None]
    tq = 0.5 * (b - a) * g[None, :] + 0.5 * (a + b)            # [nt-1, npts]
    wq = 0.5 * (b - a) * w[None, :]
    f = (tq - a) / (b - a)
    Kq = V[:-1, None] + f * (V[1:, None] - V[:-1, None])
    integrand_w = (wq * Kq * np.sin(tq)).ravel()
    x = np.cos(tq).ravel()
    R = np.empty(lmax + 1)
    p0 = np.ones_like(x); p1 = x.copy()
    for l in range(lmax + 1):
        if l == 0:
            pl = p0
        elif l == 1:
            pl = p1
        else:
            p2 = ((2 * l - 1) * x * p1 - (l - 1) * p0) / l
            p0, p1 = p1, p2
            pl = p2
        R[l] = 2.0 * math.pi * np.dot(integrand_w, pl)
    return R


def harmonic_part(k_ell: np.ndarray, R: np.ndarray, lcut: int) -> np.ndarray:
    """K^_l = K_l - R_l for l <= l_cut, 0 above (the truncated l-space part)."""
    kh = np.zeros_like(k_ell)
    kh[: lcut + 1] = k_ell[: lcut + 1] - R[: lcut + 1]
    return kh


def hat_response_matrix(n_basis: int, theta_cut: float, lmin: int, lmax: int, npts: int = 8) -> np.ndarray:
    """M[l - lmin, k] = 2 pi int hat_k(theta) P_l(cos theta) sin theta dtheta for
    l = lmin..lmax and the hat functions of the uniform nodes theta_k =
    k theta_cut / (n_basis - 1), k = 0..n_basis - 2 (the node at theta_cut is
    held at 0).  Gauss-Legendre with npts points on every node interval."""
    th = np.linspace(0.0, theta_cut, n_basis)
    g, w = np.polynomial.legendre.leggauss(npts)
    a, b = th[:-1, None], th[1:, None]
    tq = (0.5 * (b - a) * g[None, :] + 0.5 * (a + b)).ravel()          # [(n-1) npts]
    wq = np.broadcast_to(0.5 * (b - a) * w[None, :], (n_basis - 1, npts)).ravel()
    f = ((tq.reshape(n_basis - 1, npts) - a) / (b - a)).ravel()
    ivl = np.repeat(np.arange(n_basis - 1), npts)
    # hat_k on interval i: 1 - f for k = i, f for k = i + 1
    H = np.zeros((len(tq), n_basis))
    H[np.arange(len(tq)), ivl] = 1.0 - f
    H[np.arange(len(tq)), ivl + 1] = f
    P = legendre_P(lmax, np.cos(tq))[lmin:]                              # [l, q]
    M = 2.0 * math.pi * (P * (wq * np.sin(tq))[None, :]) @ H
    return M[:, : n_basis - 1]


def fit_real_kernel(k_ell: np.ndarray, lcut: int, lfit: int, theta_cut: float, n_basis: int,
                    nt_out: int, low_weight: float = 1e-3, reg: float = 1e-9):
    """Node values (nt_out uniform nodes) of the least-squares real-space part:
    minimise sum_{l=0}^{lfit} w_l (2l+1) (R_l(c) - K_l)^2 + lam |c|^2 over the
    hat-basis coefficients c, with w_l = 1 above l_cut (where the real-space part
    alone carries K_l) and w_l = low_weight at and below l_cut (there K^_l = K_l -
    R_l absorbs any mismatch; the small weight keeps the two halves from
    carrying large parts that cancel), lam = reg * trace(A^T A) / n.  The
    piecewise-linear kernel is sampled at the output nodes ((nt_out - 1) a
    multiple of (n_basis - 1), so the output table represents it exactly).
    Returns (V, sigma_rms): sigma_rms^2 = sum_{l>lcut}^{lfit} (2l+1)(R_l - K_l)^2 /
    sum_{l<=lfit} (2l+1) K_l^2 (Eq. 2 without alpha)."""
    k_ell = _f64(k_ell)
    M = hat_response_matrix(n_basis, theta_cut, 0, lfit)
    ell = np.arange(0, lfit + 1, dtype=np.float64)
    wl = np.where(ell > lcut, 1.0, low_weight)
    sw = np.sqrt(wl * (2.0 * ell + 1.0))
    A = M * sw[:, None]
    y = k_ell[: lfit + 1] * sw
    n = M.shape[1]
    lam = reg * float(np.sum(A * A)) / n
    Aa = np.vstack([A, math.sqrt(lam) * np.eye(n)])
    ya = np.concatenate([y, np.zeros(n)])
    c = np.linalg.lstsq(Aa, ya, rcond=None)[0]
    coarse = np.concatenate([c, [0.0]])
    th_out = np.linspace(0.0, theta_cut, nt_out)
    V = np.interp(th_out, np.linspace(0.0, theta_cut, n_basis), coarse)
    res = (M @ c - k_ell[: lfit + 1])[lcut + 1:]
    hi = ell[lcut + 1:]
    sig = math.sqrt(float(np.sum((2 * hi + 1) * res ** 2)) /
                    float(np.sum((2 * ell + 1) * k_ell[: lfit + 1] ** 2)))
    return V, sig


def relative_error_estimate(k_ell: np.ndarray, k_approx: np.ndarray, alpha: float = 5.0) -> float:
    """Eq. 2: sigma^2 = alpha^2 sigma_rms^2 / ((1/4pi) sum (2l+1) K_l^2), with
    sigma_rms^2 = (1/4pi) sum (2l+1) (K~_l - K_l)^2 (white-noise map rms)."""
    ell = np.arange(len(k_ell))
    srms2 = np.sum((2 * ell + 1) * (k_approx - k_ell) ** 2) / (4 * math.pi)
    den = np.sum((2 * ell + 1) * k_ell ** 2) / (4 * math.pi)
    return float(alpha * math.sqrt(srms2 / den))


# --------------------------------------------------------------------------
# Pair sums (C)
# --------------------------------------------------------------------------

def conv_brute(nside: int, V, theta_cut: float, layout: int, x, nthreads: int = 0) -> np.ndarray:
    V = _f64(V); x = _f64(x)
    y = np.empty(npix(nside))
    lib().or_conv_brute(nside, _p(V), len(V), theta_cut, layout, _p(x), _p(y), nthreads)
    return y


def conv_window(nside: int, V, theta_cut: float, layout: int, x, outs=None,
                nthreads: int = 0) -> np.ndarray:
    """Windowed direct sum; all outputs, or only pixels `outs` (returns [len(outs)])."""
    V = _f64(V); x = _f64(x)
    if outs is None:
        y = np.empty(npix(nside))
        lib().or_conv_window(nside, _p(V), len(V), theta_cut, layout, _p(x), None, 0, _p(y), nthreads)
    else:
        o = np.ascontiguousarray(outs, dtype=np.int64)
        y = np.empty(len(o))
        lib().or_conv_window(nside, _p(V), len(V), theta_cut, layout, _p(x), _p(o), len(o),
                             _p(y), nthreads)
    return y


def count_pairs(nside: int, theta_cut: float, outs=None, nthreads: int = 0) -> int:
    if outs is None:
        return int(lib().or_count_pairs(nside, theta_cut, None, 0, nthreads))
    o = np.ascontiguousarray(outs, dtype=np.int64)
    return int(lib().or_count_pairs(nside, theta_cut, _p(o), len(o), nthreads))


def grad_table(nside: int, nt: int, theta_cut: float, layout: int, x, gy,
               nthreads: int = 0) -> np.ndarray:
    """dL/dV_n = dOmega sum_o gy_o sum_{i in cut} x_i dK_lin/dV_n(gamma_oi)."""
    x = _f64(x); gy = _f64(gy)
    gV = np.empty(nt)
    lib().or_grad_table(nside, nt, theta_cut, layout, _p(x), _p(gy), _p(gV), nthreads)
    return gV


def num_threads() -> int:
    return int(lib().or_num_threads())


# --------------------------------------------------------------------------
# Plain spherical-harmonic transform for the harmonic part (small Nside only)
# --------------------------------------------------------------------------

def real_ylm(lmax: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonics, rows (l, m) for m = -l..l in order,
    columns = points.  Normalised associated Legendre functions by the standard
    three-term recurrence in l at fixed m."""
    x = np.cos(theta); sx = np.sin(theta)
    npt = len(x)
    rows = []
    # Pbar_mm, then upward in l
    pmm = np.full(npt, math.sqrt(1.0 / (4.0 * math.pi)))
    plm = {}
    for m in range(lmax + 1):
        if m > 0:
            pmm = -math.sqrt((2 * m + 1) / (2.0 * m)) * sx * pmm
        plm[(m, m)] = pmm.copy()
        if m + 1 <= lmax:
            plm[(m + 1, m)] = math.sqrt(2 * m + 3) * x * pmm
        for l in range(m + 2, lmax + 1):
            a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            plm[(l, m)] = a * (x * plm[(l - 1, m)] - b * plm[(l - 2, m)])
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            if m == 0:
                rows.append(plm[(l, 0)])
            elif m > 0:
                rows.append(math.sqrt(2.0) * plm[(l, m)] * np.cos(m * phi))
            else:
                rows.append(math.sqrt(2.0) * plm[(l, -m)] * np.sin(-m * phi))
    return np.array(rows)


def pixel_angles(nside: int):
    v = all_vecs(nside)
    theta = np.arctan2(np.hypot(v[:, 0], v[:, 1]), v[:, 2])
    phi = np.mod(np.arctan2(v[:, 1], v[:, 0]), 2 * math.pi)
    return theta, phi


def sht_convolve(nside: int, x: np.ndarray, k_ell: np.ndarray, lmax: int) -> np.ndarray:
    """Harmonic-space convolution by a plain pixel-sum SHT:
    a_lm = dOmega sum_p x_p Y_lm(p);  y_p = sum_lm K_l a_lm Y_lm(p)."""
    th, ph = pixel_angles(nside)
    Y = real_ylm(lmax, th, ph)
    dOmega = 4.0 * math.pi / npix(nside)
    a = dOmega * (Y @ _f64(x))
    kl = np.concatenate([np.full(2 * l + 1, k_ell[l]) for l in range(lmax + 1)])
    return Y.T @ (kl * a)


def _ring_geometry(nside: int):
    """Per ring (0-based): pixel count, first pixel, shift, colatitude (from ring_info)."""
    nr = 4 * nside - 1
    rows = [ring_info(nside, r) for r in range(1, nr + 1)]
    n = np.array([q[0] for q in rows], np.int64)
    st = np.array([q[1] for q in rows], np.int64)
    sh = np.array([q[2] for q in rows], np.int64)
    th = np.arctan2(np.array([q[4] for q in rows]), np.array([q[3] for q in rows]))
    return n, st, sh, th


def _lambda_lm(lmax: int, theta: np.ndarray):
    """Orthonormal associated Legendre functions lambda_lm(theta) (Y_lm = lambda_lm e^{i m phi}),
    l = 0..lmax, m = 0..l, by the same three-term recurrence in l at fixed m as real_ylm;
    returns a dict m -> array [l - m, len(theta)]."""
    x = np.cos(theta); sx = np.sin(theta)
    out = {}
    pmm = np.full(len(x), math.sqrt(1.0 / (4.0 * math.pi)))
    for m in range(lmax + 1):
        if m > 0:
            pmm = -math.sqrt((2 * m + 1) / (2.0 * m)) * sx * pmm
        rows = np.empty((lmax - m + 1, len(x)))
        rows[0] = pmm
        if m + 1 <= lmax:
            rows[1] = math.sqrt(2 * m + 3) * x * pmm
        for l in range(m + 2, lmax + 1):
            a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            rows[l - m] = a * (x * rows[l - 1 - m] - b * rows[l - 2 - m])
        out[m] = rows
    return out


def sht_analysis_rings(nside: int, x: np.ndarray, lmax: int) -> dict:
    """a_lm = dOmega sum_p x_p Y*_lm(p) for m = 0..l (complex; a_{l,-m} = (-1)^m conj a_lm
    for a real map), the pixel sum of the plain transform written ring by ring: with
    Y_lm = lambda_lm(theta) e^{i m phi} and phi_j = pi (2j + s)/n on a ring,
    a_lm = dOmega sum_r lambda_lm(theta_r) F_r(m), F_r(m) = sum_j x_j e^{-i m phi_j} =
    e^{-i pi m s / n} X_r(m mod n) with X_r the ring's DFT (numpy FFT).  FP64.
    Returns a dict m -> complex array [l - m]."""
    n, st, sh, th = _ring_geometry(nside)
    x = np.asarray(x, np.float64)
    dOmega = 4.0 * math.pi / npix(nside)
    ms = np.arange(lmax + 1)
    F = np.empty((len(n), lmax + 1), np.complex128)
    for r in range(len(n)):
        X = np.fft.fft(x[st[r]: st[r] + n[r]])
        F[r] = np.exp(-1j * math.pi * ms * sh[r] / n[r]) * X[ms % n[r]]
    lam = _lambda_lm(lmax, th)
    return {m: dOmega * (lam[m] @ F[:, m]) for m in range(lmax + 1)}


def sht_synthesis_rings(nside: int, alm: dict, lmax: int, k_ell: np.ndarray = None) -> np.ndarray:
    """y_p = sum_{l <= lmax} sum_m k_l a_lm Y_lm(p) for a real map (k_l = 1 if None):
    y = Re G_r(0) + 2 Re sum_{m >= 1} G_r(m) e^{i m phi_j}, G_r(m) = sum_l k_l a_lm
    lambda_lm(theta_r).  On a ring of n pixels e^{i m phi_j} = e^{i pi m s/n} e^{2 pi i j m/n},
    so the sum over m is an inverse DFT of the terms folded onto m mod n (numpy FFT).  FP64."""
    n, st, sh, th = _ring_geometry(nside)
    lam = _lambda_lm(lmax, th)
    kl = np.ones(lmax + 1) if k_ell is None else np.asarray(k_ell, np.float64)
    G = np.stack([(kl[m:lmax + 1, None] * lam[m] * alm[m][:, None]).sum(axis=0) for m in range(lmax + 1)],
                 axis=1)                                       # [rings, m]
    y = np.empty(npix(nside))
    ms = np.arange(lmax + 1)
    wm = np.where(ms == 0, 1.0, 2.0)
    for r in range(len(n)):
        H = np.zeros(n[r], np.complex128)
        np.add.at(H, ms % n[r], wm * G[r] * np.exp(1j * math.pi * ms * sh[r] / n[r]))
        y[st[r]: st[r] + n[r]] = (n[r] * np.fft.ifft(H)).real
    return y


def power_spectrum(alm: dict, lmax: int) -> np.ndarray:
    """C_l = (|a_l0|^2 + 2 sum_{m >= 1} |a_lm|^2) / (2l + 1) of a real map's a_lm (m >= 0)."""
    C = np.zeros(lmax + 1)
    for m in range(lmax + 1):
        C[m:] += (1.0 if m == 0 else 2.0) * np.abs(alm[m]) ** 2
    return C / (2.0 * np.arange(lmax + 1) + 1.0)


def conv_function_brute(nside: int, kernel_fn, theta_cut: float, x: np.ndarray) -> np.ndarray:
    """All-pairs sum with an exactly evaluated radial function (tiny Nside only):
    y_o = dOmega sum_{gamma <= theta_cut} kernel_fn(gamma) x_i."""
    v = all_vecs(nside)
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=-1)
    g = 2.0 * np.arcsin(np.minimum(1.0, 0.5 * d))
    K = np.where(g <= theta_cut, kernel_fn(g), 0.0)
    return (4.0 * math.pi / npix(nside)) * (K @ _f64(x))


# --------------------------------------------------------------------------
# Re-orientation onto the polar cap (Sec. 4)
# --------------------------------------------------------------------------

def ring_starts(nside: int) -> np.ndarray:
    """First pixel of each ring (0-based rings), and npix at the end."""
    nr = 4 * nside - 1
    st = [ring_info(nside, r)[1] for r in range(1, nr + 1)]
    return np.array(st + [npix(nside)], dtype=np.int64)


def resample_nearest(nside: int, x, M, ring_lo: int, ring_hi: int, src_ring_hi: int = None,
                     return_index: bool = False):
    """Nearest-centre resampling under a rotation, by brute force: for every pixel p of
    rings [ring_lo, ring_hi) (0-based), i = the pixel whose centre has the largest dot
    product with M v_p (the nearest centre; the first index on ties), and
    out[p] = x[i] if ring(i) < src_ring_hi else 0; other pixels 0.  x: [npix] or
    [batch, npix]."""
    x = np.asarray(x, dtype=np.float64)
    one = x.ndim == 1
    X = x[None, :] if one else x
    v = all_vecs(nside)
    st = ring_starts(nside)
    nr = 4 * nside - 1
    src = nr if src_ring_hi is None else int(src_ring_hi)
    p0, p1 = int(st[ring_lo]), int(st[ring_hi])
    W = v[p0:p1] @ np.asarray(M, dtype=np.float64).T          # rows: M v_p
    idx = np.empty(p1 - p0, dtype=np.int64)
    rows = max(1, (1 << 23) // len(v))                            # ~64 MB of dot products at a time
    for a in range(0, p1 - p0, rows):
        idx[a:a + rows] = np.argmax(W[a:a + rows] @ v.T, axis=1)
    ring = np.searchsorted(st, idx, side="right") - 1
    out = np.zeros_like(X)
    out[:, p0:p1] = np.where(ring < src, X[:, idx], 0.0)
    out = out[0] if one else out
    return (out, idx) if return_index else out
