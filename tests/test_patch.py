"""Re-orientation of partial-sky fields onto the polar cap (Sec. 4).

CPU: the oracle's nearest-centre resampling pinned to exact permutations of the
pixelisation (identity, the quarter turn about the pole, the half turn that swaps the
hemispheres), its source-ring limit, the rotation helper, and the claim the device
search rests on (the nearest centre lies within two rings of the ring nearest in z),
checked against brute force.  GPU: sk_resample against the oracle (index maps equal;
a pixel may differ only where two centres are equally near to FP64 rounding) and the
whole field convolution (rotate, sum the cap rings, rotate back) against the oracle's
composition of the same three steps, rms <= 1e-6.
"""
import math

import numpy as np
import pytest

import oracle as O
from inputs import ARCMIN, gaussian_beam, white_noise_maps


def ring_tables(nside):
    st = O.ring_starts(nside)
    n = np.diff(st)
    s = np.array([O.ring_info(nside, r)[2] for r in range(1, 4 * nside)])
    return st, n, s


def rot_x_pi():
    return np.diag([1.0, -1.0, -1.0])


def rot_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def random_rotation(seed):
    q = np.random.default_rng(seed).standard_normal(4)
    a, b, c, d = q / np.linalg.norm(q)
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


# ---------------------------------------------------------------- oracle pins (CPU)

@pytest.mark.parametrize("nside", [1, 2, 8])
def test_oracle_resample_exact_permutations(nside):
    npx = O.npix(nside)
    nr = 4 * nside - 1
    x = np.arange(npx, dtype=np.float64)
    st, n, s = ring_tables(nside)
    assert np.array_equal(O.resample_nearest(nside, x, np.eye(3), 0, nr), x)
    # quarter turn about the pole: pixel j of every ring -> j + n/4
    q = np.empty(npx)
    # half turn about the x axis: ring r -> its mirror, phi -> -phi (pixel j -> n - j - s)
    h = np.empty(npx)
    for r in range(nr):
        for j in range(n[r]):
            q[st[r] + j] = st[r] + (j + n[r] // 4) % n[r]
            h[st[r] + j] = st[nr - 1 - r] + (n[r] - j - s[r]) % n[r]
    assert np.array_equal(O.resample_nearest(nside, x, rot_z(math.pi / 2), 0, nr), q)
    assert np.array_equal(O.resample_nearest(nside, x, rot_x_pi(), 0, nr), h)


def test_oracle_resample_ring_range_and_source_limit():
    nside = 8
    nr = 4 * nside - 1
    st, n, s = ring_tables(nside)
    x = np.arange(O.npix(nside), dtype=np.float64) + 1.0
    y = O.resample_nearest(nside, np.stack([x, -x]), np.eye(3), 3, 20, src_ring_hi=11)
    assert np.all(y[:, : st[3]] == 0) and np.all(y[:, st[20]:] == 0)
    assert np.array_equal(y[0, st[3]: st[11]], x[st[3]: st[11]])
    assert np.all(y[:, st[11]: st[20]] == 0)
    assert np.array_equal(y[1], -y[0])


def test_rotation_to_pole():
    import paper_1211_3556_b300 as sk
    for th, ph in ((0.3, 1.1), (2.0, 5.0), (math.pi / 2, 0.0)):
        M = sk.rotation_to_pole(th, ph)
        assert np.allclose(M @ M.T, np.eye(3), atol=1e-15)
        assert np.linalg.det(M) == pytest.approx(1.0, abs=1e-14)
        v = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        assert np.allclose(M @ np.array([0.0, 0.0, 1.0]), v, atol=1e-15)


@pytest.mark.parametrize("nside", [1, 2, 4, 16])
def test_nearest_centre_within_two_rings_of_the_z_estimate(nside):
    # the device search looks at the five rings around the ring whose z is nearest
    # (continuous estimate) and, on each, the pixel nearest in phi; brute force agrees
    v = O.all_vecs(nside)
    st, n, s = ring_tables(nside)
    nr = 4 * nside - 1
    rng = np.random.default_rng(nside)
    w = rng.standard_normal((3000, 3))
    w /= np.linalg.norm(w, axis=1)[:, None]
    brute = np.argmax(w @ v.T, axis=1)
    z = np.array([O.ring_info(nside, r)[3] for r in range(1, nr + 1)])
    N = float(nside)
    for k in range(len(w)):
        zw = w[k, 2]
        if zw > 2 / 3:
            rc = N * math.sqrt(3 * (1 - zw))
        elif zw < -2 / 3:
            rc = 4 * N - N * math.sqrt(3 * (1 + zw))
        else:
            rc = N * (2 - 1.5 * zw)
        r0 = int(round(rc))
        cand = []
        for r in range(max(1, r0 - 2), min(nr, r0 + 2) + 1):
            ph = math.atan2(w[k, 1], w[k, 0]) % (2 * math.pi)
            j = int(round(ph * n[r - 1] / (2 * math.pi) - 0.5 * s[r - 1])) % n[r - 1]
            cand.append(st[r - 1] + j)
        best = max(cand, key=lambda p: (float(v[p] @ w[k]), -p))
        assert v[best] @ w[k] >= v[brute[k]] @ w[k] - 1e-15


# ---------------------------------------------------------------- device (GPU)

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


def check_index_maps(nside, got, want, M, p0):
    """Equal index maps (outputs from pixel p0 on), except where the two centres are equally
    near M v_p to FP64 rounding (1e-14 in the dot product)."""
    diff = np.nonzero(got != want)[0]
    assert len(diff) <= max(2, len(got) // 100000)
    if len(diff):
        v = O.all_vecs(nside)
        w = v[p0 + diff] @ M.T
        dg = np.einsum("ij,ij->i", w, v[got[diff]])
        dw = np.einsum("ij,ij->i", w, v[want[diff]])
        assert np.all(np.abs(dg - dw) <= 1e-14)


@pytest.mark.gpu
@pytest.mark.parametrize("nside,seed,lo,hi,src", [(16, 1, 0, 63, 40), (64, 2, 0, 255, 100), (256, 3, 300, 304, 1023),
                                                  (8, 4, 0, 31, 31), (256, 5, 0, 12, 6), (128, 6, 250, 300, 280)])
def test_resample_matches_oracle(sk, nside, seed, lo, hi, src):
    import torch
    g = sk.Geometry(sk._ctx, nside)
    M = random_rotation(seed)
    npx = g.npix
    st = O.ring_starts(nside)
    p0, p1 = int(st[lo]), int(st[hi])
    # pixel index + 1 as the value (exact in FP32 below 2^24): the output is the index map
    x = np.arange(npx, dtype=np.float32) + 1.0
    xt = torch.from_numpy(np.stack([x, -x])).cuda()
    y_all = sk.resample(g, xt, M, lo, hi).cpu().numpy()
    y_lim = sk.resample(g, xt, M, lo, hi, src_ring_hi=src).cpu().numpy()
    sk._ctx.status()
    assert np.all(y_all[:, :p0] == 0) and np.all(y_all[:, p1:] == 0)
    assert np.array_equal(y_all[1], -y_all[0])
    ref, idx = O.resample_nearest(nside, x.astype(np.float64), M, lo, hi, src_ring_hi=src, return_index=True)
    dev = y_all[0, p0:p1].astype(np.int64) - 1
    check_index_maps(nside, dev, idx, M, p0)
    # the source limit: exactly the device's own index map, masked by ring
    ring = np.searchsorted(st, dev, side="right") - 1
    assert np.array_equal(y_lim[0, p0:p1], np.where(ring < src, dev + 1, 0).astype(np.float32))
    assert np.all(y_lim[:, :p0] == 0) and np.all(y_lim[:, p1:] == 0)
    mism = np.nonzero(y_lim[0] != ref)[0]
    assert len(mism) <= max(2, (p1 - p0) // 100000)
    # the planned form writes the same (masked outputs cleared, other pixels untouched)
    plan = sk.ResamplePlan(g, M, lo, hi, src_ring_hi=src)
    info = plan.info()
    assert info["pixels"] == p1 - p0 and info["pairs"] == int(np.count_nonzero(y_lim[0, p0:p1]))
    out = torch.full_like(xt, 5.0)
    plan.apply(xt, out=out)
    o = out.cpu().numpy()
    sk._ctx.status()
    assert np.array_equal(o[:, p0:p1], y_lim[:, p0:p1])
    assert np.all(o[:, :p0] == 5.0) and np.all(o[:, p1:] == 5.0)


@pytest.mark.gpu
def test_resample_argument_errors(sk):
    import torch
    g = sk.Geometry(sk._ctx, 16)
    x = torch.zeros(1, g.npix, device="cuda")
    with pytest.raises(sk.SkError):
        sk.resample(g, x, 2.0 * np.eye(3), 0, 10)                  # not a rotation
    with pytest.raises(sk.SkError):
        sk.resample(g, x, np.eye(3), 0, 10, out=x)                 # overlapping maps
    with pytest.raises(sk.SkError):
        sk.resample(g, x, np.eye(3), 5, 4)
    with pytest.raises(sk.SkError):
        sk.resample(g, x, np.eye(3), 0, 64)


def field_mask(nside, theta0, phi0, radius):
    v = O.all_vecs(nside)
    c = np.array([math.sin(theta0) * math.cos(phi0), math.sin(theta0) * math.sin(phi0), math.cos(theta0)])
    return (v @ c) >= math.cos(radius)


@pytest.mark.gpu
@pytest.mark.parametrize("nside,theta0,phi0,radius_deg,fwhm,tcm", [
    (64, 1.2, 0.7, 12.0, 120.0, 240.0),
    (32, 2.9, 4.0, 20.0, 240.0, 480.0),      # a field that reaches over the south pole
    (64, 0.05, 1.0, 8.0, 120.0, 180.0),      # a field that holds the north pole
])
def test_polar_patch_matches_oracle_composition(sk, nside, theta0, phi0, radius_deg, fwhm, tcm):
    import torch
    tc = tcm * ARCMIN
    radius = math.radians(radius_deg)
    V = O.tabulate_real_kernel(gaussian_beam(fwhm, 2 * nside), nside // 2, 2 * nside, tc, 4096, 0)
    g = sk.Geometry(sk._ctx, nside)
    k = sk.Kernel(g, V, tc, 0)
    mask = field_mask(nside, theta0, phi0, radius)
    x = white_noise_maps(nside, 1, 1500 + nside)[0] * mask.astype(np.float32)
    patch = sk.PolarPatch(k, theta0, phi0, radius)
    y = patch.convolve(torch.from_numpy(x[None]).cuda()).cpu().numpy()[0]
    sk._ctx.status()
    # the oracle's composition: rotate the cap rings the sums read, sum the field's cap
    # rings, rotate back onto the sky rings of the field
    st = O.ring_starts(nside)
    xr = O.resample_nearest(nside, x, patch.rot, 0, patch.in_hi)
    outs = np.arange(0, int(st[patch.out_hi]), dtype=np.int64)
    yr = np.zeros(O.npix(nside))
    yr[outs] = O.conv_window(nside, V, tc, 0, xr, outs=outs)
    ref = O.resample_nearest(nside, yr, patch.rot.T, patch.sky_lo, patch.sky_hi, src_ring_hi=patch.out_hi)
    assert np.all(y[: st[patch.sky_lo]] == 0) and np.all(y[st[patch.sky_hi]:] == 0)
    f = mask
    assert f.sum() > 100
    assert rms_rel(y[f], ref[f]) <= 1e-6
    assert rms_rel(y, ref) <= 1e-6
    # the field's pixels all come back from summed cap rings, and the cap rings are few
    assert patch.out_hi < 4 * nside // 3
