"""The tensor-core form of the belt (3xTF32 tcgen05 contractions of stored weight
tiles with sliding rows of the maps) against the FP64 oracle and against the FP32
form, through the C ABI: the operator's belt-form setting, its tiles following
table updates (host and device-side), CUDA-graph capture, the operators without a
tensor form, the widened autotuner and its cache, and the plain Nside-2048
workload at full size on sampled outputs.

The operator is the real-space convolution of Sec. 2, Eq. 1 with the tabulated
kernel of Sec. 3.  Bar: rms relative error <= 1e-6 against the oracle (same
FP32 input promoted to FP64, same FP64 table); the two belt forms differ only in
rounding, so they agree to the same bar.
"""
import math

import numpy as np
import pytest

import oracle as O
from inputs import ARCMIN, WORKLOADS, add_point_sources, gaussian_beam, sample_indices, white_noise_maps

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


def table(fwhm, lmax, lcut, tc, nt, layout=0):
    return O.tabulate_real_kernel(gaussian_beam(fwhm, lmax), lcut, lmax, tc, nt, layout)


def conv(sk, k, xt, path=0):
    import torch
    y = sk.convolve(k, xt, path=path)
    torch.cuda.synchronize()
    sk._ctx.status()
    return y


def test_belt_form_selects_the_auto_path(sk):
    import torch
    nside, tc = 128, 0.03
    V = table(2.5 * tc / 3 / ARCMIN, 384, 96, tc, 2048)
    k = sk.Kernel(sk.Geometry(sk._ctx, nside), V, tc)
    assert k.config()["tensor_form_available"] and k.config()["belt_form"] == "fp32"
    x = torch.from_numpy(white_noise_maps(nside, 3, 501)).cuda()
    yf, yt = conv(sk, k, x, sk.PATH_FP32), conv(sk, k, x, sk.PATH_TENSOR)
    assert torch.equal(conv(sk, k, x), yf)
    k.set_belt_form(sk.BELT_TENSOR)
    assert k.config()["belt_form"] == "tensor"
    assert torch.equal(conv(sk, k, x), yt)
    assert torch.equal(conv(sk, k, x, sk.PATH_FP32), yf)
    k.set_belt_form(sk.BELT_FP32)
    assert torch.equal(conv(sk, k, x), yf)
    for b in range(3):
        yo = O.conv_window(nside, V, tc, 0, x[b].cpu().numpy().astype(np.float64))
        assert rms_rel(yt[b].cpu().numpy(), yo) <= RMS_BOUND
    assert rms_rel(yt.cpu().numpy(), yf.cpu().numpy()) <= RMS_BOUND


def test_operators_without_a_tensor_form(sk):
    import torch
    # rings of 4 Nside = 64 pixels are shorter than the 128-pixel minimum of the form
    nside, tc = 16, 0.3
    V = table(2.5 * tc / 3 / ARCMIN, 48, 12, tc, 512)
    k = sk.Kernel(sk.Geometry(sk._ctx, nside), V, tc)
    assert not k.config()["tensor_form_available"]
    with pytest.raises(sk.SkError):
        k.set_belt_form(sk.BELT_TENSOR)
    x = torch.from_numpy(white_noise_maps(nside, 1, 502)).cuda()
    # the tensor path runs the FP32 belt for it
    assert torch.equal(conv(sk, k, x, sk.PATH_TENSOR), conv(sk, k, x, sk.PATH_FP32))


@pytest.mark.parametrize("device_update", [False, True])
def test_tensor_tiles_follow_table_updates(sk, device_update):
    import torch
    nside, tc, nt = 64, 0.06, 1024
    V1 = table(2.5 * tc / 3 / ARCMIN, 192, 48, tc, nt)
    V2 = table(3.0 * tc / 3 / ARCMIN, 192, 48, tc, nt)
    k = sk.Kernel(sk.Geometry(sk._ctx, nside), V1, tc)
    k.set_belt_form(sk.BELT_TENSOR)
    x = torch.from_numpy(white_noise_maps(nside, 1, 503)).cuda()
    conv(sk, k, x)
    if device_update:
        k.update_values_async(torch.from_numpy(V2).cuda())
    else:
        k.update_values(V2)
    y = conv(sk, k, x)[0].cpu().numpy()
    assert rms_rel(y, O.conv_window(nside, V2, tc, 0, x[0].cpu().numpy().astype(np.float64))) <= RMS_BOUND


def test_graph_with_the_tensor_form_equals_eager(sk):
    import torch
    nside, tc = 128, 0.03
    V = table(2.5 * tc / 3 / ARCMIN, 384, 96, tc, 2048, 1)
    k = sk.Kernel(sk.Geometry(sk._ctx, nside), V, tc, 1)
    k.set_belt_form(sk.BELT_TENSOR)
    x = torch.from_numpy(white_noise_maps(nside, 2, 504)).cuda()
    ref = conv(sk, k, x)
    y = torch.zeros_like(x)
    gr = sk.Graph(sk._ctx, [(k, x, y)])
    for _ in range(2):
        y.zero_()
        gr.launch()
        torch.cuda.synchronize()
        assert torch.equal(y, ref)
    gr.close()
    sk._ctx.status()


def test_autotuner_chooses_among_forms_and_caches(sk, tmp_path):
    import torch
    nside, tc = 512, 0.0262
    V = table(2.5 * tc / 3 / ARCMIN, 1536, 384, tc, 4096)
    k = sk.Kernel(sk.Geometry(sk._ctx, nside), V, tc)
    x = torch.from_numpy(white_noise_maps(nside, 2, 505)).cuda()
    cache = tmp_path / "tune.txt"
    p = k.autotune(x, cache_path=str(cache))
    c = k.config()
    assert c["belt_p"] == p and c["belt_form"] in ("fp32", "tensor")
    line = cache.read_text().split()
    assert len(line) == 4 and int(line[1]) == p
    assert int(line[2]) == (1 if c["belt_form"] == "tensor" else 0)
    assert int(line[3]) == (1 if c["cap_weights"] == "stored" else 0)
    k2 = sk.Kernel(sk.Geometry(sk._ctx, nside), V, tc)
    assert k2.autotune(x, cache_path=str(cache)) == p and k2.config() == c     # served by the cache
    y = conv(sk, k2, x)
    for b in range(2):
        outs = sample_indices(x.shape[1], 3000, 506 + b)
        yo = O.conv_window(nside, V, tc, 0, x[b].cpu().numpy().astype(np.float64), outs)
        assert rms_rel(y[b].cpu().numpy()[outs], yo) <= RMS_BOUND


def test_tensor_form_n2048_plain_sampled_outputs(sk):
    wl = WORKLOADS["n2048_plain"]
    grp = wl.groups[0]
    ks = grp.kernel
    V = O.tabulate_real_kernel(ks.beam(), ks.lcut, ks.lmax, ks.theta_cut, ks.n_nodes, ks.layout)
    k = sk.Kernel(sk.Geometry(sk._ctx, grp.nside), V, ks.theta_cut, ks.layout)
    k.set_belt_form(sk.BELT_TENSOR)
    x = white_noise_maps(grp.nside, 1, grp.seed)
    add_point_sources(x, *wl.sources[0])
    import torch
    y = conv(sk, k, torch.from_numpy(x).cuda())[0].cpu().numpy()
    outs = sample_indices(x.shape[1], 20000, 207)
    yo = O.conv_window(grp.nside, V, ks.theta_cut, ks.layout, x[0].astype(np.float64), outs)
    assert rms_rel(y[outs], yo) <= RMS_BOUND


def test_bf16x3_form_reported_with_its_error(sk):
    # BF16x3 (BF16 hi/lo parts, three kind::f16 MMAs) keeps about 16 significant bits of
    # each operand: its error against the oracle is reported, ~1e-5 relative -- outside the
    # 1e-6 bound the other forms meet (the tuner never picks it)
    import torch
    nside, tc = 256, 0.02
    V = table(2.5 * tc / 3 / ARCMIN, 768, 192, tc, 2048)
    k = sk.Kernel(sk.Geometry(sk._ctx, nside), V, tc)
    c = k.config()
    assert c["bf16x3_form_available"] and c["tensor_form_available"]
    x = torch.from_numpy(white_noise_maps(nside, 3, 510)).cuda()
    yb = conv(sk, k, x, sk.PATH_BF16X3)
    yt = conv(sk, k, x, sk.PATH_TENSOR)
    k.set_belt_form(sk.BELT_BF16X3)
    assert k.config()["belt_form"] == "bf16x3"
    assert torch.equal(conv(sk, k, x), yb)
    for b in range(3):
        yo = O.conv_window(nside, V, tc, 0, x[b].cpu().numpy().astype(np.float64))
        eb = rms_rel(yb[b].cpu().numpy(), yo)
        et = rms_rel(yt[b].cpu().numpy(), yo)
        assert et <= RMS_BOUND
        assert 1e-6 < eb < 5e-5, eb
    k.set_belt_form(sk.BELT_FP32)
