"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the FP64 oracle.

This module holds no arithmetic of the convolution method itself: it only draws
random maps, picks point-source pixels and evaluates the closed-form Gaussian
beam transfer function that defines the workloads' input kernels (the paper's
kernel family K_l = sqrt(C_l) B_l with C_l = 1, Sec. 3, Eq. 4 of the kernel
section; the beam FWHM values of Sec. 3 and Table 1).  The split of that kernel
into a real-space table, the tabulation, and everything downstream live
separately in the product and in the oracle.

Workload recipes mirror the paper's Planck-resolution setting (HEALPix
Nside 2048, l_max 4096, Sec. 2) and the synthetic "uniform-noise" input map of
Sec. 3 read as white noise (C_l = 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ARCMIN = math.pi / (180.0 * 60.0)


def npix_of(nside: int) -> int:
    """Number of HEALPix pixels, 12 Nside^2."""
    return 12 * int(nside) * int(nside)


def white_noise_maps(nside: int, batch: int, seed: int) -> np.ndarray:
    """iid N(0,1) FP32 maps, shape [batch, 12 Nside^2], from PCG64(seed)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((batch, npix_of(nside)), dtype=np.float32)


def add_point_sources(maps: np.ndarray, count: int, amplitude: float, seed: int) -> np.ndarray:
    """Add `amplitude` at `count` distinct random pixels of every map (in place)."""
    rng = np.random.default_rng(seed)
    pix = rng.choice(maps.shape[-1], size=count, replace=False)
    maps[..., pix] += np.float32(amplitude)
    return maps


def gaussian_beam(fwhm_arcmin: float, lmax: int) -> np.ndarray:
    """Gaussian beam transfer function b_l = exp(-l(l+1) sigma^2 / 2), l = 0..lmax (FP64).

    sigma = FWHM / sqrt(8 ln 2).  With C_l = 1 this is the paper's kernel K_l.
    """
    sigma = fwhm_arcmin * ARCMIN / math.sqrt(8.0 * math.log(2.0))
    ell = np.arange(lmax + 1, dtype=np.float64)
    return np.exp(-0.5 * ell * (ell + 1.0) * sigma * sigma)


def sample_indices(n: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct indices in [0, n), sorted, from PCG64(seed)."""
    rng = np.random.default_rng(seed)
    count = min(count, n)
    return np.sort(rng.choice(n, size=count, replace=False)).astype(np.int64)


@dataclass(frozen=True)
class KernelSpec:
    """A Gaussian-beam kernel split at l_cut / theta_cut, tabulated at n_nodes."""
    fwhm_arcmin: float
    lmax: int
    lcut: int
    theta_cut_arcmin: float
    n_nodes: int
    layout: int = 0          # 0 uniform nodes, 1 half the nodes in the first 1/16

    @property
    def theta_cut(self) -> float:
        return self.theta_cut_arcmin * ARCMIN

    def beam(self) -> np.ndarray:
        return gaussian_beam(self.fwhm_arcmin, self.lmax)


@dataclass(frozen=True)
class Group:
    nside: int
    batch: int
    kernel: KernelSpec
    seed: int


@dataclass(frozen=True)
class Workload:
    name: str
    groups: tuple
    sources: tuple = field(default=())   # (count, amplitude, seed) per group, or empty


def _k(fwhm, nside, tc, nt, lmax=None, lcut=None):
    lmax = 2 * nside if lmax is None else lmax
    lcut = lmax // 4 if lcut is None else lcut
    return KernelSpec(fwhm, lmax, lcut, tc, nt)


# The workloads.  Sizes: Nside 64 .. 8192; theta_cut 5' .. 300'.
WORKLOADS = {
    "n64_plain": Workload("n64_plain", (Group(64, 1, _k(60.0, 64, 180.0, 4096, 192, 96), 101),)),
    "n2048_plain": Workload("n2048_plain",
                            (Group(2048, 1, _k(7.1, 2048, 20.0, 8192, 4096, 1024), 201),),
                            sources=((1000, 100.0, 202),)),
    "n1024x64_batched": Workload("n1024x64_batched",
                                 (Group(1024, 64, _k(10.0, 1024, 30.0, 4096), 301),)),
    "mixed_batch": Workload("mixed_batch", (
        Group(256, 8, _k(60.0, 256, 180.0, 4096), 311),
        Group(512, 8, _k(30.0, 512, 90.0, 4096), 312),
        Group(1024, 4, _k(10.0, 1024, 30.0, 4096), 313),
        Group(2048, 2, _k(5.0, 2048, 15.0, 4096), 314),
    )),
    "n1024x16_grad": Workload("n1024x16_grad",
                              (Group(1024, 16, _k(10.0, 1024, 30.0, 4096), 401),)),
    "n8192_plain": Workload("n8192_plain",
                            (Group(8192, 1, _k(2.0, 8192, 5.0, 16384, 16384, 4096), 501),)),
    # the paper's optimum split for a 7' beam (Sec. 4, Table 1: l_cut 1158, theta_cut 390')
    # at Planck resolution; ~1.6e5 neighbours per pixel
    "n2048_table1": Workload("n2048_table1", (Group(2048, 1, KernelSpec(7.0, 4096, 1158, 390.0, 8192), 801),)),
    # wide cut (the ring-pair Fourier form of the belt): 300' windows, ~2.3e4 neighbours per pixel
    "n1024_wide": Workload("n1024_wide", (Group(1024, 1, _k(60.0, 1024, 300.0, 4096), 601),)),
    # a partial-sky field (a disc of FIELD_RADIUS_DEG, ~310 square degrees, the size of the
    # ground-based surveys the paper names) at Nside 8192 with the 5' kernel
    "n8192_field": Workload("n8192_field",
                            (Group(8192, 1, _k(2.0, 8192, 5.0, 16384, 16384, 4096), 701),)),
}

# Centre (colatitude, longitude, radians) and radius of the partial-sky field.
FIELD_CENTRE = (1.0, 0.5)
FIELD_RADIUS_DEG = 10.0

# Gradient workload: the target map comes from the same maps convolved with a
# 10.5' kernel; the finite-difference entries are drawn with this seed.
GRAD_TARGET_FWHM = 10.5
GRAD_FD_SEED = 402


def make_maps(group: Group, sources=None) -> np.ndarray:
    m = white_noise_maps(group.nside, group.batch, group.seed)
    if sources:
        count, amp, seed = sources
        add_point_sources(m, count, amp, seed)
    return m
