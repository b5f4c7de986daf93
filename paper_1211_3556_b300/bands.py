"""Ring-band decomposition of one map over several devices (ranks).

The real-space sum of an output pixel reads the input pixels within theta_cut, which
lie on the rings whose colatitude is within theta_cut of its own (Sec. 2: the kernel is
truncated at theta_cut).  So a rank that owns a band of output rings [o_lo, o_hi) needs
the input rings of colatitude within theta_cut of the band, its halo [i_lo, i_hi); in
RING order both are contiguous pixel ranges.  Bands hold about equal pixel counts (the
number of in-cut pairs per pixel is nearly the same everywhere).  The input reaches
every rank by one halo exchange: each rank sends every other rank only the part of its
own band inside that rank's halo (point-to-point; exchange_halo); each rank then computes
its band with convolve_rings and the outputs stay sharded.  Host-side logic only: the ring tables follow the HEALPix
RING scheme (Gorski et al. 2005, the pixelisation of Sec. 2).

symmetric_bands gives each rank a northern range of rings and its mirror about the
equator instead (convolve_rings_sym): the polar-cap sums treat a ring and its mirror
together, so a one-sided band holding cap rings would also pay for their mirrors, and
the bands are balanced by an estimate of their cost (pixels, with the cap rings weighted
by the cost of a cap pair relative to a belt pair) rather than by pixel count.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def ring_table(nside: int):
    """Per ring (0-based, 4 nside - 1 rings): pixel count, first pixel, colatitude."""
    N = int(nside)
    nr = 4 * N - 1
    n = np.empty(nr, np.int64)
    z = np.empty(nr, np.float64)
    for r in range(1, nr + 1):
        if r < N:
            n[r - 1], z[r - 1] = 4 * r, 1.0 - r * r / (3.0 * N * N)
        elif r <= 3 * N:
            n[r - 1], z[r - 1] = 4 * N, 4.0 / 3.0 - 2.0 * r / (3.0 * N)
        else:
            rr = 4 * N - r
            n[r - 1], z[r - 1] = 4 * rr, -(1.0 - rr * rr / (3.0 * N * N))
    start = np.concatenate(([0], np.cumsum(n)[:-1]))
    return n, start, np.arccos(np.clip(z, -1.0, 1.0))


@dataclass(frozen=True)
class Band:
    rank: int
    out_rings: tuple     # [lo, hi)
    in_rings: tuple      # [lo, hi): the rings within theta_cut of the band
    out_pix: tuple       # [p0, p1) in RING order
    in_pix: tuple


def ring_bands(nside: int, theta_cut: float, world: int) -> list:
    """Split the output rings into `world` contiguous bands of about equal pixel counts."""
    n, start, theta = ring_table(nside)
    nr = len(n)
    npix = int(n.sum())
    world = max(1, min(int(world), nr))
    cum = np.cumsum(n)
    edges = [0]
    for r in range(1, world):
        edges.append(max(edges[-1] + 1, int(np.searchsorted(cum, r * npix / world)) + 1))
    edges.append(nr)
    edges = [min(e, nr) for e in edges]
    out = []
    # rings at a tie, and rings that the device's FP32 cut test (chord^2 <= its FP32 value)
    # may take in, join the halo: a margin well above FP32 rounding of the angle
    eps = 1e-6 * max(1.0, theta_cut)
    for rank in range(world):
        lo, hi = edges[rank], edges[rank + 1]
        if hi <= lo:
            out.append(Band(rank, (lo, lo), (lo, lo), (0, 0), (0, 0)))
            continue
        ilo = int(np.searchsorted(theta, theta[lo] - theta_cut - eps, side="left"))
        ihi = int(np.searchsorted(theta, theta[hi - 1] + theta_cut + eps, side="right"))
        out.append(Band(rank, (lo, hi), (ilo, ihi),
                        (int(start[lo]), int(start[hi - 1] + n[hi - 1])),
                        (int(start[ilo]), int(start[ihi - 1] + n[ihi - 1]))))
    return out


def _ranges(r) -> list:
    """A band's ring or pixel ranges as a list of (lo, hi)."""
    return [tuple(q) for q in r] if len(r) and isinstance(r[0], (tuple, list)) else [tuple(r)]


def _merge(ranges) -> tuple:
    out = []
    for lo, hi in sorted(r for r in ranges if r[1] > r[0]):
        if out and lo <= out[-1][1]:
            out[-1] = (out[-1][0], max(out[-1][1], hi))
        else:
            out.append((lo, hi))
    return tuple(out)


@dataclass(frozen=True)
class SymBand:
    rank: int
    north: tuple         # [lo, hi): northern rings (hi at most the equator ring + 1)
    out_rings: tuple     # ring ranges written: the north range and its mirror, merged where they meet
    in_rings: tuple      # ring ranges within theta_cut of them
    out_pix: tuple       # the same as pixel ranges (RING order)
    in_pix: tuple


def ring_costs(pairs, path, cost_per_pair) -> np.ndarray:
    """Cost of each output ring: its in-cut pairs (Kernel.pairs_by_ring) times the measured
    cost of one pair on the ring's path (cost_per_pair[path]: 0 belt, 1 cap, 2 per-pair,
    3 cap with wide windows)."""
    c = np.asarray(cost_per_pair, dtype=np.float64)
    return np.asarray(pairs, dtype=np.float64) * c[np.asarray(path, dtype=np.int64)]


def symmetric_bands(nside: int, theta_cut: float, world: int, cap_cost: float = 2.5, ring_cost=None) -> list:
    """Split the northern rings (the equator included) into `world` contiguous ranges of
    about equal cost, each with its mirror about the equator.  The cost of a northern ring
    is ring_cost[r] + ring_cost[mirror] (the equator once) when ring_cost (one entry per
    ring, e.g. ring_costs()) is given; otherwise the model: its pixels, twice, times
    cap_cost on the polar-cap rings (ring index below Nside, 1-based)."""
    n, start, theta = ring_table(nside)
    nr = len(n)
    N = int(nside)
    eq = 2 * N - 1                                    # the equator ring (0-based), its own mirror
    if ring_cost is not None:
        rc = np.asarray(ring_cost, dtype=np.float64)
        if rc.shape != (nr,):
            raise ValueError("ring_cost needs one entry per ring")
        w = np.array([rc[r] + (0.0 if r == eq else rc[nr - 1 - r]) for r in range(eq + 1)])
    else:
        w = np.array([n[r] * (cap_cost if r < N - 1 else 1.0) * (1.0 if r == eq else 2.0) for r in range(eq + 1)])
    cum = np.cumsum(w)
    world = max(1, min(int(world), eq + 1))
    edges = [0]
    for k in range(1, world):
        edges.append(max(edges[-1] + 1, int(np.searchsorted(cum, k * cum[-1] / world)) + 1))
    edges.append(eq + 1)
    edges = [min(e, eq + 1) for e in edges]
    eps = 1e-6 * max(1.0, theta_cut)                  # the margin of ring_bands

    def halo(lo, hi):
        ilo = int(np.searchsorted(theta, theta[lo] - theta_cut - eps, side="left"))
        ihi = int(np.searchsorted(theta, theta[hi - 1] + theta_cut + eps, side="right"))
        return ilo, ihi

    def pix(rr):
        return tuple((int(start[lo]), int(start[hi - 1] + n[hi - 1])) for lo, hi in rr)

    out = []
    for rank in range(world):
        lo, hi = edges[rank], edges[rank + 1]
        if hi <= lo:
            out.append(SymBand(rank, (lo, lo), (), (), (), ()))
            continue
        rings = _merge([(lo, hi), (nr - hi, nr - lo)])
        halos = _merge([halo(a, b) for a, b in rings])
        out.append(SymBand(rank, (lo, hi), rings, halos, pix(rings), pix(halos)))
    return out


def _intersect(a: list, b: list) -> list:
    """Pieces (lo, hi) of the ranges a that lie in the ranges b, in the order of a."""
    out = []
    for a0, a1 in a:
        for b0, b1 in b:
            lo, hi = max(a0, b0), min(a1, b1)
            if hi > lo:
                out.append((lo, hi))
    return out


def halo_plan(band, bands: list):
    """What `band`'s rank exchanges: for every other rank q, the pixel pieces of its own
    bands it sends to q (its out_pix inside q's halo) and the pieces it receives from q
    (q's out_pix inside its own halo).  Pieces are RING-order pixel ranges; both sides
    derive them from the same band table, so no sizes are exchanged."""
    me = band.rank
    mine = _ranges(band.out_pix) if len(band.out_pix) else []
    my_halo = _ranges(band.in_pix) if len(band.in_pix) else []
    send, recv = {}, {}
    for b in bands:
        if b.rank == me:
            continue
        theirs = _ranges(b.out_pix) if len(b.out_pix) else []
        their_halo = _ranges(b.in_pix) if len(b.in_pix) else []
        s = _intersect(mine, their_halo)
        r = _intersect(theirs, my_halo)
        if s:
            send[b.rank] = s
        if r:
            recv[b.rank] = r
    return send, recv


def exchange_halo(x_own, band, bands: list, npix: int, group=None, stats: dict = None, out=None):
    """The input map of `band`'s rank from every rank's own pixels, moving only halos:
    x_own [batch, own] holds this rank's band of the input (its out_pix ranges,
    concatenated in order).  Each rank sends every other rank the part of its band that
    lies in that rank's halo and receives the parts of the others' bands in its own halo
    (point-to-point, batched: NCCL or gloo).  Returns [batch, npix] with the halo (and
    the own band) filled and zeros elsewhere -- or fills `out` ([batch, npix], whose
    other pixels are left as they are: they must be finite) and returns it.  With
    `stats`, stats["recv_bytes"] and stats["send_bytes"] count the bytes moved.  Bands
    of ring_bands or symmetric_bands."""
    import torch
    import torch.distributed as dist
    batch = x_own.shape[0]
    full = out if out is not None else torch.zeros(batch, npix, dtype=x_own.dtype, device=x_own.device)
    mine = _ranges(band.out_pix) if len(band.out_pix) else []
    pos = 0
    for q0, q1 in mine:
        full[:, q0:q1] = x_own[:, pos: pos + q1 - q0]
        pos += q1 - q0
    send, recv = halo_plan(band, bands)

    def own_offset(p):                        # position of own pixel p in x_own
        off = 0
        for q0, q1 in mine:
            if q0 <= p < q1:
                return off + p - q0
            off += q1 - q0
        raise ValueError(p)

    ops, bufs = [], {}
    nb = 0
    for q, pieces in sorted(send.items()):
        t = torch.cat([x_own[:, own_offset(a): own_offset(a) + (z - a)] for a, z in pieces], dim=1).contiguous()
        ops.append(dist.P2POp(dist.isend, t, q, group=group))
        nb += t.numel() * t.element_size()
    nr = 0
    for q, pieces in sorted(recv.items()):
        t = torch.empty(batch, sum(z - a for a, z in pieces), dtype=x_own.dtype, device=x_own.device)
        bufs[q] = t
        ops.append(dist.P2POp(dist.irecv, t, q, group=group))
        nr += t.numel() * t.element_size()
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for q, pieces in recv.items():
        pos = 0
        for a, z in pieces:
            full[:, a:z] = bufs[q][:, pos: pos + z - a]
            pos += z - a
    if stats is not None:
        stats["recv_bytes"] = nr
        stats["send_bytes"] = nb
    return full
