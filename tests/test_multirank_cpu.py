"""The multi-rank (N > 1) logic of bench.py on CPU ranks over gloo, world size 2.

Under weak scaling every rank convolves its own maps (no collective on the data
path); only the step time is reduced, with MAX, and the aggregate rate is the
units of all ranks over that time.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    from inputs import white_noise_maps
    dist.init_process_group("gloo", rank=rank, world_size=world)
    maps = white_noise_maps(4, 2, 5)
    mine = bench.shard_maps(maps, rank, world)
    step_s = 0.010 * (rank + 1)                      # rank 1 is the slower one
    t = bench.max_over_ranks(step_s, world, "cpu")
    rate = bench.aggregate_rate(1000.0, world, t)
    out[rank] = (float(mine.sum()), float(mine[0, 0]), t, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_weak_scaling_logic_world_size_2():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    (s0, first0, t0, r0), (s1, first1, t1, r1) = out[0], out[1]
    assert t0 == pytest.approx(0.020) and t1 == pytest.approx(0.020)        # MAX over ranks
    assert r0 == pytest.approx(1000.0 * 2 / 0.020) and r0 == r1
    assert s0 == pytest.approx(s1, rel=1e-6)        # same data, shifted: the sums agree
    assert first0 != first1                          # but each rank has its own maps


# ---------------------------------------------------------------- ring bands of one map

def _band_rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import math
    import torch
    import torch.distributed as dist
    import oracle as O
    from inputs import gaussian_beam, white_noise_maps
    from paper_1211_3556_b300.bands import exchange_halo, ring_bands
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nside, tc = 8, math.radians(30.0)
    V = O.tabulate_real_kernel(gaussian_beam(600.0, 16), 4, 16, tc, 512, 0)
    x = white_noise_maps(nside, 1, 77)[0].astype(np.float64)
    npix = x.size
    bands = ring_bands(nside, tc, world)
    me = bands[rank]
    p0, p1 = me.out_pix
    # each rank starts from its own band of the input only
    x_own = torch.from_numpy(x[None, p0:p1].copy())
    stats = {}
    x_halo = exchange_halo(x_own, me, bands, npix, stats=stats)[0].numpy()
    # only the halo moves: the pixels of the halo that other ranks own, once each
    out[f"bytes_ok_{rank}"] = stats["recv_bytes"] == ((me.in_pix[1] - me.in_pix[0]) - (p1 - p0)) * 8
    # the oracle stands in for the device sums: this rank's outputs from its halo
    y_mine = O.conv_window(nside, V, tc, 0, x_halo, outs=np.arange(p0, p1, dtype=np.int64))
    outs = [None] * world
    dist.all_gather_object(outs, (p0, p1, y_mine.tolist()))
    if rank == 0:
        y = np.zeros(npix)
        for q0, q1, vals in outs:
            y[q0:q1] = vals
        out["stitched"] = y.tolist()
        out["full"] = O.conv_window(nside, V, tc, 0, x).tolist()
        out["halo_zero_outside"] = bool(np.all(x_halo[: me.in_pix[0]] == 0) and np.all(x_halo[me.in_pix[1]:] == 0))
    dist.barrier()
    dist.destroy_process_group()


def test_ring_bands_halo_exchange_and_stitching_world_size_2():
    # one map split into two ring bands; the halo comes by a halo-only exchange over gloo, each
    # rank sums its band (the FP64 oracle in place of the device), and the stitched map
    # equals the full sum exactly (the same terms in the same order)
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_band_rank_main, args=(world, port, out), nprocs=world, join=True)
    assert out["halo_zero_outside"]
    assert all(out[f"bytes_ok_{r}"] for r in range(world))
    assert np.array_equal(np.array(out["stitched"]), np.array(out["full"]))


@pytest.mark.parametrize("nside,deg,world", [(8, 30.0, 2), (16, 80.0, 4), (64, 3.0, 3), (32, 1.0, 7)])
def test_ring_bands_tile_the_rings_and_cover_the_windows(nside, deg, world):
    import math
    import oracle as O
    from paper_1211_3556_b300.bands import ring_bands, ring_table
    n, start, theta = ring_table(nside)
    for r in range(len(n)):                                   # ring tables pinned to the oracle's
        on, ost, _, oz, _ = O.ring_info(nside, r + 1)
        assert (n[r], start[r]) == (on, ost) and math.cos(theta[r]) == pytest.approx(oz, abs=1e-15)
    tc = math.radians(deg)
    bands = ring_bands(nside, tc, world)
    assert bands[0].out_rings[0] == 0 and bands[-1].out_rings[1] == len(n)
    for a, b in zip(bands, bands[1:]):
        assert a.out_rings[1] == b.out_rings[0] and a.out_pix[1] == b.out_pix[0]
    for b in bands:
        lo, hi = b.out_rings
        if hi == lo:
            continue
        ilo, ihi = b.in_rings
        assert ilo <= lo and ihi >= hi
        for i in range(len(n)):                               # the rings within theta_cut, and
            gap = min(abs(theta[i] - theta[o]) for o in range(lo, hi))   # those within 1e-6 rad
            if gap <= tc:                                     # of it (FP32 margin)
                assert ilo <= i < ihi
            elif ilo <= i < ihi:
                assert gap - tc <= 1e-6


# ---------------------------------------------------------------- symmetric ring bands

def _sym_band_rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import math
    import torch
    import torch.distributed as dist
    import oracle as O
    from inputs import gaussian_beam, white_noise_maps
    from paper_1211_3556_b300.bands import exchange_halo, symmetric_bands
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nside, tc = 16, math.radians(12.0)
    V = O.tabulate_real_kernel(gaussian_beam(240.0, 32), 8, 32, tc, 512, 0)
    x = white_noise_maps(nside, 1, 78)[0].astype(np.float64)
    npix = x.size
    bands = symmetric_bands(nside, tc, world)
    me = bands[rank]
    # each rank starts from its own rings only (north range and mirror, concatenated)
    outs_mine = np.concatenate([np.arange(q0, q1, dtype=np.int64) for q0, q1 in me.out_pix])
    x_own = torch.from_numpy(x[None, outs_mine].copy())
    stats = {}
    x_halo = exchange_halo(x_own, me, bands, npix, stats=stats)[0].numpy()
    halo_px = sum(p1 - p0 for p0, p1 in me.in_pix)
    out[f"bytes_ok_{rank}"] = stats["recv_bytes"] == (halo_px - len(outs_mine)) * 8
    inside = np.zeros(npix, bool)
    for p0, p1 in me.in_pix:
        inside[p0:p1] = True
    y_mine = O.conv_window(nside, V, tc, 0, x_halo, outs=outs_mine)
    res = [None] * world
    dist.all_gather_object(res, (outs_mine.tolist(), y_mine.tolist()))
    if rank == 0:
        y = np.full(npix, np.nan)
        for o, vals in res:
            assert np.all(np.isnan(y[o]))                 # every pixel written by one rank only
            y[o] = vals
        out["stitched"] = y.tolist()
        out["full"] = O.conv_window(nside, V, tc, 0, x).tolist()
    out[f"halo_ok_{rank}"] = bool(np.all(x_halo[~inside] == 0) and np.array_equal(x_halo[inside], x[inside]))
    dist.barrier()
    dist.destroy_process_group()


def test_symmetric_bands_halo_exchange_and_stitching_world_size_3():
    # bands of a northern range and its mirror: halos (two ranges, or one where they meet)
    # by a halo-only exchange, each rank's sums from its halo (the oracle in place of the device),
    # the stitched map equal to the full sum exactly
    world = 3
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_sym_band_rank_main, args=(world, port, out), nprocs=world, join=True)
    assert all(out[f"halo_ok_{r}"] for r in range(world))
    assert all(out[f"bytes_ok_{r}"] for r in range(world))
    assert np.array_equal(np.array(out["stitched"]), np.array(out["full"]))


@pytest.mark.parametrize("nside,deg,world", [(8, 30.0, 2), (16, 12.0, 3), (64, 3.0, 5), (128, 1.0, 8)])
def test_symmetric_bands_tile_the_rings_cover_the_windows_and_balance(nside, deg, world):
    import math
    from paper_1211_3556_b300.bands import ring_table, symmetric_bands
    n, start, theta = ring_table(nside)
    nr = len(n)
    tc = math.radians(deg)
    bands = symmetric_bands(nside, tc, world, cap_cost=2.5)
    owner = np.full(nr, -1)
    for b in bands:
        lo, hi = b.north
        assert 0 <= lo <= hi <= 2 * nside
        for a, z in b.out_rings:
            assert np.all(owner[a:z] == -1)
            owner[a:z] = b.rank
        for r in range(lo, hi):                               # a northern ring with its mirror
            assert owner[r] == b.rank and owner[nr - 1 - r] == b.rank
        inr = np.zeros(nr, bool)
        for a, z in b.in_rings:
            inr[a:z] = True
        outs = [o for a, z in b.out_rings for o in range(a, z)]
        for i in range(nr):
            if not outs:
                break
            gap = min(abs(theta[i] - theta[o]) for o in outs)
            if gap <= tc:
                assert inr[i]
            elif inr[i]:
                assert gap - tc <= 1e-6
        for (a, z), (p, q) in zip(b.out_rings, b.out_pix):
            assert (p, q) == (start[a], start[z - 1] + n[z - 1])
    assert np.all(owner >= 0)
    # balance of the cost estimate the split uses
    cost = []
    for b in bands:
        lo, hi = b.north
        cost.append(sum(n[r] * (2.5 if r < nside - 1 else 1.0) * (1 if r == 2 * nside - 1 else 2)
                        for r in range(lo, hi)))
    ring_max = max(n[r] * 2.5 * 2 for r in range(2 * nside))
    assert max(cost) - min(cost) <= 2 * ring_max + 1e-9


@pytest.mark.parametrize("nside,world", [(64, 4), (256, 8)])
def test_symmetric_bands_balance_given_ring_costs(nside, world):
    # with per-ring costs (pairs x the measured cost of a pair on the ring's path) every band
    # carries its share of the total within the cost of one northern ring (ring + mirror)
    from paper_1211_3556_b300.bands import ring_costs, ring_table, symmetric_bands
    n, _, _ = ring_table(nside)
    nr = len(n)
    rng = np.random.default_rng(nside + world)
    pairs = (n * rng.uniform(50, 150, nr)).astype(np.int64)
    path = np.where(np.arange(nr) < nside, 1, 0).astype(np.uint8)
    path[nr - nside:] = 1
    rc = ring_costs(pairs, path, [1.0, 4.0, 2.0, 3.0])
    assert np.allclose(rc[path == 1], 4.0 * pairs[path == 1])
    bands = symmetric_bands(nside, 0.05, world, ring_cost=rc)
    eq = 2 * nside - 1
    w = np.array([rc[r] + (0.0 if r == eq else rc[nr - 1 - r]) for r in range(eq + 1)])
    cost = [w[b.north[0]:b.north[1]].sum() for b in bands]
    assert abs(sum(cost) - w.sum()) < 1e-6 * w.sum()
    assert max(abs(c - w.sum() / world) for c in cost) <= w.max() + 1e-9 * w.sum()
    with pytest.raises(ValueError):
        symmetric_bands(nside, 0.05, world, ring_cost=rc[:-1])
