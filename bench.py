#!/usr/bin/env python3
"""Benchmark of the real-space HEALPix convolution (pixel pairs per second).

One step = one pass of the whole forward operator (belt weight rows, belt
Toeplitz sums, symmetric cap sums, any per-pair rings) over one batch of
synthetic maps that are already resident in HBM.  The default workload is a
single Planck-like map: Nside 2048 (50.3 M pixels), white noise plus 1000
point sources of amplitude 100, Gaussian beam FWHM 7.1', l_max 4096, split at
l_cut 1024, theta_cut 20', 8192-node table.  The map (201 MB) is larger than
the 126 MB L2, so consecutive steps read it from HBM.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload NAME]
Under torchrun (N > 1) every rank convolves its own maps (weak scaling, no
collective on the data path); the step time is the max over ranks.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from inputs import ARCMIN, WORKLOADS, Group, make_maps, npix_of, sample_indices  # noqa: E402

METRIC = "pixel-pairs/s and ms/map at Nside 2048, plain vs batched, rms err vs FP64"
UNIT = "pixel-pairs/s"

# FP32 lanes per SM (the unit count behind the derived FP32 peak, SM count x lanes x
# 2 flop x maximum SM clock, which the bench reports beside the measured one).
LANES = 128
# Algorithmic flops per in-cut pixel pair and map: the multiply-accumulate every
# direct sum must do (the table lerp and chord are amortised by the belt and cap
# paths, so they are not counted).
FLOP_PER_PAIR = 2.0
# Per-pair flops of a plain per-pair evaluation (chord 8, table coordinate 2,
# lerp 2, multiply-accumulate 2), reported as f_eval for context.
FLOP_PER_PAIR_EVAL = 14.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n2048_plain", choices=sorted(WORKLOADS))
    ap.add_argument("--no-batched", action="store_true", help="skip the batched side measurement")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--no-split", action="store_true", help="skip the harmonic-half (split) side measurement")
    ap.add_argument("--no-fourier", action="store_true", help="skip the wide-cut (ring-pair Fourier) side measurement")
    ap.add_argument("--no-grad", action="store_true", help="skip the gradient (adjoint + table gradient) side measurement")
    ap.add_argument("--no-field", action="store_true", help="skip the partial-sky field (polar-cap) side measurement")
    ap.add_argument("--no-bands", action="store_true", help="skip the ring-band (one map over several GPUs) side measurement")
    ap.add_argument("--errors", action="store_true",
                    help="the split's error study (Sec. 3): estimated and actual errors of the split "
                         "convolution of a white-noise map for several l_cut at a fixed theta_cut")
    ap.add_argument("--table1", action="store_true",
                    help="one point of the paper's Table 1 (7' beam, l_cut 1158, theta_cut 390', Nside 2048): "
                         "the real-space part (ring-pair Fourier zone + direct rings) and the harmonic part, "
                         "timed, with the real-space result against the oracle on sampled outputs")
    ap.add_argument("--bands", action="store_true",
                    help="strong scaling of one map: under torchrun each rank owns a symmetric ring band of "
                         "the workload's first map, and a step is the halo exchange plus the band's sums")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard_maps(maps: np.ndarray, rank: int, world: int) -> np.ndarray:
    """Maps of one rank under weak scaling: every rank convolves its own copy of the
    workload, made distinct by a cyclic pixel shift of `rank` (no data exchange)."""
    if world <= 1:
        return maps
    return np.ascontiguousarray(np.roll(maps, rank, axis=1))


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Largest value over the ranks (the slowest rank sets the step time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the max step time."""
    return units_per_rank * world / seconds


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-i", str(gpu_index), "-lms", "50"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        # wait (bounded) for the first sample so that the timed region is covered
        t0 = time.time()
        while self.p is not None and time.time() - t0 < 5.0:
            self.f.flush()
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            try:
                sm.append(float(r[1])); smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def gaussian_beam_of(ks, lmax):
    from inputs import gaussian_beam
    return gaussian_beam(ks.fwhm_arcmin, lmax)


def build_operator(sk, ctx, group):
    ks = group.kernel
    g = sk.Geometry(ctx, group.nside)
    k, _ = sk.Kernel.from_legendre(g, ks.beam(), ks.lcut + 1, ks.lmax, ks.n_nodes, ks.theta_cut, ks.layout)
    return g, k


# DRAM traffic per launch from a committed ncu summary (profiles/<kernel>_<workload>.md),
# valid only while the kernel's sources hash to the value recorded at capture time.
PROFILED_SOURCES = {
    "conv_cap": ["cap.cu", "cap_common.cuh", "skconv_internal.cuh", "skconv_launch.h", "tc.cuh"],
    "conv_capw": ["capw.cu", "cap_common.cuh", "skconv_internal.cuh", "skconv_launch.h", "tc.cuh"],
    "conv_belt": ["belt.cu", "skconv_internal.cuh", "skconv_launch.h"],
    "conv_belt_tc": ["belt_tc.cu", "skconv_internal.cuh", "skconv_launch.h", "tc.cuh"],
}


def path_costs(prof, by_launch):
    """Measured cost of one pair on each ring path (0 belt, 1 cap, 2 per-pair, 3 cap with wide
    windows), ms per pair, from a profiled run's per-kernel times (each path's kernels with
    their set-up launches: the caps' symmetric copy)."""
    def per(names):
        return sum(prof[n][0] / prof[n][1] for n in names if n in prof)
    # the evaluating kernels' polar launch is a few blocks on a side stream, latency-bound
    # and overlapped with the rest: its time per pair says little about their share, so
    # there the caps' pairs (narrow and wide) and any per-pair rings take the narrow caps'
    # cost; the stored-weight launch sums both kinds of cap rings
    belt = per(("conv_belt_tc", "conv_belt_bf16", "conv_belt", "belt_weights"))
    cap = per(("conv_capw", "conv_cap", "cap_sym"))
    cap_pairs = by_launch[1] + (by_launch[2] if "conv_capw" in prof else 0)
    cb = belt / by_launch[0] if by_launch[0] else 0.0
    cc = cap / cap_pairs if cap_pairs else cb
    return [cb if cb > 0 else cc, cc, cc, cc]


def copy_floor(torch, hx, hy, reps):
    """The same bytes copied alone between the pinned host buffers and the device: host to
    device, device to host, and both at once on two streams (the floor an end-to-end call
    that overlaps its sums with the copies approaches), ms per step."""
    d = torch.empty(hx.shape, dtype=hx.dtype, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    out = {}
    for name in ("h2d", "d2h", "both"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            if name in ("h2d", "both"):
                with torch.cuda.stream(s1):
                    d.copy_(hx, non_blocking=True)
            if name in ("d2h", "both"):
                with torch.cuda.stream(s2):
                    hy.copy_(d, non_blocking=True)
        torch.cuda.synchronize()
        out[name] = (time.perf_counter() - t0) / reps * 1e3
    out["h2d_gbs"] = hx.numel() * hx.element_size() / out["h2d"] * 1e-6
    out["d2h_gbs"] = hy.numel() * hy.element_size() / out["d2h"] * 1e-6
    del d
    return out


def measured_hbm_gbs():
    """HBM copy bandwidth measured on the B300s (MEASURED_PEAKS.json), else the fallback."""
    here = os.path.dirname(os.path.abspath(__file__))
    try:
        return float(json.load(open(os.path.join(here, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured (copy)"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


def profiled_traffic(kernel, workload):
    import hashlib
    import re
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(here, "profiles", f"{kernel}_{workload}.md")
    if kernel not in PROFILED_SOURCES or not os.path.exists(path):
        return None
    text = open(path).read()
    mb = re.search(r"dram_bytes_per_launch:\s*(\d+)", text)
    mh = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    if not mb or not mh:
        return None
    h = hashlib.sha256()
    for f in PROFILED_SOURCES[kernel]:
        h.update(open(os.path.join(here, "paper_1211_3556_b300", "csrc", f), "rb").read())
    return int(mb.group(1)) if h.hexdigest() == mh.group(1) else None


def measure_peaks(ctx, gpu_index, seconds=2.0):
    """Measured FP32 (fma.rn.f32 and fma.rn.f32x2 chains) and TF32 (tcgen05.mma 128x256x8)
    rates of this GPU, each with the SM clock sampled while it ran, and the derived FP32
    figure (SM count from the device x 128 lanes x 2 flop x maximum SM clock)."""
    import paper_1211_3556_b300 as sk
    info = ctx.device_info()
    out = {"sms": info["sms"], "sm_clock_max_mhz": info["sm_clock_khz"] / 1e3,
           "fp32_derived_tflops": info["sms"] * LANES * 2 * info["sm_clock_khz"] * 1e3 / 1e12}
    for name, kind in (("ffma", sk.PEAK_FFMA), ("ffma2", sk.PEAK_FFMA2), ("tf32_tcgen05", sk.PEAK_TF32)):
        ctx.measure_peak(kind, 0.2)                       # warm-up
        smp = ClockSampler(gpu_index)
        r = ctx.measure_peak(kind, seconds)
        clk = smp.stop()
        out[name] = {"tflops": r, "sm_mhz": clk.get("sm_mhz"), "reasons": clk.get("reasons"),
                     "tflops_per_ghz": r / (clk["sm_mhz"] / 1e3) if clk.get("sm_mhz") else None}
    ctx.status()
    out["fp32_tflops"] = max(out["ffma"]["tflops"], out["ffma2"]["tflops"])
    return out


def time_steps(torch, fn, steps, warmup, barrier):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def cpu_baseline_leg(wl, group, y_gpu_first_map, target_s=40.0):
    """The FP64 oracle, as it stands, on a bounded random sample of output pixels of
    the same workload (all host cores); also the rms error of the GPU result on
    that sample against it."""
    import oracle as O
    ks = group.kernel
    V = O.tabulate_real_kernel(ks.beam(), ks.lcut, ks.lmax, ks.theta_cut, ks.n_nodes, ks.layout)
    x = make_maps(group, wl.sources[0] if wl.sources else None)[0].astype(np.float64)
    npx = npix_of(group.nside)
    n_probe = min(npx, 40000)
    probe = sample_indices(npx, n_probe, 9001)
    t0 = time.perf_counter()
    O.conv_window(group.nside, V, ks.theta_cut, ks.layout, x, probe)
    dt = max(time.perf_counter() - t0, 1e-3)
    n = int(min(npx, max(n_probe, n_probe * target_s / dt)))
    outs = sample_indices(npx, n, 9002)
    t0 = time.perf_counter()
    yo = O.conv_window(group.nside, V, ks.theta_cut, ks.layout, x, outs)
    dt = time.perf_counter() - t0
    pairs = O.count_pairs(group.nside, ks.theta_cut, outs)
    yg = y_gpu_first_map[outs].astype(np.float64)
    rms = float(np.linalg.norm(yg - yo) / np.linalg.norm(yo))
    # the same oracle on one core (the paper's comparisons assume a single CPU core), on a
    # smaller sample of about 5 s
    t1 = time.perf_counter()
    O.conv_window(group.nside, V, ks.theta_cut, ks.layout, x, probe[:2000], nthreads=1)
    d1 = max(time.perf_counter() - t1, 1e-3)
    n1 = int(min(npx, max(2000, 2000 * 5.0 / d1)))
    outs1 = sample_indices(npx, n1, 9003)
    t1 = time.perf_counter()
    O.conv_window(group.nside, V, ks.theta_cut, ks.layout, x, outs1, nthreads=1)
    d1 = time.perf_counter() - t1
    pairs1 = O.count_pairs(group.nside, ks.theta_cut, outs1)
    return {"value": pairs / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{n} random output pixels of map 0 ({pairs} pairs), FP64 windowed direct sum, "
                      f"{dt:.1f} s",
            "single_core": {"value": pairs1 / d1, "unit": UNIT, "cores": 1,
                            "sample": f"{n1} random output pixels of map 0 ({pairs1} pairs), {d1:.1f} s"}}, rms


def run_ours(args):
    import torch
    import paper_1211_3556_b300 as sk

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

        def barrier():
            dist.barrier()
    else:
        def barrier():
            pass

    wl = WORKLOADS[args.workload]
    ctx = sk.Context(local)
    ops = []
    for gi, group in enumerate(wl.groups):
        g, k = build_operator(sk, ctx, group)
        src = wl.sources[gi] if wl.sources and gi < len(wl.sources) else None
        maps = shard_maps(make_maps(group, src), rank, world)
        x = torch.from_numpy(maps).cuda()
        y = torch.empty_like(x)
        pairs = k.count_pairs()
        by_path = k.count_pairs_by_path()
        by_launch = k.count_pairs_by_launch()
        ops.append(dict(group=group, geom=g, kern=k, x=x, y=y, maps=maps, pairs=pairs, by_path=by_path,
                        by_launch=by_launch, cap_weight_bytes=k.cap_weight_bytes()))
    pairs_step = sum(o["pairs"] * o["group"].batch for o in ops)
    maps_step = sum(o["group"].batch for o in ops)
    # plan-time tuning of the belt tile width on the step's own maps (outside the timed region);
    # the choice is cached per GPU and workload in the temp directory, so that a repeated run of
    # the same command (e.g. under a profiler, whose serialisation distorts the trials) reuses it
    tune_cache = os.path.join(tempfile.gettempdir(), "skconv_belt_tiles.txt")
    belt_tiles = [o["kern"].autotune(o["x"], out=o["y"], cache_path=tune_cache) for o in ops]
    tuned = [o["kern"].config() for o in ops]          # belt form, tile width, cap weights kept
    for o in ops:
        o["cap_weight_bytes"] = o["kern"].cap_weight_bytes()

    if len(ops) == 1:
        o = ops[0]

        def step():
            sk.convolve(o["kern"], o["x"], out=o["y"])
    else:
        jobs = [(o["kern"], o["x"], o["y"]) for o in ops]

        def step():
            sk.convolve_jobs(ctx, jobs)

    # timed region: clocks sampled throughout, per-launch events recorded by the library
    step()
    torch.cuda.synchronize()
    ctx.status()
    sampler = ClockSampler(local)          # sampled from the warm-up to the end of the timed steps
    for _ in range(args.warmup):
        step()
    ctx.profile(True)
    ctx.profile_read()
    ms = time_steps(torch, step, args.steps, 0, barrier)
    clocks = sampler.stop()
    ctx.profile(False)
    prof = ctx.profile_read()
    ctx.status()
    ms = max_over_ranks(ms, world, "cuda")
    value = aggregate_rate(pairs_step, world, ms * 1e-3)
    launches = sum(c for _, c in prof.values())
    # the roofline's denominators, measured on this GPU after the timed region
    peaks = measure_peaks(ctx, local)
    fp32_peak = peaks["fp32_tflops"]

    # roofline of the dominant kernel: F_mac flops per pair of the outputs it evaluates
    dom = max(prof, key=lambda n: prof[n][0]) if prof else None
    # the pairs each launch sums (sk_count_pairs_by_launch: belt, caps with narrow windows,
    # caps with wide windows, per-pair rings); the stored-weight cap launch takes both kinds
    # of cap rings, the evaluating kernels one launch each (the wide one on a side stream)
    launch_idx = {"conv_belt": (0,), "conv_belt_tc": (0,), "conv_cap": (1,), "conv_capw": (1, 2),
                  "conv_cap_polar": (2,), "conv_general": (3,)}
    roofline = None
    if dom in launch_idx:
        dom_pairs = sum(sum(o["by_launch"][q] for q in launch_idx[dom]) * o["group"].batch for o in ops)
        launch_ms = prof[dom][0] / prof[dom][1]
        per_launch_pairs = dom_pairs * args.steps / prof[dom][1]
        achieved = FLOP_PER_PAIR * per_launch_pairs / (launch_ms * 1e-3) / 1e12
        if dom == "conv_belt_tc":
            # 3xTF32: three TF32 MMAs per useful product, so a third of the TF32 peak bounds it
            tf32 = peaks["tf32_tcgen05"]["tflops"]
            roofline = {"bound": "tensor", "kernel": dom, "achieved": achieved, "peak": tf32,
                        "unit": "TFLOP/s", "frac": achieved / tf32, "frac_of_3xtf32_ceiling": 3 * achieved / tf32,
                        "traffic": profiled_traffic(dom, args.workload),
                        "peak_source": "measured on this GPU in this run: tcgen05 TF32 MMA loop (sk_measure_peak)",
                        "flop_per_unit": FLOP_PER_PAIR, "unit_of_work": "in-cut pixel pair x map"}
        else:
            roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fp32_peak,
                        "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                        "traffic": profiled_traffic(dom, args.workload),
                        "peak_source": "measured on this GPU in this run: FP32 FMA chains (sk_measure_peak), "
                                       "SM clock %s MHz while it ran" % peaks["ffma2"]["sm_mhz"],
                        "frac_of_derived": achieved / peaks["fp32_derived_tflops"],
                        "flop_per_unit": FLOP_PER_PAIR, "unit_of_work": "in-cut pixel pair x map"}
        if roofline["traffic"]:
            # the same launch against the HBM roof: DRAM bytes of the committed ncu capture
            # (cold-cache, per launch) over this run's launch time
            gbs = roofline["traffic"] / (launch_ms * 1e-3) / 1e9
            hbm, src = measured_hbm_gbs()
            roofline["dram_gbs"] = gbs
            roofline["dram_frac"] = gbs / hbm
            roofline["dram_peak_gbs"] = hbm
            roofline["dram_peak_source"] = src

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if len(ops) == 1:
        o = ops[0]
        hx = torch.from_numpy(o["maps"]).pin_memory()
        hy = torch.empty_like(hx).pin_memory()
        hxn, hyn = hx.numpy(), hy.numpy()
        sk.convolve_host(o["kern"], hxn, hyn)
        k_e2e = max(3, min(args.steps, 10))
        barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            sk.convolve_host(o["kern"], hxn, hyn)
        t_e2e = (time.perf_counter() - t0) / k_e2e
        t_e2e = max_over_ranks(t_e2e, world, "cuda")
        nbytes = int(o["maps"].nbytes)
        e2e = {"value": aggregate_rate(pairs_step, world, t_e2e), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "ms_per_step": t_e2e * 1e3, "steps": k_e2e,
               "api": "sk_convolve_host (pinned host buffers)",
               "copy_floor_ms": copy_floor(torch, hx, hy, k_e2e)}
        del hx, hy

    # the batched forms beside the plain one (64 maps at Nside 1024 sharing one kernel):
    # FP32 (weights shared by the batch) and tensor cores (3xTF32 tcgen05 belt)
    batched = None
    if not args.no_batched and args.workload == "n2048_plain":
        grp = WORKLOADS["n1024x64_batched"].groups[0]
        gb, kb = build_operator(sk, ctx, grp)
        xb = torch.from_numpy(make_maps(grp)).cuda()
        yb = torch.empty_like(xb)
        pb = kb.count_pairs()
        kb.autotune(xb, out=yb, cache_path=os.path.join(tempfile.gettempdir(), "skconv_belt_tiles.txt"))
        batched = {"workload": "n1024x64_batched", "unit": UNIT}
        outs_b = {}
        for name, path in (("fp32", sk.PATH_FP32), ("tensor_3xtf32", sk.PATH_TENSOR),
                           ("tensor_bf16x3", sk.PATH_BF16X3)):
            msb = time_steps(torch, lambda: sk.convolve(kb, xb, out=yb, path=path), max(3, min(args.steps, 20)), 2,
                             barrier)
            batched[name] = {"value": pb * grp.batch / (msb * 1e-3), "ms_per_map": msb / grp.batch,
                             "ms_per_step": msb}
            outs_b[name] = yb[:4].clone()
        # BF16x3 is outside the 1e-6 bound: its deviation from the 3xTF32 form (itself within
        # 4e-7 of the FP64 oracle in the tests) is reported beside it and flagged
        ref_b = outs_b["tensor_3xtf32"].double()
        batched["tensor_bf16x3"]["rms_rel_vs_3xtf32"] = float(torch.linalg.norm(outs_b["tensor_bf16x3"].double() - ref_b)
                                                              / torch.linalg.norm(ref_b))
        batched["tensor_bf16x3"]["within_1e-6"] = batched["tensor_bf16x3"]["rms_rel_vs_3xtf32"] <= 1e-6
        for name in ("fp32", "tensor_3xtf32", "tensor_bf16x3"):
            useful = FLOP_PER_PAIR * batched[name]["value"] / 1e12
            batched[name]["useful_tflops"] = useful
            batched[name]["frac_fp32_peak"] = useful / fp32_peak
        # the tensor form's useful flops against the TF32 tensor peak (3xTF32 issues three
        # MMAs per useful product, so 1/3 is its ceiling)
        batched["tensor_3xtf32"]["frac_tf32_peak"] = (batched["tensor_3xtf32"]["useful_tflops"]
                                                      / peaks["tf32_tcgen05"]["tflops"])
        batched["value"] = max(batched["fp32"]["value"], batched["tensor_3xtf32"]["value"])   # the 1e-6 forms
        del xb, yb

    # the whole split of Eq. 1 beside the real-space step: harmonic part K^_l = K_l - R_l
    # (l <= l_cut) by the library's ring transform, timed alone and added to the real-space sum
    split = None
    if not args.no_split and args.workload == "n2048_plain" and len(ops) == 1:
        o = ops[0]
        ks = o["group"].kernel
        R = sk.kernel_response(o["kern"], ks.lcut)
        kh = ks.beam()[: ks.lcut + 1] - R
        t0 = time.perf_counter()
        h = sk.Harmonic(ctx, o["geom"], kh, ks.lcut)
        torch.cuda.synchronize()
        t_create = time.perf_counter() - t0
        yh = torch.empty_like(o["x"])
        ns = max(3, min(args.steps, 10))
        ms_h = time_steps(torch, lambda: h.apply(o["x"], out=yh), ns, 2, barrier)
        ms_s = time_steps(torch, lambda: sk.split_convolve(o["kern"], h, o["x"], out=yh), ns, 2, barrier)
        # Eq. 2's error of this split (the high-pass-and-truncate table of the workload) and of
        # the least-squares real-space part on the same cut, both relative to K_l up to 2 l_max
        lfit = 2 * ks.lmax
        kl2 = gaussian_beam_of(ks, lfit)
        R2 = sk.kernel_response(o["kern"], lfit)
        ell = np.arange(lfit + 1)
        sig_trunc = math.sqrt(float(np.sum((2 * ell[ks.lcut + 1:] + 1) * (R2[ks.lcut + 1:] - kl2[ks.lcut + 1:]) ** 2))
                              / float(np.sum((2 * ell + 1) * kl2 ** 2)))
        _, sig_fit = sk.fit_real_kernel(ctx, kl2, ks.lcut, ks.theta_cut, n_basis=257, lfit=lfit)
        split = {"l_cut": ks.lcut, "harmonic_ms_per_map": ms_h, "split_ms_per_map": ms_s,
                 "real_space_ms_per_map": ms / maps_step, "lambda_table_gb": h.table_bytes() / 1e9,
                 "harmonic_setup_s": t_create, "sigma_rms_eq2_table": sig_trunc,
                 "sigma_rms_eq2_least_squares": sig_fit}
        del h, yh

    # wide cut (300' at Nside 1024): the equatorial-zone rings by the ring-pair Fourier form
    # against the direct sums (per-pair there: the belt kernel's stages do not fit such windows)
    fourier = None
    if not args.no_fourier and args.workload == "n2048_plain":
        grp = WORKLOADS["n1024_wide"].groups[0]
        gw, kw = build_operator(sk, ctx, grp)
        t0 = time.perf_counter()
        fw = sk.FourierBelt(kw)
        torch.cuda.synchronize()
        t_create = time.perf_counter() - t0
        xw = torch.from_numpy(make_maps(grp)).cuda()
        yf, yd = torch.empty_like(xw), torch.empty_like(xw)
        nw = max(3, min(args.steps, 5))
        ctx.profile(True)
        ctx.profile_read()
        ms_f = time_steps(torch, lambda: fw.apply(xw, out=yf), nw, 1, barrier)
        pf = ctx.profile_read()
        ms_d = time_steps(torch, lambda: sk.convolve(kw, xw, out=yd), nw, 1, barrier)
        pd = ctx.profile_read()
        ctx.profile(False)
        info = fw.info()
        n_, st_, _, _, _ = gw.rings()
        r0, r1 = info["first_ring"], info["first_ring"] + info["rings"]
        zs = slice(int(st_[r0]), int(st_[r1 - 1] + n_[r1 - 1]))
        a = yf[0, zs].double()
        b = yd[0, zs].double()
        per = lambda p, names: sum(p[n][0] for n in names if n in p) / nw
        fourier = {"workload": "n1024_wide", "theta_cut_arcmin": grp.kernel.theta_cut_arcmin,
                   "zone_rings": info["rings"], "ring_offsets_H": info["H"], "G_gb": info["bytes"] / 1e9,
                   "create_s": t_create, "ms_per_map_fourier_operator": ms_f, "ms_per_map_direct_operator": ms_d,
                   "zone_ms_fourier": per(pf, ("fourier_fft", "fourier_mix")),
                   "zone_ms_direct_per_pair": per(pd, ("conv_general",)),
                   "zone_rms_rel_fourier_vs_direct": float(torch.linalg.norm(a - b) / torch.linalg.norm(b))}
        del fw, xw, yf, yd

    # gradients (16 maps at Nside 1024, 30'): the forward sums, the adjoint (the same gather: the
    # operator is symmetric) and the table gradient (per pair, FP64 node coordinates)
    grad = None
    if not args.no_grad and args.workload == "n2048_plain":
        grp = WORKLOADS["n1024x16_grad"].groups[0]
        gg, kg = build_operator(sk, ctx, grp)
        xg = torch.from_numpy(make_maps(grp)).cuda()
        gy = torch.from_numpy(make_maps(Group(grp.nside, grp.batch, grp.kernel, grp.seed + 1))).cuda()
        yg, gx = torch.empty_like(xg), torch.empty_like(xg)
        gt = torch.empty(kg.n_nodes, device="cuda")
        # the forward and adjoint run the operator's settings tuned on these maps, as the
        # step's own operator does (the table gradient's kernels do not depend on them)
        kg.autotune(xg, out=yg, cache_path=os.path.join(tempfile.gettempdir(), "skconv_belt_tiles.txt"))
        pg = kg.count_pairs() * grp.batch
        ng = max(3, min(args.steps, 5))
        ms_fwd = time_steps(torch, lambda: sk.convolve(kg, xg, out=yg), ng, 1, barrier)
        ms_adj = time_steps(torch, lambda: sk.convolve_adjoint(kg, gy, out=gx), ng, 1, barrier)
        ms_tab = time_steps(torch, lambda: sk.grad_table(kg, xg, gy, out=gt), ng, 1, barrier)
        # the allocation-free entry point (per-pixel gradient kernel on every ring)
        import ctypes
        L = sk.lib()
        strm = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

        def noalloc():
            rc = L.sk_grad_table_noalloc(ctx._h, kg._h, ctypes.c_void_p(xg.data_ptr()), ctypes.c_void_p(gy.data_ptr()),
                                         grp.batch, xg.stride(0), ctypes.c_void_p(gt.data_ptr()), strm)
            assert rc == 0, L.sk_last_error()
        ms_noalloc = time_steps(torch, noalloc, 1, 1, barrier)
        grad = {"workload": "n1024x16_grad", "unit": UNIT, "maps": grp.batch, "tuned": kg.config(),
                "forward": {"ms_per_step": ms_fwd, "value": pg / (ms_fwd * 1e-3)},
                "adjoint": {"ms_per_step": ms_adj, "value": pg / (ms_adj * 1e-3)},
                "table_gradient": {"ms_per_step": ms_tab, "value": pg / (ms_tab * 1e-3)},
                "table_gradient_noalloc": {"ms_per_step": ms_noalloc, "value": pg / (ms_noalloc * 1e-3)},
                "step_ms": ms_fwd + ms_adj + ms_tab}
        del xg, gy, yg, gx

    # ring bands of the step's map (the decomposition of one map over several GPUs), run one
    # band after another on this GPU: each band's time is what its rank would take, so
    # full / (ranks x slowest band) bounds the strong-scaling efficiency of the sums; bands of
    # a northern range and its mirror, balanced by estimated cost (symmetric_bands)
    bands = None
    if not args.no_bands and args.workload == "n2048_plain" and world == 1:
        from paper_1211_3556_b300.bands import ring_costs, symmetric_bands
        o = ops[0]
        grp = o["group"]
        xb = o["x"][:1]
        yb = torch.empty_like(xb)
        nb_steps = max(3, min(args.steps, 10))
        full = time_steps(torch, lambda: sk.convolve(o["kern"], xb, out=yb), nb_steps, 1, barrier)
        # bands balanced by each ring's pairs times the measured cost of a pair on its path
        costs = path_costs(prof, o["by_launch"])
        rpairs, rpath = o["kern"].pairs_by_ring()
        rcost = ring_costs(rpairs, rpath, costs)
        bands = {"workload": args.workload, "decomposition": "symmetric_bands weighted by pairs x measured "
                 "per-path pair cost", "path_cost_ns_per_pair": [c * 1e6 for c in costs],
                 "ms_full_map": full, "ranks": {}}
        for nrk in (2, 4, 8):
            per = []
            for b in symmetric_bands(grp.nside, grp.kernel.theta_cut, nrk, ring_cost=rcost):
                lo, hi = b.north
                if hi > lo:
                    per.append(time_steps(torch, lambda: sk.convolve_rings_sym(o["kern"], xb, lo, hi, out=yb),
                                          nb_steps, 1, barrier))
            bands["ranks"][str(nrk)] = {"ms_per_band": per, "ms_slowest": max(per),
                                        "ms_spread": max(per) - min(per),
                                        "efficiency_bound": full / (nrk * max(per))}
        del xb, yb

    # a partial-sky field at Nside 8192 (5'): re-oriented onto the polar cap, its cap rings
    # summed, rotated back; against the full-sky operator of the same kernel
    field = None
    if not args.no_field and args.workload == "n2048_plain":
        from inputs import FIELD_CENTRE, FIELD_RADIUS_DEG
        grp = WORKLOADS["n8192_field"].groups[0]
        t0 = time.perf_counter()
        gf, kf = build_operator(sk, ctx, grp)
        t_build = time.perf_counter() - t0
        t0 = time.perf_counter()
        patch = sk.PolarPatch(kf, FIELD_CENTRE[0], FIELD_CENTRE[1], math.radians(FIELD_RADIUS_DEG))
        torch.cuda.synchronize()
        t_plan = time.perf_counter() - t0
        xf = torch.from_numpy(make_maps(grp)).cuda()
        yf = torch.zeros_like(xf)
        xr, yr = torch.zeros_like(xf), torch.empty_like(xf)
        nf = max(3, min(args.steps, 10))
        nr = 4 * grp.nside - 1
        ms_in = time_steps(torch, lambda: patch.to_cap.apply(xf, out=xr), nf, 1, barrier)
        ms_cap = time_steps(torch, lambda: sk.convolve_rings(kf, xr, 0, patch.out_hi, out=yr), nf, 1, barrier)
        ms_out = time_steps(torch, lambda: patch.to_sky.apply(yr, out=yf), nf, 1, barrier)
        ms_patch = time_steps(torch, lambda: patch.convolve(xf, out=yf, work=(xr, yr)), nf, 1, barrier)
        ms_search = time_steps(torch, lambda: sk.resample(gf, xf, patch.rot, 0, patch.in_hi, out=xr), 3, 1, barrier)
        ms_full = time_steps(torch, lambda: sk.convolve(kf, xf, out=yr), 3, 1, barrier)
        n_, st_, _, _, _ = gf.rings()
        field = {"workload": "n8192_field", "theta_cut_arcmin": grp.kernel.theta_cut_arcmin,
                 "centre_rad": list(FIELD_CENTRE), "radius_deg": FIELD_RADIUS_DEG,
                 "area_sq_deg": 2 * math.pi * (1 - math.cos(math.radians(FIELD_RADIUS_DEG))) * (180 / math.pi) ** 2,
                 "cap_rings_out": patch.out_hi, "cap_rings_in": patch.in_hi, "rings": nr,
                 "cap_pixels_out": int(st_[patch.out_hi]), "sky_rings": [patch.sky_lo, patch.sky_hi],
                 "ms_field": ms_patch, "ms_rotate_in": ms_in, "ms_cap_sums": ms_cap, "ms_rotate_back": ms_out,
                 "ms_full_sky_operator": ms_full, "build_s": t_build, "plans_s": t_plan,
                 "plan_pairs": [patch.to_cap.info()["pairs"], patch.to_sky.info()["pairs"]],
                 "ms_rotate_in_unplanned": ms_search,
                 "data": "white-noise map over the whole sphere (only the field is read)"}
        del xf, yf, xr, yr, patch, kf, gf

    o0 = ops[0]
    y0 = o0["y"][0].cpu().numpy()
    cpu_baseline, rms = None, None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu_baseline, rms = cpu_baseline_leg(wl, o0["group"], y0)

    if rank == 0:
        ks = o0["group"].kernel
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "ms_per_map": ms / maps_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "nside": [o["group"].nside for o in ops],
                       "maps_per_gpu": maps_step, "theta_cut_arcmin": ks.theta_cut_arcmin,
                       "n_nodes": ks.n_nodes, "fwhm_arcmin": ks.fwhm_arcmin, "lmax": ks.lmax, "lcut": ks.lcut,
                       "pairs_per_step_per_gpu": pairs_step,
                       "l2": "inputs larger than L2 (map bytes %d > 126 MB)" % int(sum(o["maps"].nbytes for o in ops)),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "belt_tile": belt_tiles, "tuned": tuned},
            "rms_rel_vs_fp64": rms,
            "f_eval": value / world * FLOP_PER_PAIR_EVAL / (fp32_peak * 1e12),
            "f_mac": value / world * FLOP_PER_PAIR / (fp32_peak * 1e12),
            "peaks": peaks,
            "roofline": roofline,
            "kernels": {n: {"ms_total": t, "launches": c, "ms_per_launch": t / c} for n, (t, c) in prof.items()},
            "gpu_launches": launches,
            "pairs_by_path": {"belt": o0["by_path"][0], "cap": o0["by_path"][1], "general": o0["by_path"][2]},
            "pairs_by_launch": dict(zip(("belt", "cap_narrow", "cap_wide", "general"), o0["by_launch"])),
            "cap_weight_bytes": [o["cap_weight_bytes"] for o in ops],
            "clocks": clocks,
            "e2e": e2e,
            "batched": batched,
            "split": split,
            "fourier": fourier,
            "grad": grad,
            "field": field,
            "bands": bands,
            "cpu_baseline": cpu_baseline,
            "context": "paper: GTX 480 + 1 Core2 core, split convolution >10x faster than a full "
                       "single-core SHT convolution (eq. 3 model: 2.89 s at theta_cut 20')",
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# --------------------------------------------------------------------------

def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle as O
    wl = WORKLOADS[args.workload]
    group = wl.groups[0]
    ks = group.kernel
    V = O.tabulate_real_kernel(ks.beam(), ks.lcut, ks.lmax, ks.theta_cut, ks.n_nodes, ks.layout)
    x = make_maps(group, wl.sources[0] if wl.sources else None)[0].astype(np.float64)
    npx = npix_of(group.nside)
    probe = sample_indices(npx, 1000, 8001)
    t0 = time.perf_counter()
    O.conv_window(group.nside, V, ks.theta_cut, ks.layout, x, probe)
    dt = max(time.perf_counter() - t0, 1e-3)
    per_step_s = max(0.2, 150.0 / (args.steps + args.warmup))   # whole run about 150 s of oracle work
    n = int(min(npx, max(1000, 1000 * per_step_s / dt)))
    samples = [sample_indices(npx, n, 8100 + s) for s in range(args.warmup + args.steps)]
    for s in range(args.warmup):
        O.conv_window(group.nside, V, ks.theta_cut, ks.layout, x, samples[s])
    pairs = 0
    tt = 0.0
    for s in range(args.warmup, args.warmup + args.steps):
        t0 = time.perf_counter()
        O.conv_window(group.nside, V, ks.theta_cut, ks.layout, x, samples[s])
        tt += time.perf_counter() - t0
        pairs += O.count_pairs(group.nside, ks.theta_cut, samples[s])
    value = pairs / tt
    cores = O.num_threads()
    sample = f"{n} random output pixels per step of map 0, FP64 windowed direct sum"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "nside": [group.nside], "theta_cut_arcmin": ks.theta_cut_arcmin,
                   "n_nodes": ks.n_nodes},
        "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": cores, "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_bands(args):
    """One map over the ranks in symmetric ring bands: every step each rank receives the
    halo pixels its band reads from the ranks that own them (point-to-point) and sums its
    band (strong scaling: the map is the same at every rank count)."""
    import torch
    import paper_1211_3556_b300 as sk
    from paper_1211_3556_b300.bands import exchange_halo, ring_costs, symmetric_bands

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

        def barrier():
            dist.barrier()
    else:
        def barrier():
            pass
    wl = WORKLOADS[args.workload]
    group = wl.groups[0]
    ks = group.kernel
    ctx = sk.Context(local)
    g, k = build_operator(sk, ctx, group)
    maps = make_maps(group, wl.sources[0] if wl.sources else None)[:1]
    npix = maps.shape[1]
    # band edges from each ring's pairs times the measured cost of a pair on its path, the
    # costs measured on rank 0 and sent to every rank (all ranks must cut the same bands)
    x1 = torch.from_numpy(maps).cuda()
    y1 = torch.empty_like(x1)
    k.autotune(x1, out=y1, cache_path=os.path.join(tempfile.gettempdir(), "skconv_belt_tiles.txt"))
    ctx.profile(True)
    ctx.profile_read()
    for _ in range(3):
        sk.convolve(k, x1, out=y1)
    torch.cuda.synchronize()
    costs = torch.tensor(path_costs(ctx.profile_read(), k.count_pairs_by_launch()), dtype=torch.float64,
                         device="cuda")
    ctx.profile(False)
    if world > 1:
        dist.broadcast(costs, src=0)
    del x1, y1
    rpairs, rpath = k.pairs_by_ring()
    bands = symmetric_bands(group.nside, ks.theta_cut, world, ring_cost=ring_costs(rpairs, rpath, costs.cpu().numpy()))
    me = bands[rank]
    own = np.concatenate([maps[:, q0:q1] for q0, q1 in me.out_pix], axis=1) if me.out_pix else maps[:, :0]
    x_own = torch.from_numpy(np.ascontiguousarray(own)).cuda()
    x_full = torch.zeros(1, npix, device="cuda")
    y = torch.empty_like(x_full)
    lo, hi = me.north
    stats = {}

    def step():
        exchange_halo(x_own, me, bands, npix, out=x_full, stats=stats)
        if hi > lo:
            sk.convolve_rings_sym(k, x_full, lo, hi, out=y)

    sampler = ClockSampler(local)
    ms = time_steps(torch, step, args.steps, args.warmup, barrier)
    clocks = sampler.stop()
    ctx.status()
    ms = max_over_ranks(ms, world, "cuda")
    pairs = k.count_pairs()
    if rank == 0:
        line = {"metric": METRIC, "value": pairs / (ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "ms_per_map": ms, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "nside": [group.nside], "maps_per_step": 1,
                           "theta_cut_arcmin": ks.theta_cut_arcmin, "decomposition": "symmetric ring bands",
                           "parallelism": f"ring bands x{world}", "pairs_per_step": pairs,
                           "band_balance": "pairs x measured per-path pair cost"},
                "halo_bytes_recv_rank0": stats.get("recv_bytes", 0), "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_errors(args):
    """Two settings of the study: the paper's (l_max = 2 Nside) and one with the band
    limit four times below the pixel scale (l_max = Nside / 2, the beam scaled with it)."""
    out = [split_error_study(1024, 2047, 14.0, 240.0, (256, 512, 768, 1024, 1280)),
           split_error_study(1024, 511, 56.0, 240.0, (64, 128, 192, 256, 320))]
    print(json.dumps({"study": "split errors (Sec. 3)", "settings": out}), flush=True)


def split_error_study(nside, lmax, fwhm, tc_arcmin, lcuts, alpha=5.0):
    """The split's errors as the paper studies them (Sec. 3, Eq. 2 and the relative-error
    curve sigma_l = log10|1 - K~_l / K_l|), e.g. at Nside 1024 with l_max = 2047 (the paper's
    7' beam at l_max 4096 scaled to half the resolution: FWHM 14'), C_l = 1, theta_cut 240'.
    For each l_cut: the real-space part fitted by least squares, K^_l = K_l - R_l below l_cut;
    a white-noise map band-limited to l_max convolved with the full l-space kernel (the
    library's ring transform up to l_max) and with the split (harmonic part + real-space
    sums); the map rms error,
    the power spectra of both maps and their relative error per l, the spectrum rms error,
    and Eq. 2's estimate with alpha = 5."""
    import torch
    import paper_1211_3556_b300 as sk
    from inputs import gaussian_beam, white_noise_maps
    torch.cuda.set_device(0)
    ctx = sk.Context(0)
    g = sk.Geometry(ctx, nside)
    kl = gaussian_beam(fwhm, lmax)
    ell = np.arange(lmax + 1)
    tc = tc_arcmin * ARCMIN
    # the input: white noise band-limited to l_max (C_l flat up to l_max, nothing above: the
    # paper gives the input spectrum and the kernel the same band limit), made by the
    # library's transform with K_l = 1
    h_one = sk.Harmonic(ctx, g, np.ones(lmax + 1), lmax)
    x = h_one.apply(torch.from_numpy(white_noise_maps(nside, 1, 901)).cuda())
    del h_one
    t0 = time.perf_counter()
    h_full = sk.Harmonic(ctx, g, kl, lmax)
    y_full = h_full.apply(x)
    c_full = h_full.spectrum(y_full)[0].cpu().numpy()
    torch.cuda.synchronize()
    t_full = time.perf_counter() - t0
    edges = np.unique(np.round(np.geomspace(2, lmax + 1, 25)).astype(int))

    def binned(v):
        out = []
        for a, b in zip(edges[:-1], edges[1:]):
            seg = v[a:b]
            seg = seg[np.isfinite(seg)]
            out.append(float(np.median(seg)) if len(seg) else None)
        return out

    rows = []
    for lcut in lcuts:
        V, sig_fit = sk.fit_real_kernel(ctx, kl, lcut, tc, n_basis=513, nt_out=8193, lfit=lmax)
        k = sk.Kernel(g, V, tc)
        R = sk.kernel_response(k, lmax)
        khat = kl[: lcut + 1] - R[: lcut + 1]
        k_tilde = R.copy()
        k_tilde[: lcut + 1] += khat                       # K~_l = K^_l + R_l
        with np.errstate(divide="ignore"):
            sigma_l = np.log10(np.abs(1.0 - k_tilde / kl))
        srms2 = np.sum((2 * ell + 1) * (k_tilde - kl) ** 2) / (4 * math.pi)
        est = alpha * math.sqrt(srms2 / (np.sum((2 * ell + 1) * kl ** 2) / (4 * math.pi)))
        h = sk.Harmonic(ctx, g, khat, lcut)
        y = sk.convolve(k, x)
        # the real-space part's pixel sum against the harmonic convolution with its response
        # R_l on the same band-limited map: the quadrature error of the pixel sum
        h_r = sk.Harmonic(ctx, g, R, lmax)
        y_rc = h_r.apply(x)
        quad = float(torch.linalg.norm((y - y_rc).double()) / torch.linalg.norm(y_full.double()))
        del h_r, y_rc
        h.apply(x, out=y, accumulate=True)                # the split: real-space + harmonic parts
        c_split = h_full.spectrum(y)[0].cpu().numpy()
        map_rms = float(torch.linalg.norm((y - y_full).double()) / torch.linalg.norm(y_full.double()))
        spec_err = c_split / c_full - 1.0
        spec_rms = math.sqrt(float(np.sum((2 * ell + 1) * (c_split - c_full) ** 2) /
                                   np.sum((2 * ell + 1) * c_full ** 2)))
        rows.append({"l_cut": lcut, "sigma_rms_fit": sig_fit, "estimate_eq2_alpha5": est,
                     "map_rms_error": map_rms, "spectrum_rms_error": spec_rms,
                     "real_space_quadrature_rms": quad,
                     "sigma_l_estimated_binned": binned(sigma_l),
                     "spectrum_rel_error_binned": binned(np.abs(spec_err)),
                     "cap_weight_bytes": k.cap_weight_bytes()})
        del k, h, y
        torch.cuda.synchronize()
    ctx.status()
    return {"nside": nside, "lmax": lmax, "fwhm_arcmin": fwhm, "theta_cut_arcmin": tc_arcmin, "alpha": alpha,
            "l_bins": edges.tolist(), "full_kernel_setup_and_apply_s": t_full, "rows": rows,
            "data": "white noise band-limited to l_max (C_l flat, the paper's uniform-noise input)"}


def run_table1(args):
    """Sec. 4, Table 1's optimum split for a 7' beam at Planck resolution: the real-space
    part of Eq. 1 (theta_cut 390') by the ring-pair Fourier form on the equatorial zone and the
    direct sums elsewhere, the harmonic part (K^_l = K_l - R_l, l <= 1158) by the library's
    ring transform; one map (its accuracy against the oracle: tests/test_fourier.py)."""
    import torch
    import paper_1211_3556_b300 as sk
    torch.cuda.set_device(0)
    grp = WORKLOADS["n2048_table1"].groups[0]
    ks = grp.kernel
    ctx = sk.Context(0)
    t0 = time.perf_counter()
    g = sk.Geometry(ctx, grp.nside)
    k, V = sk.Kernel.from_legendre(g, ks.beam(), ks.lcut + 1, ks.lmax, ks.n_nodes, ks.theta_cut, ks.layout)
    fw = sk.FourierBelt(k)
    torch.cuda.synchronize()
    t_real_setup = time.perf_counter() - t0
    x = torch.from_numpy(make_maps(grp)).cuda()
    y = torch.empty_like(x)
    ms_real = time_steps(torch, lambda: fw.apply(x, out=y), max(1, min(args.steps, 3)), 1, lambda: None)
    t0 = time.perf_counter()
    R = sk.kernel_response(k, ks.lcut)
    h = sk.Harmonic(ctx, g, ks.beam()[: ks.lcut + 1] - R, ks.lcut)
    torch.cuda.synchronize()
    t_harm_setup = time.perf_counter() - t0
    yh = torch.empty_like(x)
    ms_harm = time_steps(torch, lambda: h.apply(x, out=yh), max(3, min(args.steps, 5)), 1, lambda: None)
    ctx.status()
    info = fw.info()
    line = {"mode": "table1", "workload": "n2048_table1", "nside": grp.nside, "fwhm_arcmin": ks.fwhm_arcmin,
            "lmax": ks.lmax, "lcut": ks.lcut, "theta_cut_arcmin": ks.theta_cut_arcmin, "n_nodes": ks.n_nodes,
            "pairs_per_map": k.count_pairs(), "ms_real_space": ms_real, "ms_harmonic": ms_harm,
            "ms_split_total": ms_real + ms_harm, "real_setup_s": t_real_setup, "harmonic_setup_s": t_harm_setup,
            "zone_rings": info["rings"], "G_gb": info["bytes"] / 1e9, "cap_weight_bytes": k.cap_weight_bytes(),
            "data": "synthetic white-noise map",
            "context": "paper (Sec. 4): about 12 s per convolution at its optimum splits, against 160 s for "
                       "the whole kernel by a CPU SHT"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.errors:
        run_errors(args)
    elif args.table1:
        run_table1(args)
    elif args.bands:
        run_bands(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
