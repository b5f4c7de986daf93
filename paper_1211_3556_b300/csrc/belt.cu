// belt.cu -- equatorial-belt path: the convolution as a ring-wise Toeplitz sum.
//
// In the belt every ring has n = 4 Nside pixels, so for output pixel j of ring
// o and input pixel j + e of ring i the phi difference is pi (2e + s_i - s_o)/n:
// the pair weight dOmega K_lin(gamma) depends on (o, i, e) only, not on j.  A
// pre-pass evaluates those weight rows once per call (per-pair formula of the
// general path, FP32, exact half-angle); the main kernel is then a register-
// blocked 1-D correlation along each ring, one FMA per pair of its window.
// Same operator as the per-pair path (the real-space convolution of Sec. 2,
// Eq. 1 with the tabulated kernel of Sec. 3); only the order of work differs.
//
// Main kernel block: SK_BELT_G consecutive output rings, the same 32 P-pixel
// segment of each, computed by SK_BELT_G / 2 consumer warps (two rings each)
// plus one producer warp.  The producer streams, per input ring of the group,
// the segment's strip of that ring together with the weight rows the eight
// warps apply to it, into shared memory with 1-D TMA bulk copies
// (cp.async.bulk, 16-byte aligned pieces, the strip split where it wraps past
// phi = 2 pi) through SK_BELT_STAGES slots guarded by full/empty mbarriers.
// Weight rows are stored as ring pairs, (w of ring 2w, w of ring 2w+1) per
// offset, on one offset grid for all rings, so a lane applies both with one
// paired FMA (fma.rn.f32x2, two IEEE FMAs) to the same strip value: lane l
// owns outputs l P .. l P + P-1 of both rings (P odd: the lanes' strip reads
// hit 32 distinct banks) and slides 4 offsets at a time over a ring of strip
// values held in registers, loading 4 new values per step.
#include <algorithm>

#include "skconv.h"
#include "skconv_internal.cuh"
#include "skconv_launch.h"

namespace {

// G below: SK_BELT_G, the output rings of a group
constexpr int S = SK_BELT_STAGES;
// Shared-memory header: full[S], empty[S] and the weight barrier (8 bytes each),
// then the abort flag; the weight rows start at HDR (a multiple of 128 bytes).
constexpr int HDR = ((8 * (2 * S + 1) + 4 + 127) / 128) * 128;
static_assert(8 * (2 * S + 1) + 4 <= HDR, "belt header overlaps the weight rows");

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait on an mbarrier phase: gives up after ~2 s of wall time or when
// another thread of the block has given up, recording SK_ETIMEOUT.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *status) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > 2000000000ull) {
            *abort_flag = 1;
            sk_record_error(status, SK_ETIMEOUT);
            return false;
        }
    }
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Weight rows as ring pairs, in the order the main kernel streams them: for
// group grp, strip si (input ring i = bgrp[grp].x + si) and consumer warp w,
// with (o, nch) = bpr of that row, element c < 4 nch holds the weights at offset
// e = EMIN + o + c of output rings b_lo + grp G + 2w and + 1 against ring i,
// zero outside a row's window (or where ring i is not in that output ring's
// window list) and past 4 nch.  One thread per element.  With `gate`, nothing is
// written unless *gate is set (the table did not change: the stored rows stand).
__global__ void k_belt_pairs(const JobDesc J, int g0, int g1, float2 *w, const int *gate, bool w64) {
    constexpr int NW = SK_BELT_WARPS;
    if (gate && !*gate) return;
    const long long base = (long long)g0 * J.smax * NW * J.WPM;
    const long long n = (long long)g1 * J.smax * NW * J.WPM;
    const double half_step = SK_PI / (2.0 * (double)J.n4);
    for (long long idx = base + (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(idx % J.WPM);
        long long rest = idx / J.WPM;
        const int wp = (int)(rest % NW);
        rest /= NW;
        const int si = (int)(rest % J.smax);
        const int grp = (int)(rest / J.smax);
        const int2 gr = J.bgrp[grp];
        const int i = gr.x + si;
        const int2 on = J.bpr[rest * NW + wp];
        const int e = J.EMIN + on.x + c;
        float v[2] = {0.0f, 0.0f};
        if (i <= gr.y && c < 4 * on.y) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int rb = grp * SK_BELT_G + 2 * wp + q;
                if (rb >= J.nb) continue;
                const int ro = J.b_lo + rb;
                const int p0 = J.pair_off[ro], p1 = J.pair_off[ro + 1];
                const int p = p0 + (i - J.pairs[p0].ri);
                if (p < p0 || p >= p1) continue;
                const PairInfo P = J.pairs[p];
                const int s_o = J.rings[ro].s;
                const int ec = (s_o + 1 - P.s_i) >> 1;
                if (e < ec - P.W || e > ec + P.W) continue;
                const double xd = (double)(2 * e + P.s_i - s_o) * half_step;
                if (w64) {
                    const double2 ab = J.ab64[p];
                    v[q] = pair_weight64(xd, ab.x, ab.y, J.kp, J.kd, J.V64, J.dOmega);
                } else {
                    v[q] = pair_weight((float)xd, P.A, P.B, J.kp, J.tab);
                }
            }
        }
        w[idx] = make_float2(v[0], v[1]);
    }
}

// Consumer warp w owns output rings b_lo + grp*G + 2w and + 2w + 1; lane l owns
// pixels j0 + l P .. j0 + l P + P-1 of both.  Stage slot s holds the strip of
// input ring gr.x + si at offsets e = EMIN + m (pixel j + e of the strip is
// xs[l P + (e - EMIN) + k]; 4 values past the last offset, so that a row's
// last 4-offset chunk reads loaded values), then the eight warps' pair rows of
// that ring, then their (start, chunks).  Warps meet only at the stage
// barriers: no block-wide barrier between work items.
// BLK (operators whose outputs sum thousands of terms): each strip's contribution is
// summed apart and added to the output's total after the strip, so that the FP32
// rounding grows with the terms of one input ring and the number of rings, not with
// their product (two blocks per SM for the extra registers).
template <int P, bool BLK>
__global__ void __launch_bounds__(32 * (SK_BELT_WARPS + 1), BLK ? 2 : 3)
k_conv_belt(const __grid_constant__ JobsArg A) {
    constexpr int NW = SK_BELT_WARPS;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 8 * (2 * S + 1));
    const uint32_t full0 = smem_addr(&bars[0]);
    const uint32_t empty0 = smem_addr(&bars[S]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int TS = 32 * P;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, NW);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    uint32_t gs = 0;        // strips issued/consumed so far (stage and phase)
    // One stage layout for every job of the launch (jobs may differ in WPM): a stage
    // is sized for the widest job, so that stage s has the same bytes whichever job's
    // strip it holds (the full/empty barriers guard stage indices, not byte ranges).
    int wpm_max = 0;
    for (int j = 0; j < A.n_jobs; ++j) wpm_max = max(wpm_max, A.j[j].WPM);
    const int slot = (TS + wpm_max + 4 + 8 + 3) & ~3;               // strip floats
    const uint32_t wmax = (uint32_t)(NW * wpm_max * 8);             // pair-row bytes of a stage
    const uint32_t stage = (uint32_t)slot * 4u + wmax + NW * 8u;

    for (int f = blockIdx.x; f < A.total; f += gridDim.x) {
        if (*abort_flag) break;
        const JobDesc &J = A.j[sk_find_job(A, f)];
        const int local = f - J.flat_base;
        const int map = local / J.n_items;
        const int4 it = J.items[local - map * J.n_items];
        const int grp = it.x;
        const int j0 = it.y * TS;
        const int2 gr = J.bgrp[grp];
        const int nstrips = gr.y - gr.x + 1;
        const int L = TS + J.WPM + 4;                               // strip values this job copies
        const uint32_t wbytes = (uint32_t)(NW * J.WPM * 8);         // pair rows of one strip
        unsigned char *stage0 = smem + HDR;
        const long long js = (long long)j0 + J.EMIN;
        const int phase = (int)(((js % 4) + 4) % 4);
        const float *xmap = J.x + (long long)map * J.stride;

        if (warp == NW) {
            // ---------------- producer ----------------
            if (lane == 0) {
                const int n = J.n4;
                int pos0 = (int)(js % n);
                if (pos0 < 0) pos0 += n;
                uint32_t xbytes = 0;
                {
                    int pos = pos0, rem = L;
                    while (rem > 0) {
                        int len = min(rem, n - pos);
                        int a0 = pos & ~3, a1 = (pos + len + 3) & ~3;
                        xbytes += (uint32_t)(a1 - a0) * 4u;
                        rem -= len; pos = 0;
                    }
                }
                const size_t wrow0 = (size_t)grp * J.smax * NW;
                for (int i = 0; i < nstrips; ++i) {
                    const uint32_t g = gs + i;
                    const int s = (int)(g % S);
                    if (g >= (uint32_t)S &&
                        !mbar_wait(empty0 + 8 * s, ((g / S) - 1) & 1, abort_flag, A.status))
                        break;
                    const float *xr = xmap + J.rings[gr.x + i].start;
                    const uint32_t dst0 = smem_addr(stage0 + (size_t)s * stage);
                    mbar_expect_tx(full0 + 8 * s, xbytes + wbytes + NW * 8u);
                    int pos = pos0, rem = L, m = 0;
                    while (rem > 0) {
                        int len = min(rem, n - pos);
                        int a0 = pos & ~3, a1 = (pos + len + 3) & ~3;
                        uint32_t dst = dst0 + (uint32_t)(phase + m - (pos - a0)) * 4u;
                        bulk_g2s(dst, xr + a0, (uint32_t)(a1 - a0) * 4u, full0 + 8 * s);
                        m += len; rem -= len; pos = 0;
                    }
                    const size_t row = wrow0 + (size_t)i * NW;
                    bulk_g2s(dst0 + (uint32_t)slot * 4u, J.bwp + row * J.WPM, wbytes, full0 + 8 * s);
                    bulk_g2s(dst0 + (uint32_t)slot * 4u + wmax, J.bpr + row, NW * 8u, full0 + 8 * s);
                }
            }
        } else {
            // ---------------- consumers ----------------
            const int rb0 = grp * SK_BELT_G + 2 * warp;           // belt-relative output rings rb0, rb0 + 1
            const int ro0 = J.b_lo + rb0;
            const bool v0 = rb0 < J.nb, v1 = rb0 + 1 < J.nb;
            float2 acc[P];                                        // (ring rb0, ring rb0 + 1)
#pragma unroll
            for (int k = 0; k < P; ++k) acc[k] = make_float2(0.0f, 0.0f);
            bool ok = true;
            for (int i = 0; i < nstrips; ++i) {
                const uint32_t g = gs + i;
                const int s = (int)(g % S);
                if (!mbar_wait(full0 + 8 * s, (g / S) & 1, abort_flag, A.status)) { ok = false; break; }
                const unsigned char *sb = stage0 + (size_t)s * stage;
                const int2 r = reinterpret_cast<const int2 *>(sb + (size_t)slot * 4 + wmax)[warp];
                const float4 *wr = reinterpret_cast<const float4 *>(sb + (size_t)slot * 4) + warp * (J.WPM / 2);
                const float *xs = reinterpret_cast<const float *>(sb) + phase + lane * P + r.x;
                float2 part[BLK ? P : 1];
#pragma unroll
                for (int k = 0; k < (BLK ? P : 1); ++k) part[k] = make_float2(0.0f, 0.0f);
                // Strip values x[m] = xs[m] in a register ring of XB slots (slot m mod XB),
                // duplicated into both halves of a float2 for the paired FMA.  Chunk c
                // (offsets 4c .. 4c+3) uses x[4c .. 4c + P + 2]; while it runs, the 4
                // values chunk c + 1 adds are loaded into slots it does not use
                // (XB >= P + 7).  The chunk loop is unrolled XB / 4 times so that every
                // slot index is a compile-time constant.
                constexpr int XB = ((P + 7 + 3) / 4) * 4, U = XB / 4;
                const int nch = r.y;
                float2 xb[XB];
#pragma unroll
                for (int j = 0; j < P + 3; ++j) {
                    const float v = xs[j];
                    xb[j] = make_float2(v, v);
                }
                float4 wa = wr[0], wb = wr[1];              // weights of chunk c, loaded a chunk ahead
                for (int c0 = 0; c0 < nch; c0 += U) {
#pragma unroll
                    for (int uu = 0; uu < U; ++uu) {
                        const int c = c0 + uu;
                        if (c < nch) {
                            float4 wa_n = wa, wb_n = wb;
                            if (c + 1 < nch) {
#pragma unroll
                                for (int v = 0; v < 4; ++v) {
                                    const float t = xs[4 * c + P + 3 + v];
                                    xb[(4 * uu + P + 3 + v) % XB] = make_float2(t, t);
                                }
                                wa_n = wr[2 * c + 2];
                                wb_n = wr[2 * c + 3];
                            }
                            const float2 w4[4] = {make_float2(wa.x, wa.y), make_float2(wa.z, wa.w),
                                                  make_float2(wb.x, wb.y), make_float2(wb.z, wb.w)};
                            wa = wa_n;
                            wb = wb_n;
#pragma unroll
                            for (int u = 0; u < 4; ++u)
#pragma unroll
                                for (int k = 0; k < P; ++k) {
                                    if constexpr (BLK)
                                        part[k] = __ffma2_rn(w4[u], xb[(4 * uu + k + u) % XB], part[k]);
                                    else
                                        acc[k] = __ffma2_rn(w4[u], xb[(4 * uu + k + u) % XB], acc[k]);
                                }
                        }
                    }
                }
                if constexpr (BLK) {
#pragma unroll
                    for (int k = 0; k < P; ++k) acc[k] = make_float2(acc[k].x + part[k].x, acc[k].y + part[k].y);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(empty0 + 8 * s);
            }
            if (ok) {
                float *yb = J.y + (long long)map * J.stride;
                if (v0) {
                    float *yr = yb + J.rings[ro0].start;
#pragma unroll
                    for (int k = 0; k < P; ++k) {
                        const int j = j0 + lane * P + k;
                        if (j < J.n4) yr[j] = acc[k].x;
                    }
                }
                if (v1) {
                    float *yr = yb + J.rings[ro0 + 1].start;
#pragma unroll
                    for (int k = 0; k < P; ++k) {
                        const int j = j0 + lane * P + k;
                        if (j < J.n4) yr[j] = acc[k].y;
                    }
                }
            }
        }
        gs += (uint32_t)nstrips;
    }
}

template <int P, bool BLK>
cudaError_t launch_p(const JobsArg &a, int grid, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_belt<P, BLK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_conv_belt<P, BLK><<<grid, 32 * (SK_BELT_WARPS + 1), smem, st>>>(a);
    return cudaGetLastError();
}

template <int P, bool BLK>
int occupancy_p(size_t smem) {
    cudaFuncSetAttribute(k_conv_belt<P, BLK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_conv_belt<P, BLK>, 32 * (SK_BELT_WARPS + 1), smem);
    return nb;
}

template <bool BLK>
cudaError_t launch_any(const JobsArg &a, int P, int grid, size_t smem, cudaStream_t st) {
    switch (P) {
        case 5: return launch_p<5, BLK>(a, grid, smem, st);
        case 7: return launch_p<7, BLK>(a, grid, smem, st);
        case 9: return launch_p<9, BLK>(a, grid, smem, st);
        case 11: return launch_p<11, BLK>(a, grid, smem, st);
        case 13: return launch_p<13, BLK>(a, grid, smem, st);
        case 15: return launch_p<15, BLK>(a, grid, smem, st);
        case 17: return launch_p<17, BLK>(a, grid, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

template <bool BLK>
int occupancy_any(int P, size_t smem) {
    switch (P) {
        case 5: return occupancy_p<5, BLK>(smem);
        case 7: return occupancy_p<7, BLK>(smem);
        case 9: return occupancy_p<9, BLK>(smem);
        case 11: return occupancy_p<11, BLK>(smem);
        case 13: return occupancy_p<13, BLK>(smem);
        case 15: return occupancy_p<15, BLK>(smem);
        case 17: return occupancy_p<17, BLK>(smem);
        default: return 1;
    }
}

size_t stage_bytes(int P, int wpm) {
    const int L = 32 * P + wpm + 4;
    const int slot = (L + 8 + 3) & ~3;
    return (size_t)slot * 4 + (size_t)SK_BELT_WARPS * wpm * 8 + (size_t)SK_BELT_WARPS * 8;
}

size_t belt_smem(const JobsArg &a, int P) {
    size_t m = 0;
    for (int j = 0; j < a.n_jobs; ++j) {
        const size_t b = HDR + (size_t)S * stage_bytes(P, a.j[j].WPM);
        m = b > m ? b : m;
    }
    return m;
}

}  // namespace

cudaError_t sk_launch_belt_pairs(const JobDesc &j, int g0, int g1, float2 *w, cudaStream_t st, const int *gate,
                                 bool w64) {
    const long long n = (long long)(g1 - g0) * j.smax * SK_BELT_WARPS * j.WPM;
    if (n <= 0) return cudaSuccess;
    const long long blocks = (n + 255) / 256;
    k_belt_pairs<<<(unsigned)std::min<long long>(blocks, 1 << 20), 256, 0, st>>>(j, g0, g1, w, gate, w64);
    return cudaGetLastError();
}

size_t sk_belt_smem_bytes(int P, int wpm) { return HDR + (size_t)S * stage_bytes(P, wpm); }

cudaError_t sk_launch_conv_belt(const JobsArg &a, int P, bool blocked, int grid, cudaStream_t st) {
    if (a.total <= 0) return cudaSuccess;
    const size_t smem = belt_smem(a, P);
    return blocked ? launch_any<true>(a, P, grid, smem, st) : launch_any<false>(a, P, grid, smem, st);
}

int sk_belt_blocks_per_sm(const JobsArg &a, int P, bool blocked) {
    const size_t smem = belt_smem(a, P);
    return blocked ? occupancy_any<true>(P, smem) : occupancy_any<false>(P, smem);
}
