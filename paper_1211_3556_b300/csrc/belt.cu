// belt.cu -- equatorial-belt path: the convolution as a ring-wise Toeplitz sum.
//
// In the belt every ring has n = 4 Nside pixels, so for output pixel j of ring
// o and input pixel j + e of ring i the phi difference is pi (2e + s_i - s_o)/n:
// the pair weight dOmega K_lin(gamma) depends on (o, i, e) only, not on j.  A
// pre-pass evaluates those weight rows once per call (per-pair formula of the
// general path, FP32, exact half-angle); the main kernel is then a register-
// blocked 1-D correlation along each ring, one FFMA per in-cut pair.  Same
// operator as the per-pair path (the real-space convolution of Sec. 2, Eq. 1
// with the tabulated kernel of Sec. 3); only the order of work differs.
//
// Main kernel block: SK_BELT_G consecutive output rings, the same 32 P-pixel
// segment of each, computed by SK_BELT_G / 2 consumer warps (two rings each, so
// every staged strip value feeds two weight rows) plus one producer warp.  The
// producer streams the segment's input-ring strips into shared memory with
// 1-D TMA bulk copies (cp.async.bulk, 16-byte aligned pieces, split where the
// strip wraps past phi = 2 pi) through SK_BELT_STAGES slots guarded by
// full/empty mbarriers.  Lane l of a consumer warp owns outputs l P .. l P + P-1
// of its two rings (P odd: the lanes' strip reads hit 32 distinct banks) and
// slides 4 weights of each ring at a time over P + 3 strip values held in
// registers.  Weight rows of all rings share one offset grid, so the two rows
// of a warp line up on the same strip values.
#include "skconv.h"
#include "skconv_internal.cuh"
#include "skconv_launch.h"

namespace {

constexpr int G = SK_BELT_G;
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

// Weight rows: w[rb][d + HM][c] = dOmega K_lin for output ring b_lo + rb, input
// ring +d, pixel offset e = EMIN + c; zero outside the row's window |e - e_c| <= W.
__global__ void k_belt_weights(const JobDesc J, float *w) {
    const int R2 = 2 * J.HM + 1;
    const int row = blockIdx.x;
    const int rb = row / R2, d = row % R2 - J.HM;
    float *out = w + (size_t)row * J.WPM;
    const int2 r = (rb < J.nb) ? J.brng[row] : make_int2(1, 0);
    const int ro = J.b_lo + rb;
    PairInfo P;
    int s_o = 0, ec = 0;
    if (r.x <= r.y) {
        const int p0 = J.pair_off[ro];
        P = J.pairs[p0 + (ro + d - J.pairs[p0].ri)];
        s_o = J.rings[ro].s;
        ec = (s_o + 1 - P.s_i) >> 1;
    }
    const double half_step = SK_PI / (2.0 * (double)J.n4);
    for (int c = threadIdx.x; c < J.WPM; c += blockDim.x) {
        float v = 0.0f;
        const int e = J.EMIN + c;
        if (r.x <= r.y && e >= ec - P.W && e <= ec + P.W) {
            const float x = (float)((double)(2 * e + P.s_i - s_o) * half_step);
            v = pair_weight(x, P.A, P.B, J.kp, J.tab);
        }
        out[c] = v;
    }
}

// Consumer warp w owns output rings b_lo + grp*G + 2w and + 2w + 1; lane l owns
// pixels j0 + l P .. j0 + l P + P - 1 of both.  Strip s holds input ring
// gr.x + i at offsets e = EMIN + m - lane-independent start, so pixel j + e of
// the strip is xs[l P + (e - EMIN) + k].
template <int P>
__global__ void __launch_bounds__(32 * (SK_BELT_WARPS + 1))
k_conv_belt(const __grid_constant__ JobsArg A) {
    constexpr int NW = SK_BELT_WARPS;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 8 * (2 * S + 1));
    const uint32_t full0 = smem_addr(&bars[0]);
    const uint32_t empty0 = smem_addr(&bars[S]);
    const uint32_t wfull = smem_addr(&bars[2 * S]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int TS = 32 * P;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, NW);
        }
        mbar_init(wfull, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    uint32_t gs = 0;        // strips issued/consumed so far (stage and phase)
    uint32_t witer = 0;     // weight loads so far (phase of wfull)

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
        const int R2 = 2 * J.HM + 1;
        float *sw = reinterpret_cast<float *>(smem + HDR);
        float *szero = sw + G * R2 * J.WPM;
        int2 *srng = reinterpret_cast<int2 *>(szero + J.WPM);
        float *sstr = reinterpret_cast<float *>(srng + G * R2);
        const int L = TS + J.WPM;
        const int slot = (L + 8 + 3) & ~3;
        const long long js = (long long)j0 + J.EMIN;
        const int phase = (int)(((js % 4) + 4) % 4);
        const float *xmap = J.x + (long long)map * J.stride;

        if (warp == NW) {
            // ---------------- producer ----------------
            if (lane == 0) {
                const uint32_t wb = (uint32_t)(G * R2 * J.WPM * 4), rbytes = (uint32_t)(G * R2 * 8);
                mbar_expect_tx(wfull, wb + rbytes);
                bulk_g2s(smem_addr(sw), J.bw + (size_t)grp * G * R2 * J.WPM, wb, wfull);
                bulk_g2s(smem_addr(srng), J.brng + (size_t)grp * G * R2, rbytes, wfull);
                const int n = J.n4;
                int pos0 = (int)(js % n);
                if (pos0 < 0) pos0 += n;
                for (int i = 0; i < nstrips; ++i) {
                    const uint32_t g = gs + i;
                    const int s = (int)(g % S);
                    if (g >= (uint32_t)S &&
                        !mbar_wait(empty0 + 8 * s, ((g / S) - 1) & 1, abort_flag, A.status))
                        break;
                    const float *xr = xmap + J.rings[gr.x + i].start;
                    const uint32_t dst0 = smem_addr(sstr + (size_t)s * slot);
                    uint32_t total = 0;
                    {
                        int pos = pos0, rem = L;
                        while (rem > 0) {
                            int len = min(rem, n - pos);
                            int a0 = pos & ~3, a1 = (pos + len + 3) & ~3;
                            total += (uint32_t)(a1 - a0) * 4u;
                            rem -= len; pos = 0;
                        }
                    }
                    mbar_expect_tx(full0 + 8 * s, total);
                    int pos = pos0, rem = L, m = 0;
                    while (rem > 0) {
                        int len = min(rem, n - pos);
                        int a0 = pos & ~3, a1 = (pos + len + 3) & ~3;
                        uint32_t dst = dst0 + (uint32_t)(phase + m - (pos - a0)) * 4u;
                        bulk_g2s(dst, xr + a0, (uint32_t)(a1 - a0) * 4u, full0 + 8 * s);
                        m += len; rem -= len; pos = 0;
                    }
                }
            }
        } else {
            // ---------------- consumers ----------------
            for (int c = threadIdx.x; c < J.WPM; c += 32 * NW) szero[c] = 0.0f;
            asm volatile("bar.sync 1, %0;" ::"r"(32 * NW));       // consumers only
            const int rb0 = grp * G + 2 * warp;                   // belt-relative output rings rb0, rb0 + 1
            const int ro0 = J.b_lo + rb0;
            const bool v0 = rb0 < J.nb, v1 = rb0 + 1 < J.nb;
            float acc0[P], acc1[P];
#pragma unroll
            for (int k = 0; k < P; ++k) { acc0[k] = 0.0f; acc1[k] = 0.0f; }
            bool ok = mbar_wait(wfull, witer & 1, abort_flag, A.status);
            for (int i = 0; i < nstrips && ok; ++i) {
                const uint32_t g = gs + i;
                const int s = (int)(g % S);
                if (!mbar_wait(full0 + 8 * s, (g / S) & 1, abort_flag, A.status)) { ok = false; break; }
                const int d0 = gr.x + i - ro0, d1 = d0 - 1;
                const bool u0 = v0 && d0 >= -J.HM && d0 <= J.HM;
                const bool u1 = v1 && d1 >= -J.HM && d1 <= J.HM;
                const int2 r0 = u0 ? srng[(2 * warp) * R2 + d0 + J.HM] : make_int2(1, 0);
                const int2 r1 = u1 ? srng[(2 * warp + 1) * R2 + d1 + J.HM] : make_int2(1, 0);
                const int ca = min(r0.x, r1.x), cb = max(r0.y, r1.y);
                const float *wr0 = (r0.x <= r0.y) ? sw + (size_t)((2 * warp) * R2 + d0 + J.HM) * J.WPM : szero;
                const float *wr1 = (r1.x <= r1.y) ? sw + (size_t)((2 * warp + 1) * R2 + d1 + J.HM) * J.WPM : szero;
                const float *xs = sstr + (size_t)s * slot + phase + lane * P;
                for (int c = ca; c <= cb; ++c) {
                    const float4 wa = *reinterpret_cast<const float4 *>(wr0 + 4 * c);
                    const float4 wb = *reinterpret_cast<const float4 *>(wr1 + 4 * c);
                    float xv[P + 3];
#pragma unroll
                    for (int u = 0; u < P + 3; ++u) xv[u] = xs[4 * c + u];
#pragma unroll
                    for (int k = 0; k < P; ++k) acc0[k] = fmaf(wa.x, xv[k], acc0[k]);
#pragma unroll
                    for (int k = 0; k < P; ++k) acc1[k] = fmaf(wb.x, xv[k], acc1[k]);
#pragma unroll
                    for (int k = 0; k < P; ++k) acc0[k] = fmaf(wa.y, xv[k + 1], acc0[k]);
#pragma unroll
                    for (int k = 0; k < P; ++k) acc1[k] = fmaf(wb.y, xv[k + 1], acc1[k]);
#pragma unroll
                    for (int k = 0; k < P; ++k) acc0[k] = fmaf(wa.z, xv[k + 2], acc0[k]);
#pragma unroll
                    for (int k = 0; k < P; ++k) acc1[k] = fmaf(wb.z, xv[k + 2], acc1[k]);
#pragma unroll
                    for (int k = 0; k < P; ++k) acc0[k] = fmaf(wa.w, xv[k + 3], acc0[k]);
#pragma unroll
                    for (int k = 0; k < P; ++k) acc1[k] = fmaf(wb.w, xv[k + 3], acc1[k]);
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
                        if (j < J.n4) yr[j] = acc0[k];
                    }
                }
                if (v1) {
                    float *yr = yb + J.rings[ro0 + 1].start;
#pragma unroll
                    for (int k = 0; k < P; ++k) {
                        const int j = j0 + lane * P + k;
                        if (j < J.n4) yr[j] = acc1[k];
                    }
                }
            }
        }
        gs += (uint32_t)nstrips;
        ++witer;
        __syncthreads();
    }
}

template <int P>
cudaError_t launch_p(const JobsArg &a, int grid, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_belt<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_conv_belt<P><<<grid, 32 * (SK_BELT_WARPS + 1), smem, st>>>(a);
    return cudaGetLastError();
}

template <int P>
int occupancy_p(size_t smem) {
    cudaFuncSetAttribute(k_conv_belt<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_conv_belt<P>, 32 * (SK_BELT_WARPS + 1), smem);
    return nb;
}

size_t belt_smem(const JobsArg &a, int P) {
    size_t m = 0;
    for (int j = 0; j < a.n_jobs; ++j) {
        const JobDesc &J = a.j[j];
        const int R2 = 2 * J.HM + 1;
        const int L = 32 * P + J.WPM;
        const int slot = (L + 8 + 3) & ~3;
        size_t b = HDR + (size_t)G * R2 * J.WPM * 4 + (size_t)J.WPM * 4 + (size_t)G * R2 * 8 + (size_t)S * slot * 4;
        m = b > m ? b : m;
    }
    return m;
}

}  // namespace

cudaError_t sk_launch_belt_weights(const JobDesc &j, float *w, cudaStream_t st) {
    const int groups = (j.nb + G - 1) / G;
    const int rows = groups * G * (2 * j.HM + 1);
    k_belt_weights<<<rows, 32, 0, st>>>(j, w);
    return cudaGetLastError();
}

cudaError_t sk_launch_conv_belt(const JobsArg &a, int P, int grid, cudaStream_t st) {
    if (a.total <= 0) return cudaSuccess;
    size_t smem = belt_smem(a, P);
    switch (P) {
        case 5: return launch_p<5>(a, grid, smem, st);
        case 7: return launch_p<7>(a, grid, smem, st);
        case 9: return launch_p<9>(a, grid, smem, st);
        case 11: return launch_p<11>(a, grid, smem, st);
        case 13: return launch_p<13>(a, grid, smem, st);
        case 15: return launch_p<15>(a, grid, smem, st);
        case 17: return launch_p<17>(a, grid, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

int sk_belt_blocks_per_sm(const JobsArg &a, int P) {
    size_t smem = belt_smem(a, P);
    switch (P) {
        case 5: return occupancy_p<5>(smem);
        case 7: return occupancy_p<7>(smem);
        case 9: return occupancy_p<9>(smem);
        case 11: return occupancy_p<11>(smem);
        case 13: return occupancy_p<13>(smem);
        case 15: return occupancy_p<15>(smem);
        case 17: return occupancy_p<17>(smem);
        default: return 0;
    }
}
