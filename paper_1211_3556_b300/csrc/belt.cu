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
// Main kernel block: SK_BELT_G consumer warps (one output ring each, the same
// 32 P-pixel segment of consecutive rings) plus one producer warp.  The
// producer streams the segment's input-ring strips into shared memory with
// 1-D TMA bulk copies (cp.async.bulk, 16-byte aligned pieces, split where the
// strip wraps past phi = 2 pi) through SK_BELT_STAGES slots guarded by
// full/empty mbarriers.  Lane l of a consumer warp owns outputs l P .. l P + P-1
// (P odd: the lanes' strip reads hit 32 distinct banks) and slides 4 weights
// at a time over P + 3 strip values held in registers.
#include "skconv.h"
#include "skconv_internal.cuh"
#include "skconv_launch.h"

namespace {

constexpr int G = SK_BELT_G;
constexpr int S = SK_BELT_STAGES;

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
// ring +d, pixel offset e = e_lo + c (zero outside the row's chunks).
__global__ void k_belt_weights(const JobDesc J, float *w) {
    const int R2 = 2 * J.HM + 1;
    const int row = blockIdx.x;
    const int rb = row / R2, d = row % R2 - J.HM;
    float *out = w + (size_t)row * J.WPM;
    const int2 r = (rb < J.nb) ? J.brng[row] : make_int2(0, 0);
    const int ro = J.b_lo + rb;
    PairInfo P;
    int s_o = 0;
    if (r.y > 0) {
        const int p0 = J.pair_off[ro];
        P = J.pairs[p0 + (ro + d - J.pairs[p0].ri)];
        s_o = J.rings[ro].s;
    }
    const double half_step = SK_PI / (2.0 * (double)J.n4);
    for (int c = threadIdx.x; c < J.WPM; c += blockDim.x) {
        float v = 0.0f;
        if (c < 4 * r.y) {
            const int e = r.x + c;
            const float x = (float)((double)(2 * e + P.s_i - s_o) * half_step);
            v = pair_weight(x, P.A, P.B, J.kp, J.tab);
        }
        out[c] = v;
    }
}

template <int P>
__global__ void __launch_bounds__(32 * (G + 1))
k_conv_belt(const __grid_constant__ JobsArg A) {
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
            mbar_init(empty0 + 8 * s, G);
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
        float *sw = reinterpret_cast<float *>(smem + 128);
        int2 *srng = reinterpret_cast<int2 *>(sw + G * R2 * J.WPM);
        float *sstr = reinterpret_cast<float *>(srng + G * R2);
        const int L = TS + J.EMAX - J.EMIN;
        const int slot = (L + 8 + 3) & ~3;
        const long long js = (long long)j0 + J.EMIN;
        const int phase = (int)(((js % 4) + 4) % 4);
        const float *xmap = J.x + (long long)map * J.stride;

        if (warp == G) {
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
            const int ro = J.b_lo + grp * G + warp;
            const bool valid = (grp * G + warp) < J.nb;
            float acc[P];
#pragma unroll
            for (int k = 0; k < P; ++k) acc[k] = 0.0f;
            bool ok = mbar_wait(wfull, witer & 1, abort_flag, A.status);
            for (int i = 0; i < nstrips && ok; ++i) {
                const uint32_t g = gs + i;
                const int s = (int)(g % S);
                if (!mbar_wait(full0 + 8 * s, (g / S) & 1, abort_flag, A.status)) { ok = false; break; }
                const int d = gr.x + i - ro;
                if (valid && d >= -J.HM && d <= J.HM) {
                    const int row = warp * R2 + d + J.HM;
                    const int2 r = srng[row];
                    const float *xs = sstr + (size_t)s * slot + phase + lane * P + (r.x - J.EMIN);
                    const float *wr = sw + (size_t)row * J.WPM;
                    for (int c = 0; c < r.y; ++c) {
                        const float4 w4 = *reinterpret_cast<const float4 *>(wr + 4 * c);
                        float xv[P + 3];
#pragma unroll
                        for (int u = 0; u < P + 3; ++u) xv[u] = xs[4 * c + u];
#pragma unroll
                        for (int k = 0; k < P; ++k) acc[k] = fmaf(w4.x, xv[k], acc[k]);
#pragma unroll
                        for (int k = 0; k < P; ++k) acc[k] = fmaf(w4.y, xv[k + 1], acc[k]);
#pragma unroll
                        for (int k = 0; k < P; ++k) acc[k] = fmaf(w4.z, xv[k + 2], acc[k]);
#pragma unroll
                        for (int k = 0; k < P; ++k) acc[k] = fmaf(w4.w, xv[k + 3], acc[k]);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(empty0 + 8 * s);
            }
            if (valid && ok) {
                float *yr = J.y + (long long)map * J.stride + J.rings[ro].start;
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    const int j = j0 + lane * P + k;
                    if (j < J.n4) yr[j] = acc[k];
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
    k_conv_belt<P><<<grid, 32 * (G + 1), smem, st>>>(a);
    return cudaGetLastError();
}

template <int P>
int occupancy_p(size_t smem) {
    cudaFuncSetAttribute(k_conv_belt<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_conv_belt<P>, 32 * (G + 1), smem);
    return nb;
}

size_t belt_smem(const JobsArg &a, int P) {
    size_t m = 0;
    for (int j = 0; j < a.n_jobs; ++j) {
        const JobDesc &J = a.j[j];
        const int R2 = 2 * J.HM + 1;
        const int L = 32 * P + J.EMAX - J.EMIN;
        const int slot = (L + 8 + 3) & ~3;
        size_t b = 128 + (size_t)G * R2 * J.WPM * 4 + (size_t)G * R2 * 8 + (size_t)S * slot * 4;
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
