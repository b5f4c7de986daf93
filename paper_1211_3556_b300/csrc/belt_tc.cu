// belt_tc.cu -- batched tensor-core form of the belt path (tcgen05, 3xTF32).
//
// For many maps sharing one kernel the belt sums are a dense contraction per
// ring block: for input ring i and output ring o (both with 4 Nside pixels)
//   Y[o][j][b] += sum_k W_{o,i}[j, k] X[i][k][b],   W_{o,i}[j, k] = w(o, i, e = k - j)
// with the Toeplitz weight rows w of the belt path (the same operator: the
// real-space convolution of Sec. 2, Eq. 1 with the tabulated kernel of Sec. 3).
//
// Work item: 16 consecutive belt rings x 64 consecutive pixels x 32 maps.
//  * MMA shape M = 128 (16 rings x 8 output pixels), N = 32 maps, K = 8.
//  * A (weights, 128 x KT): row (r, n) = ring r of the block, output pixel n of
//    an 8-pixel segment; column k = input pixel j0s + EMIN4 + k.  Toeplitz, so
//    the same tile serves all 8 segments of the item; rebuilt per input ring.
//  * B (maps, 32 x XL): the 32 maps' pixels j0 + EMIN4 .. j0 + EMIN4 + XL of
//    input ring i (wrapped around the ring); segment s uses columns 8s ..
//    8s + KT, i.e. the same tile with the descriptor start moved by 32 bytes
//    per segment.
//  * 3xTF32: A and B are split into TF32 hi/lo parts (both rounded to nearest)
//    and hi*hi + hi*lo + lo*hi approximates the FP32 product.
//  * D: per segment two 128 x 32 accumulators in tensor memory (all 512
//    columns): one for hi*hi, one for the small hi*lo + lo*hi terms.  The
//    tensor core adds each MMA's products into its FP32 accumulator with a
//    truncation relative to the accumulator; keeping the small terms apart
//    keeps that error ~2^-10 smaller for them, and the two are added in FP32
//    when read back.
// Warp-specialised: 15 builder warps write the operands into 128-byte-swizzled
// K-major shared memory (two stages), loading the next input ring's maps and
// weight rows into registers while the current one is built, and arrive on
// the stage's "full" mbarrier; one MMA warp waits on it, issues the MMAs (the
// descriptors differ only in their start-address field) and commits them to
// the stage's "empty" mbarrier, which releases the stage to the builders.
// Bounded waits record SK_ETIMEOUT.
#include <string.h>

#include <algorithm>

#include "skconv_host.h"
#include "tc.cuh"

namespace {

constexpr int NB = SK_TC_MAPS;         // maps per item (MMA N)
constexpr int RG = SK_BELT_G;          // rings per item
constexpr int SO = 128 / RG;           // output pixels per ring per segment (8)
constexpr int NSEG = 256 / NB;         // segments per item (two accumulators each in 512 columns)
constexpr int SEGW = SO * NSEG;        // output pixels per ring per item (128)
static_assert(RG * SO == 128, "M must be 128");
static_assert(SEGW == SK_TC_SEGW, "item width");

struct Lay {
    uint32_t a_bytes, x_bytes, w_off, stage;
};

__host__ __device__ inline Lay layout(const TcGeom &g, int wpm) {
    Lay l;
    l.a_bytes = (uint32_t)g.ka * 128 * 128;
    l.x_bytes = (uint32_t)g.xa * NB * 128;
    l.w_off = 2 * l.a_bytes + 2 * l.x_bytes;
    l.stage = (l.w_off + (uint32_t)RG * wpm * 4 + 1023) & ~1023u;
    return l;
}

constexpr int NT = 512;                 // threads per block: 15 builder warps + 1 MMA warp
constexpr int NBLD = NT - 32;           // builder threads
constexpr int XQ = 2;                   // 16-byte map chunks per builder thread per strip
constexpr int WQ = 2;                   // weight-row values per builder thread per strip

// Loads (into registers) of one strip: the maps' pixels and the 16 weight rows.
struct Prefetch {
    float4 x[XQ];
    float w[WQ];
};

__device__ __forceinline__ void load_strip(Prefetch &pf, const JobDesc &J, const TcGeom &tg, int grp, int ri,
                                           int j0, int b0, int nmaps) {
    const int t = threadIdx.x;
    const int nq = tg.xl >> 2;
    const int emin4 = J.EMIN - tg.off4;
    const long long st_i = J.rings[ri].start;
#pragma unroll
    for (int u = 0; u < XQ; ++u) {
        const int q = t + u * NBLD;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q < NB * nq) {
            const int m = q / nq, c4 = q - m * nq;
            int pos = (j0 + emin4 + 4 * c4) % J.n4;
            if (pos < 0) pos += J.n4;
            if (m < nmaps) v = __ldg(reinterpret_cast<const float4 *>(J.x + (long long)(b0 + m) * J.stride + st_i + pos));
        }
        pf.x[u] = v;
    }
    const int R2 = 2 * J.HM + 1;
#pragma unroll
    for (int u = 0; u < WQ; ++u) {
        const int q = t + u * NBLD;
        float v = 0.0f;
        if (q < RG * J.WPM) {
            const int r = q / J.WPM, c = q - r * J.WPM;
            const int rb = grp * RG + r, d = ri - (J.b_lo + rb);
            if (rb < J.nb && d >= -J.HM && d <= J.HM) v = __ldg(J.bw + ((size_t)rb * R2 + d + J.HM) * J.WPM + c);
        }
        pf.w[u] = v;
    }
}

__device__ __forceinline__ void bld_sync() { asm volatile("bar.sync 1, %0;" ::"r"(NBLD) : "memory"); }
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(NT, 1)
k_belt_tc(const __grid_constant__ JobsArg A, const TcGeom tg) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[2];      // builders -> MMA warp: operands of a stage ready
    __shared__ __align__(8) uint64_t empty_bar[2];     // MMA completion -> builders: stage free
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const bool mma_warp = warp == NT / 32 - 1;

    if (warp == 0) tc::tmem_alloc(&tslot, 512);
    if (t == 0) {
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(tc::smem_u32(&full_bar[s]), NBLD / 32);
            tc::mbar_init(tc::smem_u32(&empty_bar[s]), 1);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;
    const uint32_t idesc = tc::idesc_tf32(128, NB);
    const unsigned long long LIMIT = 2000000000ull;

    uint32_t gi = 0;                                   // strips so far (stage, phase)
    for (int f = blockIdx.x; f < A.total && !abort_flag; f += gridDim.x) {
        const JobDesc &J = A.j[sk_find_job(A, f)];
        const Lay L = layout(tg, J.WPM);
        const int local = f - J.flat_base;
        const int mb = local / J.n_items;
        const int4 it = J.items[local - mb * J.n_items];
        const int grp = it.x, j0 = it.y * SEGW;
        const int b0 = mb * NB, nmaps = min(NB, J.batch - b0);
        const int2 gr = J.bgrp[grp];
        const int nstrips = gr.y - gr.x + 1;
        const int n4 = J.n4;
        const uint32_t gi0 = gi;

        if (!mma_warp) {
            // ---------------- builders ----------------
            Prefetch pf;
            load_strip(pf, J, tg, grp, gr.x, j0, b0, nmaps);
            const int nq = tg.xl >> 2;
            const int ach = tg.kt8 >> 2;                   // 16-byte chunks per weight-tile row
            for (int i = 0; i < nstrips; ++i) {
                const uint32_t g = gi0 + i;
                const int st = (int)(g & 1);
                unsigned char *a_hi = base + st * L.stage;
                unsigned char *a_lo = a_hi + L.a_bytes;
                unsigned char *x_hi = a_lo + L.a_bytes;
                unsigned char *x_lo = x_hi + L.x_bytes;
                float *wrow = reinterpret_cast<float *>(a_hi + L.w_off);
                if (g >= 2 && !tc::mbar_wait(tc::smem_u32(&empty_bar[st]), ((g >> 1) - 1) & 1, LIMIT)) {
                    abort_flag = 1;
                    atomicCAS(A.status, 0, SK_ETIMEOUT);
                }
                bld_sync();                                // every builder decides on the same flag
                if (abort_flag) break;
#pragma unroll
                for (int u = 0; u < WQ; ++u) {
                    const int q = t + u * NBLD;
                    if (q < RG * J.WPM) wrow[q] = pf.w[u];
                }
#pragma unroll
                for (int u = 0; u < XQ; ++u) {
                    const int q = t + u * NBLD;
                    if (q < NB * nq) {
                        const int m = q / nq, k = 4 * (q - m * nq);
                        float4 hi, lo;
                        tc::split_tf32(pf.x[u].x, hi.x, lo.x);
                        tc::split_tf32(pf.x[u].y, hi.y, lo.y);
                        tc::split_tf32(pf.x[u].z, hi.z, lo.z);
                        tc::split_tf32(pf.x[u].w, hi.w, lo.w);
                        const uint32_t off = (uint32_t)(k >> 5) * NB * 128 + tc::sw128_offset(m, k);
                        *reinterpret_cast<float4 *>(x_hi + off) = hi;
                        *reinterpret_cast<float4 *>(x_lo + off) = lo;
                    }
                }
                if (i + 1 < nstrips) load_strip(pf, J, tg, grp, gr.x + i + 1, j0, b0, nmaps);
                bld_sync();                                // weight rows visible to all builders
                // A: 16-byte chunk (row, k..k+3), row = (r, n): w_r[k + u - n - off4]
                for (int q = t; q < 128 * ach; q += NBLD) {
                    const int row = q / ach, k = 4 * (q - row * ach);
                    const int r = row >> 3, n = row & 7;
                    const float *wr = wrow + r * J.WPM;
                    float v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int c = k + u - n - tg.off4;
                        v[u] = (c >= 0 && c < J.WPM) ? wr[c] : 0.0f;
                    }
                    float4 hi, lo;
                    tc::split_tf32(v[0], hi.x, lo.x);
                    tc::split_tf32(v[1], hi.y, lo.y);
                    tc::split_tf32(v[2], hi.z, lo.z);
                    tc::split_tf32(v[3], hi.w, lo.w);
                    const uint32_t off = (uint32_t)(k >> 5) * 128 * 128 + tc::sw128_offset(row, k);
                    *reinterpret_cast<float4 *>(a_hi + off) = hi;
                    *reinterpret_cast<float4 *>(a_lo + off) = lo;
                }
                tc::fence_smem_to_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(tc::smem_u32(&full_bar[st]));
            }
        } else if (lane == 0) {
            // ---------------- MMA issuer ----------------
            for (int i = 0; i < nstrips; ++i) {
                const uint32_t g = gi0 + i;
                const int st = (int)(g & 1);
                if (!tc::mbar_wait(tc::smem_u32(&full_bar[st]), (g >> 1) & 1, LIMIT)) {
                    abort_flag = 1;
                    atomicCAS(A.status, 0, SK_ETIMEOUT);
                }
                if (abort_flag) break;
                tc::fence_after_sync();
                unsigned char *a_hi = base + st * L.stage;
                const uint64_t dah0 = tc::sw128_desc(tc::smem_u32(a_hi));
                const uint64_t dal0 = tc::sw128_desc(tc::smem_u32(a_hi + L.a_bytes));
                const uint64_t dxh0 = tc::sw128_desc(tc::smem_u32(a_hi + 2 * L.a_bytes));
                const uint64_t dxl0 = tc::sw128_desc(tc::smem_u32(a_hi + 2 * L.a_bytes + L.x_bytes));
                for (int s = 0; s < NSEG; ++s) {
                    const uint32_t d_big = taddr + (uint32_t)(s * NB);
                    const uint32_t d_small = taddr + 256u + (uint32_t)(s * NB);
                    for (int tk = 0; tk < tg.kt8 / 8; ++tk) {
                        const int ka = 8 * tk, kx = 8 * s + 8 * tk;
                        // the start address is the descriptor's low field (in 16-byte units)
                        const uint64_t ao = ((uint32_t)(ka >> 5) * 128 * 128 + (uint32_t)(ka & 31) * 4) >> 4;
                        const uint64_t xo = ((uint32_t)(kx >> 5) * NB * 128 + (uint32_t)(kx & 31) * 4) >> 4;
                        const int acc = (i > 0 || tk > 0) ? 1 : 0;
                        tc::mma_tf32(d_big, dah0 + ao, dxh0 + xo, idesc, acc);
                        tc::mma_tf32(d_small, dah0 + ao, dxl0 + xo, idesc, acc);
                        tc::mma_tf32(d_small, dal0 + ao, dxh0 + xo, idesc, 1);
                    }
                }
                tc::mma_commit(tc::smem_u32(&empty_bar[st]));
            }
        }
        gi = gi0 + (uint32_t)nstrips;
        __syncthreads();
        if (abort_flag) break;
        // all MMAs of the item are done once the last commit has landed
        const uint32_t last = gi - 1;
        if (!tc::mbar_wait(tc::smem_u32(&empty_bar[last & 1]), (last >> 1) & 1, LIMIT)) {
            if (t == 0) { abort_flag = 1; atomicCAS(A.status, 0, SK_ETIMEOUT); }
        }
        __syncthreads();
        if (abort_flag) break;
        tc::fence_after_sync();
        {
            // warp w reads lane quadrant w % 4 (rows 32 (w % 4) ..) of segments s = w / 4, w / 4 + 4, ...
            const int quad = warp & 3;
            const int row = quad * 32 + lane;
            const int r = row / SO, n = row - r * SO;
            const int rb = grp * RG + r;
            const bool valid = rb < J.nb;
            float *yr = J.y + (long long)b0 * J.stride + (valid ? J.rings[J.b_lo + rb].start : 0);
            for (int s = warp >> 2; s < NSEG; s += NT / 128) {
                float v[16], w[16];
                for (int h = 0; h < NB / 16; ++h) {
                    const uint32_t lane_base = taddr + ((uint32_t)(quad * 32) << 16) + (uint32_t)(s * NB + 16 * h);
                    tc::tmem_ld16(lane_base, v);
                    tc::tmem_ld16(lane_base + 256u, w);
                    const int j = j0 + s * SO + n;
                    if (valid && j < n4) {
#pragma unroll
                        for (int m = 0; m < 16; ++m)
                            if (16 * h + m < nmaps) yr[(long long)(16 * h + m) * J.stride + j] = v[m] + w[m];
                    }
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    // leave no MMA in flight before releasing tensor memory (bounded)
    if (gi > 0) {
        const uint32_t last = gi - 1;
        tc::mbar_wait(tc::smem_u32(&empty_bar[last & 1]), (last >> 1) & 1, LIMIT);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(taddr, 512);
    }
}

}  // namespace

bool sk_tc_geometry(int wpm, int emin, int n4, TcGeom *g) {
    const int emin4 = emin >= 0 ? (emin & ~3) : -(((-emin) + 3) & ~3);
    g->off4 = emin - emin4;
    const int kt = wpm + (SO - 1) + g->off4;
    g->kt8 = (kt + 7) & ~7;
    g->ka = (g->kt8 + 31) / 32;
    g->xl = ((8 * (NSEG - 1) + g->kt8) + 31) & ~31;
    g->xa = g->xl / 32;
    if (g->ka > 2 || n4 % SEGW) return false;
    if (NB * (g->xl / 4) > XQ * NBLD || RG * wpm > WQ * NBLD) return false;   // per-thread prefetch slots
    return sk_tc_smem(*g, wpm) <= 220 * 1024;
}

size_t sk_tc_smem(const TcGeom &g, int wpm) { return 1024 + 2 * (size_t)layout(g, wpm).stage; }

cudaError_t sk_launch_belt_tc(const JobsArg &a, const TcGeom &g, int wpm_max, int grid, cudaStream_t st) {
    if (a.total <= 0) return cudaSuccess;
    // at least 120 KB so that one block holds an SM (it allocates all 512 tensor-memory columns)
    const size_t smem = std::max(sk_tc_smem(g, wpm_max), (size_t)120 * 1024);
    cudaError_t e = cudaFuncSetAttribute(k_belt_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_belt_tc<<<grid, NT, smem, st>>>(a, g);
    return cudaGetLastError();
}
