// grad.cu -- gradient of a loss with respect to the kernel table nodes.
//
// With y_o = dOmega sum_i K_lin(gamma_oi) x_i and K_lin = V_k (1 - f) + V_{k+1} f
// (linear interpolation of the tabulated kernel, Sec. 3),
//   dL/dV_n = dOmega sum_b sum_o gy_bo sum_{i in cut} x_bi [(1 - f) delta_{n,k} + f delta_{n,k+1}],
// a binned scatter-add over all in-cut pairs.  (k, f) come from FP64 chord
// arithmetic (an FP32 node coordinate u would carry an absolute error near
// u * 6e-8, which the bins see undamped); the pair sums v are FP32.  The work
// follows the forward paths' structure:
//  * belt rings: every pair (o, j) - (i, j + e) of a ring pair has the same (k, f),
//    so the pairs of one (o, i, e) add up to one cross-correlation
//    C_oi(e) = sum_b sum_j gy_bo[j] x_bi[j + e] before touching the bins
//    (k_grad_belt: a block per output ring, lanes over offsets, warps over pixels);
//  * cap rings: a base pair and its 16 symmetric images share (k, f), so one FP64
//    evaluation serves 16 products per map (k_grad_cap, inputs from the caps'
//    symmetric copy, four maps per pass; the node coordinate in double-float FP32 where
//    the cut is small, FP64 otherwise, evaluated on the first pass and cached for the
//    others; each lane starts its window walk at its own position so that a warp's bin
//    updates spread over the table);
//  * the remaining rings: one thread per output pixel walks its window
//    (k_grad_general).
// Each block adds its bins (FP32 in shared memory, or FP64 directly for the belt's
// few values) into an FP64 accumulator in global memory; a last kernel scales by
// dOmega and rounds.
#include "skconv.h"
#include "skconv_internal.cuh"
#include "skconv_launch.h"

namespace {

// ---------------------------------------------------------------------------
// Double-float arithmetic: an unevaluated sum hi + lo of two FP32 values (about 44
// significant bits), products by FMA (two-product), sums by Knuth's two-sum (Knuth,
// TAOCP vol. 2, 4.2.2; Dekker 1971).  The table gradient uses it where FP64 would do
// and FP64 issue would be the limit (B300 runs FP64 at about 1/64 of the FP32 rate).
// The _rn intrinsics keep the compiler from contracting or reassociating the steps.
// ---------------------------------------------------------------------------
struct dfloat {
    float hi, lo;
};
__device__ __forceinline__ dfloat df_from(double v) {
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {     // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
    const dfloat s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfloat df_mul_f(dfloat a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return df_fast_two_sum(p, e);
}

// Per-ring-pair and per-kernel constants of pair_kf_df, split from their FP64 values.
struct PairDF {
    dfloat c0, A, B;
};
struct KernDF {
    dfloat tcut, inv_h;
};

// pair_kf64's node interval and fraction in double-float, for the uniform node layout
// with theta_cut <= 0.15 and |x| <= 1/8 (returns -1 otherwise: the caller takes
// pair_kf64); 1 inside the cut, 0 outside.  q is the exact integer of the half-angle
// x = q c0 (|q| < 2^24).  Same mathematics as pair_kf64:
//   sin^2 x = x^2 (1 + R), R = -x^2/3 + 2x^4/45 - x^6/315 + 2x^8/14175 in FP32 (|R| <= 5.2e-3,
//     so its rounding is below 3.1e-10 of sin^2 x; the next term is 4e-15 of it);
//   t = A + B sin^2 x, the cut t <= tcut in double-float;
//   c = sqrt(t): the FP32 root refined by one Newton step on the double-float t;
//   gamma = c (1 + Qm1), Qm1 = t/24 + 3t^2/640 + 5t^3/7168 + 35t^4/294912 in FP32
//     (|Qm1| <= 1e-3: rounding below 1.2e-10 of gamma; truncation 1.3e-13);
//   u = gamma inv_h, k = floor(u) (at most nt - 2), f = u - k.
// About 2.5e-10 relative in gamma at worst, i.e. below 1e-6 in f for 4096 nodes.
__device__ __forceinline__ int pair_kf_df(float q, const PairDF &P, const KernDF &K, const KernParams &kp,
                                          int &k, float &f) {
    const dfloat x = df_mul_f(P.c0, q);
    if (!(fabsf(x.hi) <= 0.125f)) return -1;
    const dfloat x2 = df_mul(x, x);
    const float y = x2.hi;
    float R = __fmaf_rn(y, 2.0f / 14175.0f, -1.0f / 315.0f);
    R = __fmaf_rn(y, R, 2.0f / 45.0f);
    R = __fmaf_rn(y, R, -1.0f / 3.0f);
    R = __fmul_rn(R, y);
    const dfloat s2 = df_add(x2, df_mul_f(x2, R));
    const dfloat t = df_add(P.A, df_mul(P.B, s2));
    if (!(t.hi < K.tcut.hi || (t.hi == K.tcut.hi && t.lo <= K.tcut.lo))) return 0;
    float uh = 0.0f, ul = 0.0f;
    if (t.hi > 0.0f) {
        const float c32 = __fsqrt_rn(t.hi);
        const float p = __fmul_rn(c32, c32);
        const float e = __fmaf_rn(c32, c32, -p);
        const float r = __fadd_rn(__fsub_rn(__fsub_rn(t.hi, p), e), t.lo);     // t - c32^2
        const dfloat c = df_fast_two_sum(c32, __fmul_rn(r, __fdiv_rn(0.5f, c32)));
        const float th = t.hi;
        float Q = __fmaf_rn(th, 35.0f / 294912.0f, 5.0f / 7168.0f);
        Q = __fmaf_rn(th, Q, 3.0f / 640.0f);
        Q = __fmaf_rn(th, Q, 1.0f / 24.0f);
        Q = __fmul_rn(Q, th);
        const dfloat u = df_mul(df_add(c, df_mul_f(c, Q)), K.inv_h);
        uh = u.hi;
        ul = u.lo;
    }
    float kf = floorf(uh);
    float fr = __fadd_rn(__fsub_rn(uh, kf), ul);         // uh - kf is exact (uh < 2^23)
    if (fr < 0.0f) { kf -= 1.0f; fr += 1.0f; }
    int kk = (int)kf;
    if (kk > kp.nt - 2) { fr += (float)(kk - (kp.nt - 2)); kk = kp.nt - 2; }
    k = kk;
    f = fr;
    return 1;
}


constexpr int GB = 8;           // maps folded into one pair visit

__global__ void __launch_bounds__(128)
k_grad_general(const __grid_constant__ JobsArg A, const float *__restrict__ gy, double *acc) {
    extern __shared__ float bins[];
    const JobDesc &J = A.j[0];
    const int nt = J.kp.nt;
    for (int k = threadIdx.x; k < nt; k += blockDim.x) bins[k] = 0.0f;
    __syncthreads();
    const int nchunk = (J.batch + GB - 1) / GB;
    const int total = J.n_items * nchunk;
    for (int f = blockIdx.x; f < total; f += gridDim.x) {
        const int chunk = f / J.n_items;
        const int4 it = J.items[f - chunk * J.n_items];
        const int b0 = chunk * GB;
        const int nb = min(GB, J.batch - b0);
        const int ro = it.x;
        const RingDev R = J.rings[ro];
        const int jo = it.y + (int)threadIdx.x;
        if (jo >= R.n) continue;
        float g[GB];
        bool any = false;
#pragma unroll
        for (int b = 0; b < GB; ++b) {
            g[b] = b < nb ? gy[(long long)(b0 + b) * J.stride + R.start + jo] : 0.0f;
            any |= g[b] != 0.0f;
        }
        if (!any) continue;
        const float *xb = J.x + (long long)b0 * J.stride;
        for (int p = J.pair_off[ro]; p < J.pair_off[ro + 1]; ++p) {
            const PairInfo P = J.pairs[p];
            const double2 ab = J.ab64[p];
            const double c0 = SK_PI / (2.0 * (double)P.n_i * (double)R.n);
            const float *xr = xb + J.rings[P.ri].start;
            int jlo, cnt;
            pair_window(jo, R.n, R.s, P, jlo, cnt);
            long long q = pair_q(jlo, jo, R.n, R.s, P);
            int j = jlo % P.n_i; if (j < 0) j += P.n_i;
            const int dq = 2 * R.n;
            for (int m = 0; m < cnt; ++m) {
                int k; float fr;
                if (pair_kf64((double)q * c0, ab.x, ab.y, J.kp, J.kd, k, fr)) {
                    float v = 0.0f;
#pragma unroll
                    for (int b = 0; b < GB; ++b)
                        if (b < nb) v = fmaf(g[b], __ldg(xr + (long long)b * J.stride + j), v);
                    atomicAdd(&bins[k], v - fr * v);
                    atomicAdd(&bins[k + 1], fr * v);
                }
                q += dq;
                if (++j == P.n_i) j = 0;
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nt; k += blockDim.x)
        if (bins[k] != 0.0f) atomicAdd(&acc[k], (double)bins[k]);
}

// Belt rings, step 1: C[o][i][c] = sum_b sum_j gy_bo[j] x_bi[j + e], e = EMIN + c, for every
// belt output ring o, input ring i of its window and offset c < WPM.  A block per (OB
// consecutive belt output rings, pair of maps, chunk of RC positions of their windows);
// the input rings the OB windows share are staged once.  A thread per (output ring,
// quarter of the pixels (G groups), window ring, 8 consecutive offsets).  The two maps
// travel together as float2 (gy pairs and x pairs interleaved in shared memory), so one
// paired FMA does both; a thread keeps the 8 x pairs its offsets need at pixel j in
// registers and, from pixel to pixel, loads one new pair (the window slides by one) and
// one gy pair (shared by the threads of its output ring): 8 paired FMAs per two 64-bit
// shared loads.  Pixels in segments of GT_SEG; each segment's sums go into a second
// accumulator (blocked summation over the 4N pixels x maps).
constexpr int GT_SEG = 256;     // pixels of a segment
constexpr int GT_LAG = 8;       // offsets per thread
__host__ __device__ __forceinline__ int gt_row(int segn, int ncb) { return segn + GT_LAG * ncb + 1; }   // odd: rows spread over banks

__global__ void __launch_bounds__(512)
k_grad_belt(const JobDesc J, const float *__restrict__ gy, float *C, int RC, int G, int OB, int NR) {
    extern __shared__ float2 sm2[];
    const int n = J.n4, R2 = 2 * J.HM + 1;
    const int rb0 = blockIdx.x * OB, nout = min(OB, J.nb - rb0);
    const int pc = blockIdx.z * RC;                    // the chunk's first position in each window
    const int ncb = (J.WPM + GT_LAG - 1) / GT_LAG;
    const int segn = min(n, GT_SEG);
    const int LR = gt_row(segn, ncb);
    // the rings the chunk covers in the block's windows (contiguous: windows are ring ranges
    // that move with the output ring)
    int rlo = 1 << 30, rhi = -1;
    for (int k = 0; k < nout; ++k) {
        const int o = J.b_lo + rb0 + k;
        const int a = J.pair_off[o] + pc, e = min(J.pair_off[o] + pc + RC, J.pair_off[o + 1]) - 1;
        if (a <= e) {
            rlo = min(rlo, J.pairs[a].ri);
            rhi = max(rhi, J.pairs[e].ri);
        }
    }
    if (rhi < rlo) return;
    const int nrows = min(rhi - rlo + 1, NR);
    float2 *gys = sm2;                                 // [OB][segn]
    float2 *xs = gys + (size_t)OB * segn;              // [NR][LR]
    long long *xrow = reinterpret_cast<long long *>(xs + (size_t)NR * LR);   // [NR] input ring starts
    const int t = threadIdx.x;
    const int tpg = blockDim.x / (OB * G);
    const int ob = t / (G * tpg), rem = t - ob * G * tpg, grp = rem / tpg, tt = rem - grp * tpg;
    const int pp = tt % RC, cb = tt / RC;
    const int o = J.b_lo + rb0 + ob;
    const int np = ob < nout ? min(RC, J.pair_off[o + 1] - J.pair_off[o] - pc) : 0;
    const int row = pp < np ? J.pairs[J.pair_off[o] + pc + pp].ri - rlo : 0;
    const bool active = pp < np && cb < ncb && row < nrows;
    const int qn = segn / G, qa = grp * qn;            // this group's pixels of a segment
    const int b0 = 2 * blockIdx.y;
    const bool two = b0 + 1 < J.batch;
    float2 acc[GT_LAG];
#pragma unroll
    for (int m = 0; m < GT_LAG; ++m) acc[m] = make_float2(0.0f, 0.0f);
    const int stage_w = segn + GT_LAG * ncb;           // x positions a segment needs per ring
    for (int r = t; r < nrows; r += blockDim.x) xrow[r] = (long long)b0 * J.stride + J.rings[rlo + r].start;
    const int lane = t & 31, nw = blockDim.x >> 5;
    for (int s0 = 0; s0 < n; s0 += segn) {
        __syncthreads();                               // the previous segment is consumed (and xrow is set)
        for (int e = t; e < nout * segn; e += blockDim.x) {
            const int k = e / segn, q = e - k * segn;
            const float *g0 = gy + (long long)b0 * J.stride + J.rings[J.b_lo + rb0 + k].start + s0 + q;
            gys[e] = make_float2(*g0, two ? g0[J.stride] : 0.0f);
        }
        // a warp per staged row, lanes along it (coalesced)
        for (int r = t >> 5; r < nrows; r += nw) {
            const float *xr = J.x + xrow[r];
            float2 *dst = xs + r * LR;
            for (int q = lane; q < stage_w; q += 32) {
                int pos = s0 + q + J.EMIN;             // in (-n, 2n)
                pos = pos < 0 ? pos + n : (pos >= n ? pos - n : pos);
                dst[q] = make_float2(xr[pos], two ? xr[pos + J.stride] : 0.0f);
            }
        }
        __syncthreads();
        if (active) {
            const float2 *xr = xs + row * LR + GT_LAG * cb + qa;
            const float2 *gq = gys + ob * segn + qa;
            float2 w[GT_LAG], a[GT_LAG];
#pragma unroll
            for (int m = 0; m < GT_LAG; ++m) {
                w[m] = xr[m];
                a[m] = make_float2(0.0f, 0.0f);
            }
            // at pixel q + u, offset m reads position q + u + m: slot (u + m) mod 8, slot u
            // taking position q + u + 8 once pixel q + u is done
            for (int q = 0; q < qn; q += GT_LAG) {
#pragma unroll
                for (int u = 0; u < GT_LAG; ++u) {
                    const float2 g = gq[q + u];
#pragma unroll
                    for (int m = 0; m < GT_LAG; ++m) a[m] = __ffma2_rn(g, w[(u + m) % GT_LAG], a[m]);
                    w[u] = xr[q + u + GT_LAG];
                }
            }
#pragma unroll
            for (int m = 0; m < GT_LAG; ++m) acc[m] = __fadd2_rn(acc[m], a[m]);
        }
    }
    if (active) {
#pragma unroll
        for (int m = 0; m < GT_LAG; ++m) {
            const int c = GT_LAG * cb + m;
            if (c < J.WPM) atomicAdd(&C[((size_t)(rb0 + ob) * R2 + pc + pp) * J.WPM + c], acc[m].x + acc[m].y);
        }
    }
}

// Belt rings, step 2: the pairs' node intervals (FP64, once per call) and the bins: a
// thread per (belt ring, input ring, offset) of C.
__global__ void k_grad_belt_bins(const JobDesc J, const float *C, double *acc) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int R2 = 2 * J.HM + 1;
    if (idx >= (long long)J.nb * R2 * J.WPM) return;
    const int c = (int)(idx % J.WPM), pp = (int)((idx / J.WPM) % R2), rb = (int)(idx / ((long long)J.WPM * R2));
    const int o = J.b_lo + rb;
    const int p0 = J.pair_off[o];
    if (pp >= J.pair_off[o + 1] - p0) return;
    const PairInfo P = J.pairs[p0 + pp];
    const int s_o = J.rings[o].s;
    const int e = J.EMIN + c;
    const int ec = (s_o + 1 - P.s_i) >> 1;            // offset of the nearest input pixel
    if (P.W < 0 || e < ec - P.W || e > ec + P.W) return;
    const double2 ab = J.ab64[p0 + pp];
    int k;
    float fr;
    if (pair_kf64((double)(2 * e + P.s_i - s_o) * (SK_PI / (2.0 * (double)J.n4)), ab.x, ab.y, J.kp, J.kd, k, fr)) {
        const double v = (double)C[idx];
        atomicAdd(&acc[k], v * (1.0 - (double)fr));
        atomicAdd(&acc[k + 1], v * (double)fr);
    }
}

__device__ __forceinline__ float dot4(const float *g, float4 h) {
    return fmaf(g[0], h.x, fmaf(g[1], h.y, fmaf(g[2], h.z, g[3] * h.w)));
}

// Cap rings: a thread per base output of a cap item (the forward's items: 256 base
// outputs, taken 32 at a time by a warp), maps four at a time.  The 16 images of the base output (quarter turns,
// hemispheres, reflection; 8 on a symmetry axis) take gy_b from the map, the images of
// the input pixel a come from the symmetric copy H (H[a], H[a + n/4], and the reflection
// b = n/4 - s - a: H[b], H[b + n/4]), in the pairing the forward kernel uses; one (k, f)
// per base pair and four maps (double-float, or FP64).
constexpr int GC = SK_GRAD_CAP_MAPS;     // maps per pass of the cap gradient
__global__ void __launch_bounds__(SK_GRAD_CAP_THREADS, 2)
k_grad_cap(const __grid_constant__ JobsArg A, const float *__restrict__ gy, double *acc, int2 *__restrict__ kfc,
           int kf_steps) {
    extern __shared__ float bins[];
    const JobDesc &J = A.j[0];
    const int nt = J.kp.nt;
    for (int k = threadIdx.x; k < nt; k += blockDim.x) bins[k] = 0.0f;
    __syncthreads();
    // node coordinates in double-float where pair_kf_df applies (uniform nodes, small cut)
    const bool dfpath = J.kp.small_angle && J.kp.layout == 0;
    const KernDF KD{df_from(J.kd.tcut), df_from(J.kd.inv_h)};
    // warps take tasks of 32 base outputs (an eighth of an item) from a queue, in the
    // items' order (heaviest first): no lane waits on a short ring's item, no warp on a
    // block's last item
    const int lane = threadIdx.x & 31;
    // this warp's cache of (k, f), one entry per step of a lane's walk over its windows
    // (kf_steps of them): the first pass over the maps writes it, the others read it
    int2 *const kw = kf_steps > 0
                         ? kfc + ((long long)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kf_steps) * 32 + lane
                         : nullptr;
    for (;;) {
        int task = 0;
        if (lane == 0) task = atomicAdd(A.queue, 1);
        task = __shfl_sync(0xffffffffu, task, 0);
        if (task >= 8 * J.n_items) break;
        const int4 it = J.items[task >> 3];
        const int ro = it.x, j1 = it.y + 32 * (task & 7), jo = j1 + lane;
        const RingDev R = J.rings[ro];
        const int Qo = R.n >> 2;
        const int T = R.s ? (Qo + 1) / 2 : Qo / 2 + 1;
        if (jo >= T) continue;
        const int jr = Qo - jo - R.s;
        const bool refl = jr < Qo && jr >= T;
        const long long so = R.start, ss = J.rings[J.nr - 1 - ro].start;
        for (int b0 = 0; b0 < J.batch; b0 += GC) {
            const int nb = min(GC, J.batch - b0);
            float g[GC][16];
#pragma unroll
            for (int u = 0; u < GC; ++u) {
                // maps past the batch, and the reflected images of an output on a symmetry
                // axis, get gy = 0 (their loads read the base output, which exists)
                const float *yb = gy + (long long)(b0 + (u < nb ? u : 0)) * J.stride;
                const float ok = u < nb ? 1.0f : 0.0f;
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float o2 = (r == 0 || refl) ? ok : 0.0f;
                    const int j = (r == 1 && refl) ? jr : jo;
                    g[u][8 * r + 0] = o2 * yb[so + j];
                    g[u][8 * r + 1] = o2 * yb[so + j + 2 * Qo];
                    g[u][8 * r + 2] = o2 * yb[ss + j];
                    g[u][8 * r + 3] = o2 * yb[ss + j + 2 * Qo];
                    g[u][8 * r + 4] = o2 * yb[so + j + Qo];
                    g[u][8 * r + 5] = o2 * yb[so + j + 3 * Qo];
                    g[u][8 * r + 6] = o2 * yb[ss + j + Qo];
                    g[u][8 * r + 7] = o2 * yb[ss + j + 3 * Qo];
                }
            }
            int s = 0;          // step of the walk
            for (int p = J.pair_off[ro]; p < J.pair_off[ro + 1]; ++p) {
                const PairInfo P = J.pairs[p];
                const int Qi = P.n_i >> 2;
                const float4 *h0 = J.hx + (long long)b0 * J.hstride + J.rings[P.ri].start;
                int jlo, cnt;
                pair_window(jo, R.n, R.s, P, jlo, cnt);
                // the pair's FP64 constants, unless every step of its walk is in the cache
                double2 ab = make_double2(0.0, 0.0);
                double c0 = 0.0;
                PairDF PD{};
                if (!(b0 > 0 && s + cnt <= kf_steps)) {
                    ab = J.ab64[p];
                    c0 = SK_PI / (2.0 * (double)P.n_i * (double)R.n);
                    PD = PairDF{df_from(c0), df_from(ab.x), df_from(ab.y)};
                }
                // Each lane walks its window from its own position (lane mod cnt) and wraps
                // to the window's start: the lanes' outputs are neighbours, so at one position
                // of their windows their pairs mostly fall in one node interval, and the bin
                // updates of a warp would all hit the same two addresses.
                const int r0 = lane % cnt, js = jlo + r0, wrap = cnt - r0;
                long long q = pair_q(js, jo, R.n, R.s, P);
                // pixels a (rising from js, back to jlo after the wrap), a + n/4 and their
                // reflections n/4 - s - a, + n/4 (falling), kept reduced mod n
                const int n_i = P.n_i, hn = n_i >> 1, cm = cnt % n_i;
                int pa = js % n_i; if (pa < 0) pa += n_i;
                int pb = pa + Qi; if (pb >= n_i) pb -= n_i;
                int pc = (Qi - P.s_i - js) % n_i; if (pc < 0) pc += n_i;
                int pd = pc + Qi; if (pd >= n_i) pd -= n_i;
                for (int m = 0; m < cnt; ++m, ++s, q += 2 * R.n) {
                    if (m == wrap) {        // back to the window's first pixel
                        q -= 2LL * R.n * cnt;
                        pa -= cm; if (pa < 0) pa += n_i;
                        pb -= cm; if (pb < 0) pb += n_i;
                        pc += cm; if (pc >= n_i) pc -= n_i;
                        pd += cm; if (pd >= n_i) pd -= n_i;
                    }
                    const int ia = (pa & 1) * hn + (pa >> 1), ib = (pb & 1) * hn + (pb >> 1);
                    const int ic = (pc & 1) * hn + (pc >> 1), id = (pd & 1) * hn + (pd >> 1);
                    pa = pa + 1 == n_i ? 0 : pa + 1;
                    pb = pb + 1 == n_i ? 0 : pb + 1;
                    pc = pc == 0 ? n_i - 1 : pc - 1;
                    pd = pd == 0 ? n_i - 1 : pd - 1;
                    int k = -1;
                    float fr = 0.0f;
                    bool hit;
                    if (b0 > 0 && s < kf_steps) {
                        const int2 c = __ldcg(kw + (long long)s * 32);
                        k = c.x;
                        fr = __int_as_float(c.y);
                        hit = k >= 0;
                    } else {
                        // |q| < 2^24 on the cap windows (checked when the plan was built): exact in FP32
                        const int in = dfpath ? pair_kf_df((float)q, PD, KD, J.kp, k, fr) : -1;
                        hit = in > 0 || (in < 0 && pair_kf64((double)q * c0, ab.x, ab.y, J.kp, J.kd, k, fr));
                        if (b0 == 0 && s < kf_steps)
                            __stcg(kw + (long long)s * 32, make_int2(hit ? k : -1, __float_as_int(hit ? fr : 0.0f)));
                    }
                    if (!hit) continue;
                    float v = 0.0f;
#pragma unroll
                    for (int u = 0; u < GC; ++u) {
                        if (u >= nb) break;
                        const float4 *h = h0 + (long long)u * J.hstride;
                        v += dot4(&g[u][0], __ldg(h + ia)) + dot4(&g[u][4], __ldg(h + ib)) +
                             dot4(&g[u][8], __ldg(h + ic)) + dot4(&g[u][12], __ldg(h + id));
                    }
                    atomicAdd(&bins[k], v - fr * v);
                    atomicAdd(&bins[k + 1], fr * v);
                }
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nt; k += blockDim.x)
        if (bins[k] != 0.0f) atomicAdd(&acc[k], (double)bins[k]);
}

__global__ void k_grad_finish(const double *acc, int nt, double scale, float *out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nt) out[k] = (float)(acc[k] * scale);
}

}  // namespace

cudaError_t sk_launch_grad_general(const JobsArg &a, const float *gy, double *acc, int grid,
                                   cudaStream_t st) {
    if (a.n_jobs <= 0 || a.j[0].batch <= 0) return cudaSuccess;
    const size_t smem = (size_t)a.j[0].kp.nt * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_grad_general, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_grad_general<<<grid, 128, smem, st>>>(a, gy, acc);
    return cudaGetLastError();
}

size_t sk_grad_belt_floats(const JobDesc &j) { return (size_t)j.nb * (2 * j.HM + 1) * j.WPM; }

cudaError_t sk_launch_grad_belt(const JobDesc &j, const float *gy, float *C, double *acc, const int *h_lo,
                                const int *h_np, cudaStream_t st) {
    if (j.nb <= 0 || j.batch <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(C, 0, sizeof(float) * sk_grad_belt_floats(j), st);
    if (e != cudaSuccess) return e;
    // window positions per block (RC), output rings per block (OB) and pixel groups (G): a
    // thread per (output, group, position, 8 offsets), at most 512; the staged rows of a
    // block (its outputs' windows at the chunk, NR at most) in about 200 KB of shared memory
    const int R2 = 2 * j.HM + 1, ncb = (j.WPM + GT_LAG - 1) / GT_LAG;
    const int segn = j.n4 < GT_SEG ? j.n4 : GT_SEG;
    const size_t row = sizeof(float2) * (size_t)gt_row(segn, ncb) + sizeof(long long);
    const size_t smem_max = 200 * 1024;
    if (ncb > 512) return cudaErrorInvalidConfiguration;
    int RC = R2 * ncb > 512 ? 512 / ncb : R2;
    int OB = 4;
    auto rows_needed = [&](int ob, int rc) {           // max over blocks of the staged rows
        int nr = 1;
        for (int rb0 = 0; rb0 < j.nb; rb0 += ob)
            for (int pc = 0; pc < R2; pc += rc) {
                int lo = 1 << 30, hi = -1;
                for (int k = 0; k < ob && rb0 + k < j.nb; ++k) {
                    const int a = pc, z = (pc + rc < h_np[rb0 + k] ? pc + rc : h_np[rb0 + k]) - 1;
                    if (a <= z) {
                        lo = lo < h_lo[rb0 + k] + a ? lo : h_lo[rb0 + k] + a;
                        hi = hi > h_lo[rb0 + k] + z ? hi : h_lo[rb0 + k] + z;
                    }
                }
                if (hi >= lo && hi - lo + 1 > nr) nr = hi - lo + 1;
            }
        return nr;
    };
    int tpg = (RC * ncb + 31) / 32 * 32;
    while (OB > 1 && OB * tpg > 512) --OB;
    int NR = rows_needed(OB, RC);
    while (sizeof(float2) * OB * segn + row * NR > smem_max && (OB > 1 || RC > 1)) {
        if (OB > 1) --OB;
        else RC = RC > 1 ? RC / 2 : 1;
        tpg = (RC * ncb + 31) / 32 * 32;
        NR = rows_needed(OB, RC);
    }
    if (sizeof(float2) * OB * segn + row * NR > smem_max) return cudaErrorInvalidConfiguration;
    int G = 512 / (OB * tpg);
    G = G > 4 ? 4 : (G < 1 ? 1 : G);
    while (G > 1 && (segn % (8 * G)) != 0) --G;
    const size_t smem = sizeof(float2) * OB * segn + row * NR;
    e = cudaFuncSetAttribute(k_grad_belt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((j.nb + OB - 1) / OB, (j.batch + 1) / 2, (R2 + RC - 1) / RC);
    k_grad_belt<<<grid, OB * G * tpg, smem, st>>>(j, gy, C, RC, G, OB, NR);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long nbins = (long long)sk_grad_belt_floats(j);
    k_grad_belt_bins<<<(unsigned)((nbins + 255) / 256), 256, 0, st>>>(j, C, acc);
    return cudaGetLastError();
}

cudaError_t sk_launch_grad_cap(const JobsArg &a, const float *gy, double *acc, int grid, int2 *kfc, int kf_steps,
                               cudaStream_t st) {
    if (a.n_jobs <= 0 || a.j[0].batch <= 0 || a.j[0].n_items <= 0) return cudaSuccess;
    const size_t smem = (size_t)a.j[0].kp.nt * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_grad_cap, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (!a.queue) return cudaErrorInvalidValue;       // the task queue (zeroed by the caller)
    if (kf_steps > 0 && !kfc) return cudaErrorInvalidValue;
    k_grad_cap<<<grid, SK_GRAD_CAP_THREADS, smem, st>>>(a, gy, acc, kfc, kf_steps);
    return cudaGetLastError();
}

cudaError_t sk_launch_grad_finish(const double *acc, int nt, double scale, float *out, cudaStream_t st) {
    k_grad_finish<<<(nt + 255) / 256, 256, 0, st>>>(acc, nt, scale, out);
    return cudaGetLastError();
}
