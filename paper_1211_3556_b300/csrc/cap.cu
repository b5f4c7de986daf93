// cap.cu -- polar-cap path: one weight evaluation shared by up to 16 symmetric pairs.
//
// The HEALPix pixelisation is invariant under
//   * a quarter turn in phi (pixel j -> j + n/4 on every ring),
//   * the reflection phi -> pi/2 - phi (pixel j -> n/4 - j - s on a ring whose
//     pixels sit at phi = pi (2j + s) / n),
//   * the mirror about the equator (ring r <-> ring 4N - r, same phis),
// and the angle between two pixel centres is invariant under all three.  So a
// pair (o, i) and its images have the same weight dOmega K_lin(gamma).  A
// thread owns one "base" output of the first half quarter of a northern ring,
// evaluates the weight of each window pair once (the per-pair formula:
// chord from A + B sin^2(dphi/2), asin series, table lerp), and applies it to
// the 16 images: 4 quarter turns x 2 hemispheres x {pair, reflected pair}.
// Outputs on a symmetry axis (phi = 0 or pi/4) are their own reflections (or
// a quarter turn of it): they keep the 8 images without reflection, so no
// output is written twice.  Same operator as the per-pair path (Sec. 2, Eq. 1
// with the tabulated kernel of Sec. 3); only the order of work differs.
//
// Work item: (northern output ring, first base pixel) for CT base outputs,
// CT / 2 threads, each owning two adjacent base outputs jA, jB = jA + 1; a
// block runs two work items side by side (each half with its own named
// barrier), so that they share one copy of the node table.  For every input
// ring of the window a half stages 4 rows (quarter turns) of float4 (north
// pixel, its reflection, south pixel, its reflection) covering the union of
// its CT windows, unwrapped, even positions before odd ones, with cp.async
// into two buffers (ring p + 1 is copied while ring p is summed; one barrier
// per ring).  A thread
// walks the union of its two windows (they start at most a pixel or two
// apart): one 128-bit load feeds 4 of the 16 images of both outputs, and both
// weights come from one paired evaluation (fma.rn.f32x2: two IEEE
// operations).  The node values V_k dOmega sit in shared memory (FP32, the
// slope formed on the fly): the lanes of a warp look up nodes spread over a
// few hundred entries, a gather that costs a few bank wavefronts from shared
// memory but one L1 wavefront per distinct line from global memory.
#include "skconv.h"
#include "skconv_internal.cuh"
#include "skconv_launch.h"

namespace {

constexpr int CT = SK_CAP_CT;       // base outputs per work item
constexpr int NTH = CT / 2;         // threads per work item: two adjacent base outputs each
constexpr int HALVES = SK_CAP_ITEMS_PER_BLOCK;   // work items in flight per block (one node table)
// strip buffers per work item: two (stage ring p + 1 while ring p is summed) where they fit
template <int LS>
__host__ __device__ constexpr int cap_bufs() { return LS <= 320 ? 2 : 1; }

__device__ __forceinline__ void half_sync(int half) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + half), "r"(NTH) : "memory");
}

__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
    uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Nearest input pixel of output jo: floor(num / (2 n_o)) with num below 2^31
// (in the caps jo < n_o / 4 <= 2 Nside and n_i <= 4 Nside <= 32768), by the
// item's multiply-high constants for the divisor 2 n_o: mg = ceil(2^(31+l) / d),
// l = ceil(log2 d), quotient = umulhi(num, mg) >> (l - 1), exact for every
// num < 2^31 (Granlund and Montgomery 1994, Thm 4.2).
__device__ __forceinline__ int centre_of(int jo, int n_o, int s_o, const PairInfo &P, unsigned mg, int sh) {
    const unsigned num = (unsigned)(2 * jo + s_o) * (unsigned)P.n_i + (unsigned)(1 - P.s_i) * (unsigned)n_o;
    return (int)(__umulhi(num, mg) >> sh);
}

// q of window pixel jlo (may be negative) for output jo: both products are below 2^31.
__device__ __forceinline__ int q_of(int jlo, int jo, int n_o, int s_o, const PairInfo &P) {
    return (2 * jlo + P.s_i) * n_o - (2 * jo + s_o) * P.n_i;
}

// Window start relative to the centre, and length, of input ring P.
__device__ __forceinline__ void win_shape(const PairInfo &P, int &before, int &cnt) {
    if (P.W < 0) { before = (P.n_i - 1) / 2; cnt = P.n_i; }
    else         { before = P.W; cnt = 2 * P.W + 1; }
}

// Base outputs of a quarter ring of Q pixels with shift s: [0, T).
__device__ __forceinline__ int base_count(int Q, int s) { return s ? (Q + 1) / 2 : Q / 2 + 1; }

// Strip layout of one row: even positions first, then odd ones.  A lane owns
// two adjacent outputs, so at one step the lanes of a warp read positions about
// two apart; with this layout they read consecutive float4 (one parity) instead
// of every other one.
template <int LS>
__device__ __forceinline__ int split_index(int m) { return (m & 1) * (LS / 2) + (m >> 1); }

// Stage row k, element m = (xN[a], xN[b], xS[a], xS[b]) with a = u0 + m + kQ and
// b = Q - s - (u0 + m) + kQ (indices mod n): the pixel and its reflection on the
// northern ring and on its southern mirror, at split_index(m).
template <int LS>
__device__ __forceinline__ void stage_ring(float4 *buf, const JobDesc &J, const float *xmap,
                                           const PairInfo &P, int ri_south, int u0, int L, int t) {
    const int n = P.n_i, Q = n >> 2, s = P.s_i;
    const float *xn = xmap + J.rings[P.ri].start, *xs = xmap + J.rings[ri_south].start;
    float *b = reinterpret_cast<float *>(buf);
    // first element of this thread, reduced into [0, n) (u0 > -n, the offsets stay below 2n + NTH)
    int io0 = u0 + t;
    while (io0 < 0) io0 += n;
    while (io0 >= n) io0 -= n;
    int ir0 = Q - s - u0 - t;
    while (ir0 < 0) ir0 += n;
    while (ir0 >= n) ir0 -= n;
    for (int k = 0; k < 4; ++k) {
        int io = io0 + k * Q, ir = ir0 + k * Q;
        if (io >= n) io -= n;
        if (ir >= n) ir -= n;
        for (int m = t; m < L; m += NTH) {
            float *d = b + 4 * (k * LS + split_index<LS>(m));
            cp_async4(d, xn + io);
            cp_async4(d + 1, xn + ir);
            cp_async4(d + 2, xs + io);
            cp_async4(d + 3, xs + ir);
            io += NTH;
            while (io >= n) io -= n;
            ir -= NTH;
            while (ir < 0) ir += n;
        }
    }
}

// acc[k] += w (v.x, v.y), acc[4 + k] += w (v.z, v.w) for the staged pixel m of
// each quarter turn k: (north pair, north reflected), (south pair, south reflected).
template <int LS>
__device__ __forceinline__ void mac16(float2 *acc, float w, const float4 *xs, int m) {
    const float2 ww = f2(w);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 v = xs[k * LS + m];
        acc[k] = __ffma2_rn(ww, make_float2(v.x, v.y), acc[k]);
        acc[4 + k] = __ffma2_rn(ww, make_float2(v.z, v.w), acc[4 + k]);
    }
}

template <int LS, int MODE>
__global__ void __launch_bounds__(NTH * HALVES)
k_conv_cap(const __grid_constant__ JobsArg A) {
    constexpr bool SERIES = (MODE & 1) != 0, SMALLA = (MODE & 2) != 0, BIASED = (MODE & 4) != 0;
    constexpr int NB = cap_bufs<LS>();
    // [HALVES][NB][4][LS] strip rows, then the node values (one table: every job of a launch
    // uses the same kernel table)
    extern __shared__ __align__(16) float4 sx[];
    float *stab = reinterpret_cast<float *>(sx + HALVES * NB * 4 * LS);
    for (int k = threadIdx.x; k < A.j[0].kp.nt; k += NTH * HALVES) stab[k] = A.j[0].tab[k].x;
    __syncthreads();
    const int half = threadIdx.x / NTH, t = threadIdx.x % NTH;
    float4 *const sbuf = sx + half * NB * 4 * LS;
    // work queue: each half takes the next item (items are ordered heaviest first), so the
    // halves that drew light items take more of them and all finish together
    __shared__ int s_item[HALVES];
    for (;;) {
        if (t == 0) s_item[half] = atomicAdd(A.queue, 1);
        half_sync(half);
        const int f = s_item[half];
        if (f >= A.total) break;
        const JobDesc &J = A.j[sk_find_job(A, f)];
        const int local = f - J.flat_base;
        const int map = local / J.n_items;
        const int4 it = J.items[local - map * J.n_items];
        const int ro = it.x, j0 = it.y;
        const unsigned mg = (unsigned)it.z;            // division by 2 n_o (centre_of)
        const int sh = it.w;
        const RingDev R = J.rings[ro];
        const int Qo = R.n >> 2;
        const int T = base_count(Qo, R.s);
        const int jlast = min(j0 + CT - 1, T - 1);
        const int jA = j0 + 2 * t, jB = jA + 1;
        const bool actA = jA < T, actB = jB < T;
        const int jrA = Qo - jA - R.s, jrB = Qo - jB - R.s;   // reflections in the quarter
        const bool reflA = actA && jrA < Qo && jrA >= T;
        const bool reflB = actB && jrB < Qo && jrB >= T;
        const int ro_s = J.nr - 1 - ro;
        const float *xmap = J.x + (long long)map * J.stride;
        const int p0 = J.pair_off[ro], p1 = J.pair_off[ro + 1];

        // accX[k] = (north pair, north reflected), accX[4 + k] = (south pair, south
        // reflected) of quarter turn k, for outputs jA and jB
        float2 accA[8], accB[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) { accA[s] = make_float2(0.0f, 0.0f); accB[s] = make_float2(0.0f, 0.0f); }

        auto stage = [&](int p, float4 *dst) {
            const PairInfo Pn = J.pairs[p];
            int before, cnt;
            win_shape(Pn, before, cnt);
            const int c0 = centre_of(j0, R.n, R.s, Pn, mg, sh), c1 = centre_of(jlast, R.n, R.s, Pn, mg, sh);
            stage_ring<LS>(dst, J, xmap, Pn, J.nr - 1 - Pn.ri, c0 - before, c1 - c0 + cnt, t);
            cp_commit();
        };
        if (NB == 2) stage(p0, sbuf);
        for (int p = p0; p < p1; ++p) {
            float4 *const xbuf = sbuf + (NB == 2 ? ((p - p0) & 1) : 0) * 4 * LS;
            if (NB == 2) {
                // ring p's copies (issued during ring p - 1) are complete for this thread; after
                // the barrier they are for every thread, and every thread is done with ring
                // p - 1, whose buffer then receives ring p + 1 while ring p is summed
                cp_wait0();
                half_sync(half);
                if (p + 1 < p1) stage(p + 1, sbuf + ((p + 1 - p0) & 1) * 4 * LS);
            } else {
                // one buffer: stage ring p once every thread is done with ring p - 1
                half_sync(half);
                stage(p, xbuf);
                cp_wait0();
                half_sync(half);
            }
            if (actA) {
                const PairInfo P = J.pairs[p];
                int before, cnt;
                win_shape(P, before, cnt);
                const int cb = centre_of(j0, R.n, R.s, P, mg, sh);
                const int cA = centre_of(jA, R.n, R.s, P, mg, sh);
                const int dl = actB ? centre_of(jB, R.n, R.s, P, mg, sh) - cA : 0;   // 0, 1 or 2
                const int cnt_u = cnt + dl;             // union of the two windows, from A's start
                // |q| < 2^24 on these windows (checked when the plan was built): exact in FP32
                const float qA0 = (float)q_of(cA - before, jA, R.n, R.s, P);
                const float dqo = (float)(2 * R.n);     // q step per input pixel
                const float dqi = (float)(2 * P.n_i);   // q of output jA minus q of output jB
                const float4 *xrow = xbuf;
                const int pA = cA - cb;                 // strip position of the union's first pixel
                if (SERIES) {
                    // narrow windows only: a pixel of the union outside one output's window is
                    // outside its cut, and the cut test gives it weight 0.  Pixels go in pairs
                    // (pA + m, pA + m + 1): one of each parity, at x0[i] and x1[i], i = m / 2.
                    const float4 *x0 = xrow + split_index<LS>(pA);
                    const float4 *x1 = xrow + split_index<LS>(pA + 1);
                    float2 q = make_float2(qA0, qA0 - dqi);   // q of pixel m for outputs (A, B)
#pragma unroll 1
                    for (int m = 0; m < cnt_u; m += 2) {
                        const int i = m >> 1;
                        const float2 q1 = __fadd2_rn(q, f2(dqo));
                        const float2 w0 = fast_weight2<SMALLA, BIASED>(__fmul2_rn(q, f2(P.c0)), P.A, P.B, J.kp, stab);
                        const float2 w1 = fast_weight2<SMALLA, BIASED>(__fmul2_rn(q1, f2(P.c0)), P.A, P.B, J.kp, stab);
                        q = __fadd2_rn(q1, f2(dqo));
                        mac16<LS>(accA, w0.x, x0, i);
                        mac16<LS>(accB, w0.y, x0, i);
                        if (m + 1 < cnt_u) {
                            mac16<LS>(accA, w1.x, x1, i);
                            mac16<LS>(accB, w1.y, x1, i);
                        }
                    }
                } else {
                    // windows may be whole rings: restrict each output to its own window
                    for (int m = 0; m < cnt_u; ++m) {
                        const float qa = fmaf((float)m, dqo, qA0);
                        float wa = fast_weight<SERIES, SMALLA, BIASED>(qa * P.c0, P.A, P.B, J.kp, stab);
                        float wb = fast_weight<SERIES, SMALLA, BIASED>((qa - dqi) * P.c0, P.A, P.B, J.kp, stab);
                        wa = m < cnt ? wa : 0.0f;
                        wb = m >= dl ? wb : 0.0f;
                        const float4 *xm = xrow + split_index<LS>(pA + m);
                        mac16<LS>(accA, wa, xm, 0);
                        mac16<LS>(accB, wb, xm, 0);
                    }
                }
            }
        }
        // the next item stages into this half's buffers: everyone must be done reading them
        half_sync(half);
        float *yn = J.y + (long long)map * J.stride + R.start;
        float *ys = J.y + (long long)map * J.stride + J.rings[ro_s].start;
        if (actA) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                yn[jA + k * Qo] = accA[k].x;
                ys[jA + k * Qo] = accA[4 + k].x;
            }
            if (reflA) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    yn[jrA + k * Qo] = accA[k].y;
                    ys[jrA + k * Qo] = accA[4 + k].y;
                }
            }
        }
        if (actB) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                yn[jB + k * Qo] = accB[k].x;
                ys[jB + k * Qo] = accB[4 + k].x;
            }
            if (reflB) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    yn[jrB + k * Qo] = accB[k].y;
                    ys[jrB + k * Qo] = accB[4 + k].y;
                }
            }
        }
    }
}

size_t cap_smem(int LS, int nt) {
    const int nb = LS <= 320 ? 2 : 1;         // cap_bufs<LS>()
    return (size_t)HALVES * nb * 4 * LS * sizeof(float4) + (size_t)nt * sizeof(float);
}

int max_nt(const JobsArg &a) {
    int m = 2;
    for (int j = 0; j < a.n_jobs; ++j) m = a.j[j].kp.nt > m ? a.j[j].kp.nt : m;
    return m;
}

template <int LS, int MODE>
cudaError_t launch_lm(const JobsArg &a, int grid, cudaStream_t st) {
    const size_t smem = cap_smem(LS, max_nt(a));
    cudaError_t e = cudaFuncSetAttribute(k_conv_cap<LS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_conv_cap<LS, MODE><<<grid, NTH * HALVES, smem, st>>>(a);
    return cudaGetLastError();
}

template <int LS, int MODE>
int occupancy_lm(int nt) {
    const size_t smem = cap_smem(LS, nt);
    cudaFuncSetAttribute(k_conv_cap<LS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_conv_cap<LS, MODE>, NTH * HALVES, smem);
    return nb;
}

template <int LS>
cudaError_t launch_ls(const JobsArg &a, int mode, int grid, cudaStream_t st) {
    switch (mode) {
        case 0: return launch_lm<LS, 0>(a, grid, st);
        case 1: return launch_lm<LS, 1>(a, grid, st);
        case 2: return launch_lm<LS, 2>(a, grid, st);
        case 3: return launch_lm<LS, 3>(a, grid, st);
        case 4: return launch_lm<LS, 4>(a, grid, st);
        case 5: return launch_lm<LS, 5>(a, grid, st);
        case 6: return launch_lm<LS, 6>(a, grid, st);
        case 7: return launch_lm<LS, 7>(a, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int LS>
int occupancy_ls(int mode, int nt) {
    switch (mode) {
        case 0: return occupancy_lm<LS, 0>(nt);
        case 1: return occupancy_lm<LS, 1>(nt);
        case 2: return occupancy_lm<LS, 2>(nt);
        case 3: return occupancy_lm<LS, 3>(nt);
        case 4: return occupancy_lm<LS, 4>(nt);
        case 5: return occupancy_lm<LS, 5>(nt);
        case 6: return occupancy_lm<LS, 6>(nt);
        case 7: return occupancy_lm<LS, 7>(nt);
        default: return 0;
    }
}

}  // namespace

cudaError_t sk_launch_conv_cap(const JobsArg &a, int ls, int mode, int grid, cudaStream_t st) {
    if (a.total <= 0) return cudaSuccess;
    switch (ls) {
        case SK_CAP_LS[0]: return launch_ls<SK_CAP_LS[0]>(a, mode, grid, st);
        case SK_CAP_LS[1]: return launch_ls<SK_CAP_LS[1]>(a, mode, grid, st);
        case SK_CAP_LS[2]: return launch_ls<SK_CAP_LS[2]>(a, mode, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

int sk_cap_blocks_per_sm(int ls, int mode, int nt) {
    switch (ls) {
        case SK_CAP_LS[0]: return occupancy_ls<SK_CAP_LS[0]>(mode, nt);
        case SK_CAP_LS[1]: return occupancy_ls<SK_CAP_LS[1]>(mode, nt);
        case SK_CAP_LS[2]: return occupancy_ls<SK_CAP_LS[2]>(mode, nt);
        default: return 0;
    }
}
