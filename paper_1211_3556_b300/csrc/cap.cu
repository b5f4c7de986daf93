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
// Work item: (northern output ring, first base pixel) for CT base outputs.
// For every input ring of the window the block stages 4 rows (quarter turns) of
// float4 (north pixel, its reflection, south pixel, its reflection) covering
// the union of the CT windows, unwrapped, with cp.async, double-buffered; one
// 128-bit load then feeds 4 of the 16 images.  The node values V_k dOmega sit
// in shared memory (FP32, the slope formed on the fly): the lanes of a warp
// look up nodes spread over a few hundred entries, a gather that costs a few
// bank wavefronts from shared memory but one L1 wavefront per distinct line
// from global memory.
#include "skconv.h"
#include "skconv_internal.cuh"
#include "skconv_launch.h"

namespace {

constexpr int CT = SK_CAP_CT;

__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
    uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
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

// Stage row k, element m = (xN[a], xN[b], xS[a], xS[b]) with a = u0 + m + kQ and
// b = Q - s - (u0 + m) + kQ (indices mod n): the pixel and its reflection on the
// northern ring and on its southern mirror.
template <int LS>
__device__ __forceinline__ void stage_ring(float4 *buf, const JobDesc &J, const float *xmap,
                                           const PairInfo &P, int ri_south, int u0, int L) {
    const int n = P.n_i, Q = n >> 2, s = P.s_i;
    const float *xn = xmap + J.rings[P.ri].start, *xs = xmap + J.rings[ri_south].start;
    float *b = reinterpret_cast<float *>(buf);
    // first element of this thread, reduced into [0, n) (u0 > -n, the offsets stay below 2n + CT)
    int io0 = u0 + (int)threadIdx.x;
    while (io0 < 0) io0 += n;
    while (io0 >= n) io0 -= n;
    int ir0 = Q - s - u0 - (int)threadIdx.x;
    while (ir0 < 0) ir0 += n;
    while (ir0 >= n) ir0 -= n;
    for (int k = 0; k < 4; ++k) {
        int io = io0 + k * Q, ir = ir0 + k * Q;
        if (io >= n) io -= n;
        if (ir >= n) ir -= n;
        for (int m = threadIdx.x; m < L; m += CT) {
            float *d = b + 4 * (k * LS + m);
            cp_async4(d, xn + io);
            cp_async4(d + 1, xn + ir);
            cp_async4(d + 2, xs + io);
            cp_async4(d + 3, xs + ir);
            io += CT;
            while (io >= n) io -= n;
            ir -= CT;
            while (ir < 0) ir += n;
        }
    }
}

template <int LS, int MODE>
__global__ void __launch_bounds__(CT)
k_conv_cap(const __grid_constant__ JobsArg A) {
    constexpr bool SERIES = (MODE & 1) != 0, SMALLA = (MODE & 2) != 0, BIASED = (MODE & 4) != 0;
    extern __shared__ __align__(16) float4 sx[];      // [2][4][LS] strips, then the node values
    float *stab = reinterpret_cast<float *>(sx + 2 * 4 * LS);
    const int t = threadIdx.x;
    int cur_job = -1;
    for (int f = blockIdx.x; f < A.total; f += gridDim.x) {
        const int jn = sk_find_job(A, f);
        const JobDesc &J = A.j[jn];
        if (jn != cur_job) {                 // uniform across the block
            __syncthreads();
            for (int k = t; k < J.kp.nt; k += CT) stab[k] = J.tab[k].x;
            __syncthreads();
            cur_job = jn;
        }
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
        const int jo = j0 + t;
        const bool active = jo < T;
        const int jr = Qo - jo - R.s;                       // reflection of jo in the quarter
        const bool refl = active && jr < Qo && jr >= T;
        const int ro_s = J.nr - 1 - ro;
        const float *xmap = J.x + (long long)map * J.stride;
        const int p0 = J.pair_off[ro], p1 = J.pair_off[ro + 1];

        // acc2[k] = (north pair, north reflected), acc2[4 + k] = (south pair, south reflected)
        // of quarter turn k
        float2 acc2[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) acc2[s] = make_float2(0.0f, 0.0f);

        {
            const PairInfo P = J.pairs[p0];
            int before, cnt;
            win_shape(P, before, cnt);
            const int c0 = centre_of(j0, R.n, R.s, P, mg, sh), c1 = centre_of(jlast, R.n, R.s, P, mg, sh);
            stage_ring<LS>(sx, J, xmap, P, J.nr - 1 - P.ri, c0 - before, c1 - c0 + cnt);
            cp_commit();
        }
        for (int p = p0; p < p1; ++p) {
            const int buf = (p - p0) & 1;
            if (p + 1 < p1) {
                const PairInfo Pn = J.pairs[p + 1];
                int before, cnt;
                win_shape(Pn, before, cnt);
                const int c0 = centre_of(j0, R.n, R.s, Pn, mg, sh), c1 = centre_of(jlast, R.n, R.s, Pn, mg, sh);
                stage_ring<LS>(sx + (buf ^ 1) * 4 * LS, J, xmap, Pn, J.nr - 1 - Pn.ri, c0 - before,
                               c1 - c0 + cnt);
            }
            cp_commit();
            cp_wait1();
            __syncthreads();
            if (active) {
                const PairInfo P = J.pairs[p];
                int before, cnt;
                win_shape(P, before, cnt);
                const int cb = centre_of(j0, R.n, R.s, P, mg, sh);
                const int c = centre_of(jo, R.n, R.s, P, mg, sh);
                // |q| < 2^24 on this window (checked when the plan was built): qf + m dq is exact
                const float qf = (float)q_of(c - before, jo, R.n, R.s, P);
                const float dq = (float)(2 * R.n);
                const float4 *xs = sx + buf * 4 * LS + (c - cb);
                int m = 0;
                if (SERIES) {
                    // two window pixels per step in paired FP32 arithmetic
                    float2 mm = make_float2(0.0f, 1.0f);
                    for (; m + 1 < cnt; m += 2) {
                        const float2 w = fast_weight2<SMALLA, BIASED>(
                            __fmul2_rn(__ffma2_rn(mm, f2(dq), f2(qf)), f2(P.c0)), P.A, P.B, J.kp, stab);
                        mm = __fadd2_rn(mm, f2(2.0f));
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float2 wh = f2(h ? w.y : w.x);
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const float4 v = xs[k * LS + m + h];
                                acc2[k] = __ffma2_rn(wh, make_float2(v.x, v.y), acc2[k]);        // north: pair, reflected
                                acc2[4 + k] = __ffma2_rn(wh, make_float2(v.z, v.w), acc2[4 + k]);  // south: pair, reflected
                            }
                        }
                    }
                }
                for (; m < cnt; ++m) {
                    const float2 w = f2(fast_weight<SERIES, SMALLA, BIASED>(fmaf((float)m, dq, qf) * P.c0, P.A, P.B,
                                                                            J.kp, stab));
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float4 v = xs[k * LS + m];
                        acc2[k] = __ffma2_rn(w, make_float2(v.x, v.y), acc2[k]);
                        acc2[4 + k] = __ffma2_rn(w, make_float2(v.z, v.w), acc2[4 + k]);
                    }
                }
            }
            __syncthreads();
        }
        if (active) {
            float *yn = J.y + (long long)map * J.stride + R.start;
            float *ys = J.y + (long long)map * J.stride + J.rings[ro_s].start;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                yn[jo + k * Qo] = acc2[k].x;
                ys[jo + k * Qo] = acc2[4 + k].x;
            }
            if (refl) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    yn[jr + k * Qo] = acc2[k].y;
                    ys[jr + k * Qo] = acc2[4 + k].y;
                }
            }
        }
    }
}

size_t cap_smem(int LS, int nt) { return (size_t)2 * 4 * LS * sizeof(float4) + (size_t)nt * sizeof(float); }

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
    k_conv_cap<LS, MODE><<<grid, CT, smem, st>>>(a);
    return cudaGetLastError();
}

template <int LS, int MODE>
int occupancy_lm(int nt) {
    const size_t smem = cap_smem(LS, nt);
    cudaFuncSetAttribute(k_conv_cap<LS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_conv_cap<LS, MODE>, CT, smem);
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
