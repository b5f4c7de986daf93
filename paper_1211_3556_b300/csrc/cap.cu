// cap.cu -- polar-cap path: per-pair weights shared by the 8 symmetric images.
//
// Every HEALPix ring is invariant under a quarter turn in phi (pixel j ->
// j + n/4) and the pixelisation is mirror-symmetric about the equator (ring r
// <-> ring 4N - r with the same pixel phis).  So the pair (o, i) and its images
// under the 4 rotations and the mirror have the same angle and the same
// weight dOmega K_lin(gamma).  A thread owns one output pixel in the first
// quarter of a northern ring and the 7 images of it, evaluates each pair's
// weight once (chord, asin series, table lerp -- the per-pair formula of the
// general path) and applies it with 8 FFMAs.  Same operator as the per-pair
// path (the real-space convolution of Sec. 2, Eq. 1, tabulated kernel of
// Sec. 3); only the order of work differs.
//
// Work item: (northern output ring, first quarter-ring pixel) for 128 outputs.
// For each input ring of the window the block stages 8 strips (4 rotations x
// 2 hemispheres, each the union of the 128 outputs' phi windows, unwrapped)
// into shared memory with cp.async, double-buffered; a strip row has LS
// floats, so the 8 images of one input pixel sit at fixed offsets k * LS.
#include "skconv.h"
#include "skconv_internal.cuh"
#include "skconv_launch.h"

namespace {

constexpr int CT = 128;

__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
    uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ int centre_of(int jo, int n_o, int s_o, const PairInfo &P) {
    long long num = (long long)(2 * jo + s_o) * P.n_i + (long long)(1 - P.s_i) * n_o;
    return (int)(num / (2LL * n_o));
}

// Window start relative to the centre, and length, of input ring P.
__device__ __forceinline__ void win_shape(const PairInfo &P, int &before, int &cnt) {
    if (P.W < 0) { before = (P.n_i - 1) / 2; cnt = P.n_i; }
    else         { before = P.W; cnt = 2 * P.W + 1; }
}

template <int LS>
__device__ __forceinline__ void stage_ring(float *buf, const JobDesc &J, const float *xmap,
                                           const PairInfo &P, int ri_south, int u0, int L) {
    const int n = P.n_i, Q = n >> 2;
    const long long st_n = J.rings[P.ri].start, st_s = J.rings[ri_south].start;
    for (int k = 0; k < 4; ++k) {
        int idx = (u0 + (int)threadIdx.x + k * Q) % n;
        if (idx < 0) idx += n;
        for (int m = threadIdx.x; m < L; m += CT) {
            cp_async4(buf + k * LS + m, xmap + st_n + idx);
            cp_async4(buf + (4 + k) * LS + m, xmap + st_s + idx);
            idx += CT;
            while (idx >= n) idx -= n;
        }
    }
}

template <int LS>
__global__ void __launch_bounds__(CT)
k_conv_cap(const __grid_constant__ JobsArg A) {
    extern __shared__ __align__(16) float sx[];       // [2][8][LS]
    const int t = threadIdx.x;
    for (int f = blockIdx.x; f < A.total; f += gridDim.x) {
        const JobDesc &J = A.j[sk_find_job(A, f)];
        const int local = f - J.flat_base;
        const int map = local / J.n_items;
        const int4 it = J.items[local - map * J.n_items];
        const int ro = it.x, j0 = it.y;
        const RingDev R = J.rings[ro];
        const int Qo = R.n >> 2;
        const int jlast = min(j0 + CT - 1, Qo - 1);
        const int jo = j0 + t;
        const bool active = jo < Qo;
        const int ro_s = J.nr - 1 - ro;
        const float *xmap = J.x + (long long)map * J.stride;
        const int p0 = J.pair_off[ro], p1 = J.pair_off[ro + 1];

        float acc[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) acc[s] = 0.0f;

        // prologue: stage the first input ring
        {
            const PairInfo P = J.pairs[p0];
            int before, cnt;
            win_shape(P, before, cnt);
            const int c0 = centre_of(j0, R.n, R.s, P), c1 = centre_of(jlast, R.n, R.s, P);
            stage_ring<LS>(sx, J, xmap, P, J.nr - 1 - P.ri, c0 - before, c1 - c0 + cnt);
            cp_commit();
        }
        for (int p = p0; p < p1; ++p) {
            const int buf = (p - p0) & 1;
            if (p + 1 < p1) {
                const PairInfo Pn = J.pairs[p + 1];
                int before, cnt;
                win_shape(Pn, before, cnt);
                const int c0 = centre_of(j0, R.n, R.s, Pn), c1 = centre_of(jlast, R.n, R.s, Pn);
                stage_ring<LS>(sx + (buf ^ 1) * 8 * LS, J, xmap, Pn, J.nr - 1 - Pn.ri, c0 - before, c1 - c0 + cnt);
            }
            cp_commit();
            cp_wait1();
            __syncthreads();
            if (active) {
                const PairInfo P = J.pairs[p];
                int before, cnt;
                win_shape(P, before, cnt);
                const int cb = centre_of(j0, R.n, R.s, P);
                const int c = centre_of(jo, R.n, R.s, P);
                const int jlo = c - before;
                // |q| < 2^24 on this window (checked when the plan was built): exact in FP32
                float qf = (float)pair_q(jlo, jo, R.n, R.s, P);
                const float dq = (float)(2 * R.n);
                const float *xs = sx + buf * 8 * LS + (c - cb);
                for (int m = 0; m < cnt; ++m) {
                    const float w = pair_weight(qf * P.c0, P.A, P.B, J.kp, J.tab);
                    qf += dq;
#pragma unroll
                    for (int s = 0; s < 8; ++s) acc[s] = fmaf(w, xs[s * LS + m], acc[s]);
                }
            }
            __syncthreads();
        }
        if (active) {
            float *yn = J.y + (long long)map * J.stride + R.start;
            float *ys = J.y + (long long)map * J.stride + J.rings[ro_s].start;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                yn[jo + k * Qo] = acc[k];
                ys[jo + k * Qo] = acc[4 + k];
            }
        }
    }
}

template <int LS>
cudaError_t launch_ls(const JobsArg &a, int grid, cudaStream_t st) {
    const size_t smem = (size_t)2 * 8 * LS * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_conv_cap<LS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_conv_cap<LS><<<grid, CT, smem, st>>>(a);
    return cudaGetLastError();
}

template <int LS>
int occupancy_ls() {
    const size_t smem = (size_t)2 * 8 * LS * sizeof(float);
    cudaFuncSetAttribute(k_conv_cap<LS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_conv_cap<LS>, CT, smem);
    return nb;
}

}  // namespace

cudaError_t sk_launch_conv_cap(const JobsArg &a, int ls, int grid, cudaStream_t st) {
    if (a.total <= 0) return cudaSuccess;
    switch (ls) {
        case 256: return launch_ls<256>(a, grid, st);
        case 512: return launch_ls<512>(a, grid, st);
        case 1024: return launch_ls<1024>(a, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

int sk_cap_blocks_per_sm(int ls) {
    switch (ls) {
        case 256: return occupancy_ls<256>();
        case 512: return occupancy_ls<512>();
        case 1024: return occupancy_ls<1024>();
        default: return 0;
    }
}
