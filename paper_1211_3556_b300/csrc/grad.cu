// grad.cu -- gradient of a loss with respect to the kernel table nodes.
//
// With y_o = dOmega sum_i K_lin(gamma_oi) x_i and K_lin = V_k (1 - f) + V_{k+1} f
// (linear interpolation of the tabulated kernel, Sec. 3),
//   dL/dV_n = dOmega sum_b sum_o gy_bo sum_{i in cut} x_bi [(1 - f) delta_{n,k} + f delta_{n,k+1}],
// a binned scatter-add over all in-cut pairs.  One thread per output pixel
// walks its window like the per-pair forward path.  Per pair it sums
// v = sum_b gy_bo x_bi over the maps (FP32), takes (k, f) from FP64 chord
// arithmetic (an FP32 node coordinate u would carry an absolute error near
// u * 6e-8, which the bins see undamped), and adds (1-f) v and f v into FP32
// bins in shared memory.  Each persistent block adds its bins into an FP64
// accumulator in global memory; a last kernel scales by dOmega and rounds.
#include "skconv.h"
#include "skconv_internal.cuh"
#include "skconv_launch.h"

namespace {

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

cudaError_t sk_launch_grad_finish(const double *acc, int nt, double scale, float *out, cudaStream_t st) {
    k_grad_finish<<<(nt + 255) / 256, 256, 0, st>>>(acc, nt, scale, out);
    return cudaGetLastError();
}
