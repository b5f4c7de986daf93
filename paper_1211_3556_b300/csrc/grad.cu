// grad.cu -- gradient of a loss with respect to the kernel table nodes.
//
// With y_o = dOmega sum_i K_lin(gamma_oi) x_i and K_lin = V_k (1 - f) + V_{k+1} f
// (linear interpolation of the tabulated kernel, Sec. 3),
//   dL/dV_n = dOmega sum_o gy_o sum_{i in cut} x_i [(1 - f) delta_{n,k} + f delta_{n,k+1}],
// a binned scatter-add over all in-cut pairs.  One thread per output pixel
// walks its window like the per-pair forward path and adds (1-f) gy_o x_i and
// f gy_o x_i into FP32 bins in shared memory; each persistent block then adds
// its bins into an FP64 accumulator in global memory, and a last kernel scales
// by dOmega and rounds to FP32.
#include "skconv.h"
#include "skconv_internal.cuh"
#include "skconv_launch.h"

namespace {

__global__ void __launch_bounds__(128)
k_grad_general(const __grid_constant__ JobsArg A, const float *__restrict__ gy, double *acc) {
    extern __shared__ float bins[];
    const int nt = A.j[0].kp.nt;
    for (int k = threadIdx.x; k < nt; k += blockDim.x) bins[k] = 0.0f;
    __syncthreads();
    for (int f = blockIdx.x; f < A.total; f += gridDim.x) {
        const JobDesc &J = A.j[0];
        const int map = f / J.n_items;
        const int4 it = J.items[f - map * J.n_items];
        const int ro = it.x;
        const RingDev R = J.rings[ro];
        const int jo = it.y + (int)threadIdx.x;
        if (jo >= R.n) continue;
        const float g = gy[(long long)map * J.stride + R.start + jo];
        if (g == 0.0f) continue;
        const float *xb = J.x + (long long)map * J.stride;
        for (int p = J.pair_off[ro]; p < J.pair_off[ro + 1]; ++p) {
            const PairInfo P = J.pairs[p];
            const float *xr = xb + J.rings[P.ri].start;
            int jlo, cnt;
            pair_window(jo, R.n, R.s, P, jlo, cnt);
            long long q = pair_q(jlo, jo, R.n, R.s, P);
            int j = jlo % P.n_i; if (j < 0) j += P.n_i;
            const int dq = 2 * R.n;
            for (int m = 0; m < cnt; ++m) {
                const float x = (float)q * P.c0;
                const float s = (fabsf(x) <= 0.125f) ? sin_small(x) : sinf(x);
                const float t = fmaf(P.B, s * s, P.A);
                if (t <= J.kp.tcut) {
                    int k; float fr;
                    chord_kf(t, J.kp, k, fr);
                    const float v = g * __ldg(xr + j);
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
    if (a.total <= 0) return cudaSuccess;
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
