// conv_general.cu -- per-pair evaluation path: one thread per output pixel.
//
// For every input pixel in the output's window rings the thread evaluates the
// pair weight dOmega K_lin(gamma) from the chord (no 1 - cos cancellation) and
// the linearly interpolated kernel table (Sec. 3), and accumulates
// weight * x.  It handles every ring pair (polar caps, whole-ring windows over
// the poles, the belt), so it is the fallback for rings that the belt and cap
// paths do not cover, and the path SK_PATH_GENERAL selects.
//
// Work item: (output ring, first pixel) for a block of 128 outputs of one map.
#include "skconv_internal.cuh"
#include "skconv_launch.h"

namespace {

__global__ void __launch_bounds__(128)
k_conv_general(const __grid_constant__ JobsArg A) {
    for (int f = blockIdx.x; f < A.total; f += gridDim.x) {
        const JobDesc &J = A.j[sk_find_job(A, f)];
        const int local = f - J.flat_base;
        const int map = local / J.n_items;
        const int4 it = J.items[local - map * J.n_items];
        const int ro = it.x;
        const RingDev R = J.rings[ro];
        const int jo = it.y + threadIdx.x;
        if (jo >= R.n) continue;
        const float *xb = J.x + (long long)map * J.stride;
        float acc = 0.0f;
        for (int p = J.pair_off[ro]; p < J.pair_off[ro + 1]; ++p) {
            const PairInfo P = J.pairs[p];
            const long long st_i = J.rings[P.ri].start;
            int jlo, cnt;
            pair_window(jo, R.n, R.s, P, jlo, cnt);
            long long q = pair_q(jlo, jo, R.n, R.s, P);
            int j = jlo % P.n_i; if (j < 0) j += P.n_i;
            const float *xr = xb + st_i;
            const int dq = 2 * R.n;
            for (int m = 0; m < cnt; ++m) {
                float w = pair_weight((float)q * P.c0, P.A, P.B, J.kp, J.tab);
                if (w != 0.0f) acc = fmaf(w, __ldg(xr + j), acc);
                q += dq;
                if (++j == P.n_i) j = 0;
            }
        }
        J.y[(long long)map * J.stride + R.start + jo] = acc;
    }
}

}  // namespace

cudaError_t sk_launch_conv_general(const JobsArg &a, int grid, cudaStream_t st) {
    if (a.total <= 0) return cudaSuccess;
    k_conv_general<<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}
