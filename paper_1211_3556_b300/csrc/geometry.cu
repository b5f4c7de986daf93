// geometry.cu -- device-side set-up kernels, all FP64:
//  * HEALPix RING ring tables (the paper's pixelisation, Sec. 2; formulas of
//    Gorski et al. 2005, RING numbering of the HEALPix library);
//  * per-output-ring window rings and phi half-widths (rings within theta_cut,
//    phi window from the haversine relation);
//  * Legendre tabulation of the real-space part of a split kernel (Sec. 2,
//    Eq. 1: the Legendre transform operator P_{l theta}), with a taper;
//  * conversion of node values into the FP32 (value, slope) table with the
//    pixel area folded in;
//  * the exact in-cut pair count.
#include "skconv_internal.cuh"
#include "skconv_launch.h"

namespace {

__device__ void ring_of(long long N, int r, int &n, long long &start, int &s, double &z, double &rho) {
    const long long npix = 12LL * N * N;
    if (r < N) {
        n = 4 * r; start = 2LL * r * (r - 1); s = 1;
        double omz = (double)r * (double)r / (3.0 * (double)N * (double)N);
        z = 1.0 - omz; rho = sqrt(omz * (2.0 - omz));
    } else if (r <= 3 * N) {
        n = (int)(4 * N); start = 2LL * N * (N - 1) + 4LL * N * (r - N);
        s = (int)((r - N + 1) & 1);
        z = (double)(2 * (2 * N - r)) / (3.0 * (double)N);
        rho = sqrt((1.0 - z) * (1.0 + z));
    } else {
        int rp = (int)(4 * N - r);
        n = 4 * rp; start = npix - 2LL * rp * (rp + 1); s = 1;
        double omz = (double)rp * (double)rp / (3.0 * (double)N * (double)N);
        z = -(1.0 - omz); rho = sqrt(omz * (2.0 - omz));
    }
}

__global__ void k_ring_geom(long long N, RingDev *rings, double *z, double *rho, double *theta) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int nr = (int)(4 * N - 1);
    if (idx >= nr) return;
    int n, s; long long st; double zz, rr;
    ring_of(N, idx + 1, n, st, s, zz, rr);
    rings[idx].n = n; rings[idx].s = s; rings[idx].start = st;
    z[idx] = zz; rho[idx] = rr; theta[idx] = atan2(rr, zz);
}

// Rings ri with |theta_i - theta_o| <= theta_cut (+ a tiny margin) for every o.
__global__ void k_pair_ranges(int nr, const double *theta, double tc, int *lo, int *hi) {
    int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nr) return;
    double lim = tc + 1e-9 * (1.0 + tc);
    int a = o, b = o;
    while (a > 0 && fabs(theta[a - 1] - theta[o]) <= lim) --a;
    while (b < nr - 1 && fabs(theta[b + 1] - theta[o]) <= lim) ++b;
    lo[o] = a; hi[o] = b;
}

__device__ double hav(double x) { double s = sin(0.5 * x); return s * s; }

// hav(dphi_max) = (hav tc - hav(th_o - th_i)) / (rho_o rho_i); >= 1 means the whole ring.
__device__ double window_hav(double tc, double tho, double thi, double ro, double rhi) {
    return (hav(tc) - hav(tho - thi)) / (ro * rhi);
}

__global__ void k_pair_info(int nr, const RingDev *rings, const double *z, const double *rho,
                            const double *theta, const int *off, const int *lo, double tc,
                            PairInfo *pairs, double *dphimax, double2 *ab64) {
    int o = blockIdx.x;
    if (o >= nr) return;
    int cnt = off[o + 1] - off[o];
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        int i = lo[o] + t;
        PairInfo P;
        P.ri = i;
        P.n_i = rings[i].n; P.s_i = rings[i].s; P.pad = 0;
        double dz = z[o] - z[i], dr = rho[o] - rho[i];
        const double A = dz * dz + dr * dr, B = 4.0 * rho[o] * rho[i];
        P.A = (float)A;
        P.B = (float)B;
        if (ab64) ab64[off[o] + t] = make_double2(A, B);
        P.c0 = (float)(SK_PI / (2.0 * (double)rings[i].n * (double)rings[o].n));
        double h = window_hav(tc, theta[o], theta[i], rho[o], rho[i]);
        double dpm;
        if (h >= 1.0) {
            P.W = -1; dpm = 4.0;          // > pi: whole ring
        } else {
            double hc = h < 0.0 ? 0.0 : h;
            dpm = 2.0 * asin(sqrt(hc));
            double D = dpm * (double)P.n_i / (2.0 * SK_PI);
            if (h < 0.0) dpm = -1.0;      // no pixel of this ring is within the cut
            // nearest-pixel centre c: |j - jc| <= D implies |j - c| <= D + 1/2
            long long W = (long long)floor(D + 0.5 + 1e-9);
            if (2 * W + 1 >= P.n_i) P.W = -1; else P.W = (int)W;
        }
        pairs[off[o] + t] = P;
        if (dphimax) dphimax[off[o] + t] = dpm;
    }
}

// V_k = taper(theta_k) sum_{l=lmin}^{lmax} (2l+1)/(4 pi) K_l P_l(cos theta_k), Bonnet recurrence.
__global__ void k_tabulate(const double *kl, int lmin, int lmax, int nt, double tc, int layout,
                           double taper_start, double *V) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    double th;
    if (layout == 0) {
        th = (double)k * tc / (double)(nt - 1);
    } else {
        int M = nt / 2; double t1 = tc / 16.0;
        th = (k <= M) ? (double)k * t1 / (double)M
                      : t1 + (double)(k - M) * (tc - t1) / (double)(nt - 1 - M);
    }
    double x = cos(th);
    double p0 = 1.0, p1 = x, acc = 0.0;
    for (int l = 0; l <= lmax; ++l) {
        double pl;
        if (l == 0) pl = p0;
        else if (l == 1) pl = p1;
        else { double p2 = ((2.0 * l - 1.0) * x * p1 - (l - 1.0) * p0) / (double)l; p0 = p1; p1 = p2; pl = p2; }
        if (l >= lmin) acc += (2.0 * l + 1.0) / (4.0 * SK_PI) * kl[l] * pl;
    }
    double w = 1.0;
    if (taper_start < 1.0) {
        double t0 = taper_start * tc;
        if (th >= tc) w = 0.0;
        else if (th > t0) w = 0.5 * (1.0 + cos(SK_PI * (th - t0) / (tc - t0)));
    }
    V[k] = acc * w;
}

__global__ void k_make_table(const double *V, int nt, double dOmega, float2 *tab, const int *gate) {
    if (gate && !*gate) return;                  // values unchanged: the table stands
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    double v = V[k];
    double d = (k + 1 < nt) ? V[k + 1] - v : 0.0;
    tab[k] = make_float2((float)(v * dOmega), (float)(d * dOmega));
}

// Exact pair count: on ring i the in-cut pixels of output (o, jo) are those with
// |phi_j - phi_o| <= dphi_max (gamma grows with |dphi|), an integer interval.
__global__ void k_count_pairs(int nr, const RingDev *rings, const int *off, const PairInfo *pairs,
                              const double *dphimax, const unsigned char *cls, unsigned long long *total,
                              bool per_ring) {
    int o = blockIdx.y;
    int jo = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c = 0;
    if (o < nr && jo < rings[o].n) {
        double phio = SK_PI * (double)(2 * jo + rings[o].s) / (double)rings[o].n;
        for (int p = off[o]; p < off[o + 1]; ++p) {
            const PairInfo &P = pairs[p];
            double dpm = dphimax[p];
            if (dpm >= SK_PI) { c += P.n_i; continue; }
            double sc = (double)P.n_i / (2.0 * SK_PI);
            double a = (phio - dpm) * sc - 0.5 * P.s_i;
            double b = (phio + dpm) * sc - 0.5 * P.s_i;
            long long lo = (long long)ceil(a), hi = (long long)floor(b);
            long long k = hi - lo + 1;
            if (k < 0) k = 0;
            if (k > P.n_i) k = P.n_i;
            c += (unsigned long long)k;
        }
    }
    __shared__ unsigned long long red[256];
    red[threadIdx.x] = c;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0 && red[0]) atomicAdd(total + (per_ring ? o : (cls && o < nr ? cls[o] : 0)), red[0]);
}

}  // namespace

cudaError_t sk_launch_ring_geom(long long nside, RingDev *rings, double *z, double *rho,
                                double *theta, cudaStream_t st) {
    int nr = (int)(4 * nside - 1);
    k_ring_geom<<<(nr + 255) / 256, 256, 0, st>>>(nside, rings, z, rho, theta);
    return cudaGetLastError();
}

cudaError_t sk_launch_pair_ranges(int nr, const double *theta, double tc, int *lo, int *hi,
                                  cudaStream_t st) {
    k_pair_ranges<<<(nr + 255) / 256, 256, 0, st>>>(nr, theta, tc, lo, hi);
    return cudaGetLastError();
}

cudaError_t sk_launch_pair_info(int nr, const RingDev *rings, const double *z, const double *rho,
                                const double *theta, const int *off, const int *lo, double tc,
                                PairInfo *pairs, double *dphimax, double2 *ab64, cudaStream_t st) {
    k_pair_info<<<nr, 64, 0, st>>>(nr, rings, z, rho, theta, off, lo, tc, pairs, dphimax, ab64);
    return cudaGetLastError();
}

cudaError_t sk_launch_tabulate(const double *kl, int lmin, int lmax, int nt, double tc, int layout,
                               double taper_start, double *V, cudaStream_t st) {
    k_tabulate<<<(nt + 127) / 128, 128, 0, st>>>(kl, lmin, lmax, nt, tc, layout, taper_start, V);
    return cudaGetLastError();
}

cudaError_t sk_launch_make_table(const double *V, int nt, double dOmega, float2 *tab, cudaStream_t st,
                                 const int *gate) {
    k_make_table<<<(nt + 255) / 256, 256, 0, st>>>(V, nt, dOmega, tab, gate);
    return cudaGetLastError();
}

// New node values from device memory (nt <= 16384, one block): *changed = whether any
// differs from V, and V takes them if so.
__global__ void __launch_bounds__(1024) k_update_values(const double *nv, double *V, int nt, int *changed) {
    int diff = 0;
    for (int k = threadIdx.x; k < nt; k += blockDim.x) diff |= nv[k] != V[k];
    diff = __syncthreads_or(diff);
    if (diff)
        for (int k = threadIdx.x; k < nt; k += blockDim.x) V[k] = nv[k];
    if (threadIdx.x == 0) *changed = diff ? 1 : 0;
}

cudaError_t sk_launch_update_values(const double *nv, double *V, int nt, int *changed, cudaStream_t st) {
    k_update_values<<<1, 1024, 0, st>>>(nv, V, nt, changed);
    return cudaGetLastError();
}

cudaError_t sk_launch_count_pairs(int nr, int max_n, const RingDev *rings, const int *off,
                                  const PairInfo *pairs, const double *dphimax, const unsigned char *cls,
                                  unsigned long long *total, cudaStream_t st, bool per_ring) {
    dim3 grid((max_n + 255) / 256, nr);
    k_count_pairs<<<grid, 256, 0, st>>>(nr, rings, off, pairs, dphimax, cls, total, per_ring);
    return cudaGetLastError();
}
