// harmonic.cu -- the harmonic half of the split convolution (Sec. 2, Eq. 1):
//
//     y_p (+)= sum_{l <= L} sum_m K^_l a_lm Y_lm(p),   a_lm = dOmega sum_q x_q Y*_lm(q)
//
// for l <= L = l_cut, the part of the kernel the paper hands to a spherical
// harmonic transform (libpsht on the CPU in the paper).  With Y_lm(theta, phi) =
// lambda_lm(theta) e^{i m phi} and real maps this is, ring by ring,
//
//   F_r(m)  = sum_j x_{r,j} e^{-i m phi_{r,j}}                          (ring DFT)
//   a_lm    = dOmega sum_r lambda_lm(theta_r) F_r(m)                     (Legendre analysis)
//   G_r(m)  = sum_{l >= m} K^_l a_lm lambda_lm(theta_r)                  (Legendre synthesis)
//   y_{r,j} = Re G_r(0) + 2 Re sum_{m=1}^{L} G_r(m) e^{i m phi_{r,j}}     (ring inverse DFT)
//
// lambda_lm are the orthonormal associated Legendre functions (the standard
// three-term recurrence in l at fixed m), tabulated once per handle in FP64 and
// stored in FP32 for the northern rings and the equator: the southern ring
// 4N - r has lambda_lm(pi - theta) = (-1)^(l+m) lambda_lm(theta), so the sums use
// E_r = F_r + F_r' (l + m even) and O_r = F_r - F_r' (l + m odd).  Table layout
// [m][l - m][r] (r fastest): the analysis reads it with lanes along r, the
// synthesis with threads along r, the tabulation writes it with threads along r.
//
// Ring DFTs: the 2N + 1 rings of 4N pixels (equatorial zone) go through one
// batched cuFFT R2C / C2R plan straight on the map; the polar-cap rings (4r
// pixels, r < N) are summed directly against a twiddle table in shared memory
// (their bins alias when 4r < 2L + 1, which the direct sum does by itself).
// Phases: phi_{r,j} = pi (2j + s_r) / n_r, so F_r(m) = e^{-i pi m s_r / n_r} X_r(m)
// with X_r the plain DFT.
#include <cufft.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "skconv_host.h"

struct sk_harm {
    sk_ctx *ctx = nullptr;
    const sk_geom *g = nullptr;
    int L = 0;
    int nrh = 0;                 // northern rings and the equator: 0-based rings 0 .. 2N - 1
    double *d_kl = nullptr;      // K^_l, l = 0..L
    float *d_lam = nullptr;      // lambda table [m][l - m][r]
    long long *d_moff = nullptr; // start of block m in d_lam
    long long *d_aoff = nullptr; // start of block m in a (l = m..L)
    long long lam_n = 0, a_n = 0;
    // per-call buffers (sized for `cap_batch` maps, grown on demand)
    long long cap_batch = 0;
    float2 *d_F = nullptr;       // [batch][nr][L + 1] ring coefficients F, then G
    float2 *d_a = nullptr;       // [batch][a_n]
    // equatorial-zone FFTs (rings N-1 .. 3N-1, 0-based, all 4N pixels)
    cufftHandle p_r2c = 0, p_c2r = 0;
    bool plans = false;
    float2 *d_X = nullptr;       // [(2N+1)][2N+1] bins of one map
    float *d_tmp = nullptr;      // [(2N+1) * 4N] synthesised zone of one map
    // twiddles and ring phases, FP64-accurate, stored FP32 (built once per handle)
    float2 *d_tw = nullptr;      // cap ring of 4r pixels: e^{-2 pi i k / 4r} at [2r(r-1) + k]
    float2 *d_ph = nullptr;      // cap ring r: e^{-i pi m / 4r} at [(r-1)(L+1) + m]
    float2 *d_zph = nullptr;     // rings of 4N pixels with s = 1: e^{-i pi m / 4N}, m = 0..L
};

namespace {

constexpr int HT = 256;
constexpr int RESYNC = 32;     // ring DFTs: Horner blocks of RESYNC terms, exact twiddle per block
constexpr int CH = 4;          // ring DFTs: independent chains per thread

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// lambda_lm(theta_r) for l = m..L, FP64 three-term recurrence with an exponent
// offset: lambda_mm = (-1)^m sqrt((2m+1)/(4 pi) prod_{k<=m} (2k-1)/(2k)) sin^m theta
// underflows FP64 for large m near the poles; the recurrence runs on
// v = lambda 2^E and drops E as v grows (values below FP32 range are stored as 0).
// lg2c[m] = log2 of the constant factor.  One thread per (m, r).
__global__ void k_lambda(const double *theta, const double *lg2c, const long long *moff, int L, int nrh,
                         float *lam) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)(L + 1) * nrh) return;
    const int m = (int)(idx / nrh), r = (int)(idx % nrh);
    const double th = theta[r];
    const double x = cos(th), sx = sin(th);
    float *out = lam + moff[m] + r;
    // log2 |lambda_mm|
    const double lg = lg2c[m] + (m > 0 ? m * log2(sx) : 0.0);
    int E = 0;
    if (lg < -900.0) E = (int)(-lg) - 600;          // v_mm about 2^-600
    double v0 = exp2(lg + E);
    if (m & 1) v0 = -v0;
    double vm1 = 0.0, v = v0;                        // v_{l-1}, v_l
    for (int l = m; l <= L; ++l) {
        if (l == m + 1) {
            vm1 = v;
            v = sqrt(2.0 * m + 3.0) * x * vm1;
        } else if (l > m + 1) {
            const double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
            const double b = sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
            const double vn = a * (x * v - b * vm1);
            vm1 = v;
            v = vn;
        }
        if (E > 0 && fabs(v) > 0x1p400) {            // take part of the offset out
            const int d = E < 400 ? E : 400;
            v = ldexp(v, -d);
            vm1 = ldexp(vm1, -d);
            E -= d;
        }
        out[(long long)(l - m) * nrh] = (float)ldexp(v, -E);
    }
}

// Twiddle and phase tables of the ring DFTs (FP64 sincospi, stored FP32).
__global__ void k_ring_tables(int nside, int L, float2 *tw, float2 *ph, float2 *zph) {
    const long long ntw = 2LL * nside * (nside - 1);               // sum of 4r, r < N
    const long long nph = (long long)(nside - 1) * (L + 1);
    const long long tot = ntw + nph + (L + 1);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        double sn, cs;
        if (i < ntw) {
            // ring r (1-based) owns [2r(r-1), 2r(r+1)): solve 2r(r-1) <= i
            long long r = (long long)((1.0 + sqrt(1.0 + 2.0 * (double)i)) * 0.5);
            while (2 * r * (r - 1) > i) --r;
            while (2 * (r + 1) * r <= i) ++r;
            const long long k = i - 2 * r * (r - 1);
            sincospi(2.0 * (double)k / (double)(4 * r), &sn, &cs);
            tw[i] = make_float2((float)cs, (float)-sn);
        } else if (i < ntw + nph) {
            const long long j = i - ntw;
            const long long r = j / (L + 1) + 1, m = j % (L + 1);
            sincospi(-(double)m / (double)(4 * r), &sn, &cs);
            ph[j] = make_float2((float)cs, (float)sn);
        } else {
            const long long m = i - ntw - nph;
            sincospi(-(double)m / (double)(4 * nside), &sn, &cs);
            zph[m] = make_float2((float)cs, (float)sn);
        }
    }
}

// Polar-cap rings: F_r(m) = e^{-i pi m s / n} sum_j x_j e^{-2 pi i m j / n}, m = 0..L.
// One block per (cap ring, map); cap ring c < N - 1 is 0-based ring c, else its
// southern mirror.  Twiddles w_k = e^{-2 pi i k / n} in shared memory.
__global__ void k_dft_cap(const RingDev *rings, int nside, const float *x, long long stride, int L,
                          int nr, const float2 *twg, const float2 *phg, float2 *F) {
    extern __shared__ float2 sh[];
    const int ncap = nside - 1;
    const int c = blockIdx.x, b = blockIdx.y;
    const int r = c < ncap ? c : nr - 1 - (c - ncap);
    const RingDev R = rings[r];
    const int n = R.n;
    float2 *tw = sh;
    float *xs = reinterpret_cast<float *>(sh + n);
    const float *xr = x + (long long)b * stride + R.start;
    const int r1 = n / 4;                            // cap ring of 4 r1 pixels (shift 1)
    const float2 *twr = twg + 2LL * r1 * (r1 - 1);
    const float2 *phr = phg + (long long)(r1 - 1) * (L + 1);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        tw[k] = twr[k];
        xs[k] = xr[k];
    }
    __syncthreads();
    float2 *Fr = F + ((long long)b * nr + r) * (L + 1);
    // CH multipoles per thread, their Horner chains interleaved (independent, one load of x_j each)
    for (int mb = threadIdx.x; mb <= L; mb += CH * blockDim.x) {
        // blocks of RESYNC pixels: S_b = sum_t x_{j0+t} w^t by Horner's rule (w = e^{-2 pi i m / n},
        // rounding grows with the block length only), F += w^{j0} S_b with w^{j0} exact
        int step[CH];
        float2 rot[CH];
        float re[CH], im[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int m = min(mb + c * (int)blockDim.x, L);
            step[c] = m % n;
            rot[c] = tw[step[c]];
            re[c] = 0.0f;
            im[c] = 0.0f;
        }
        for (int j0 = 0; j0 < n; j0 += RESYNC) {
            const int j1 = min(j0 + RESYNC, n);
            float hr[CH], hi[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) { hr[c] = xs[j1 - 1]; hi[c] = 0.0f; }
            for (int j = j1 - 2; j >= j0; --j) {
                const float xv = xs[j];
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    const float nr = fmaf(hr[c], rot[c].x, fmaf(-hi[c], rot[c].y, xv));
                    hi[c] = fmaf(hr[c], rot[c].y, hi[c] * rot[c].x);
                    hr[c] = nr;
                }
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const float2 w0 = tw[(int)(((long long)step[c] * j0) % n)];
                re[c] = fmaf(hr[c], w0.x, fmaf(-hi[c], w0.y, re[c]));
                im[c] = fmaf(hr[c], w0.y, fmaf(hi[c], w0.x, im[c]));
            }
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int m = mb + c * (int)blockDim.x;
            if (m > L) continue;
            Fr[m] = cmulf(make_float2(re[c], im[c]), phr[m]);
        }
    }
}

// Equatorial zone after the R2C: F_r(m) = e^{-i pi m s / n} X_r(m), m = 0..L.
__global__ void k_zone_in(const RingDev *rings, int nside, const float2 *X, int L, int nr, long long b,
                          const float2 *zph, float2 *F) {
    const int zr = blockIdx.x;                       // 0 .. 2N
    const int r = nside - 1 + zr;
    const int nb = 2 * nside + 1;
    const int s = rings[r].s;
    float2 *Fr = F + (b * nr + r) * (L + 1);
    for (int m = threadIdx.x; m <= L; m += blockDim.x) {
        const float2 v = X[(long long)zr * nb + m];
        Fr[m] = s ? cmulf(v, zph[m]) : v;
    }
}

// Legendre analysis: a_lm = dOmega sum_r lambda_lm(theta_r) (E_r or O_r), one
// block per (m, map), a warp per l, lanes along r, warp sum.
__global__ void k_leg_analysis(const float *lam, const long long *moff, const long long *aoff, const float2 *F,
                               int L, int nr, int nrh, long long a_n, float domega, float2 *a) {
    extern __shared__ float2 sEO[];                  // [nrh] E, then [nrh] O
    const int m = blockIdx.x, b = blockIdx.y;
    const float2 *Fb = F + (long long)b * nr * (L + 1);
    for (int r = threadIdx.x; r < nrh; r += blockDim.x) {
        const float2 fn = Fb[(long long)r * (L + 1) + m];
        const int rs = nr - 1 - r;
        if (rs == r) {                               // equator: lambda_lm(pi/2) = 0 for l + m odd
            sEO[r] = fn;
            sEO[nrh + r] = make_float2(0.0f, 0.0f);
        } else {
            const float2 fs = Fb[(long long)rs * (L + 1) + m];
            sEO[r] = make_float2(fn.x + fs.x, fn.y + fs.y);
            sEO[nrh + r] = make_float2(fn.x - fs.x, fn.y - fs.y);
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const float *lm = lam + moff[m];
    const int n4 = nrh >> 2;                          // rings in fours (nrh = 2 Nside, a multiple of 4)
    for (int l = m + warp; l <= L; l += nw) {
        const float4 *row = reinterpret_cast<const float4 *>(lm + (long long)(l - m) * nrh);
        const float4 *S = reinterpret_cast<const float4 *>(sEO + (((l + m) & 1) ? nrh : 0));
        float re0 = 0.0f, im0 = 0.0f, re1 = 0.0f, im1 = 0.0f;
        int q = lane;
        for (; q + 32 < n4; q += 64) {               // two 16-byte loads in flight per lane
            const float4 w = row[q], v = row[q + 32];
            const float4 s0 = S[2 * q], s1 = S[2 * q + 1], t0 = S[2 * (q + 32)], t1 = S[2 * (q + 32) + 1];
            re0 = fmaf(w.x, s0.x, re0); im0 = fmaf(w.x, s0.y, im0);
            re1 = fmaf(w.y, s0.z, re1); im1 = fmaf(w.y, s0.w, im1);
            re0 = fmaf(w.z, s1.x, re0); im0 = fmaf(w.z, s1.y, im0);
            re1 = fmaf(w.w, s1.z, re1); im1 = fmaf(w.w, s1.w, im1);
            re0 = fmaf(v.x, t0.x, re0); im0 = fmaf(v.x, t0.y, im0);
            re1 = fmaf(v.y, t0.z, re1); im1 = fmaf(v.y, t0.w, im1);
            re0 = fmaf(v.z, t1.x, re0); im0 = fmaf(v.z, t1.y, im0);
            re1 = fmaf(v.w, t1.z, re1); im1 = fmaf(v.w, t1.w, im1);
        }
        for (; q < n4; q += 32) {
            const float4 w = row[q];
            const float4 s0 = S[2 * q], s1 = S[2 * q + 1];
            re0 = fmaf(w.x, s0.x, re0); im0 = fmaf(w.x, s0.y, im0);
            re1 = fmaf(w.y, s0.z, re1); im1 = fmaf(w.y, s0.w, im1);
            re0 = fmaf(w.z, s1.x, re0); im0 = fmaf(w.z, s1.y, im0);
            re1 = fmaf(w.w, s1.z, re1); im1 = fmaf(w.w, s1.w, im1);
        }
        float re = re0 + re1, im = im0 + im1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (lane == 0) a[(long long)b * a_n + aoff[m] + (l - m)] = make_float2(domega * re, domega * im);
    }
}
__global__ void k_leg_synthesis(const float *lam, const long long *moff, const long long *aoff, const double *kl,
                                const float2 *a, int L, int nr, int nrh, long long a_n, float2 *G) {
    extern __shared__ float2 sb[];                   // b_l = K^_l a_lm, l = m..L
    const int m = blockIdx.x, b = blockIdx.y;
    for (int l = m + threadIdx.x; l <= L; l += blockDim.x) {
        const float2 v = a[(long long)b * a_n + aoff[m] + (l - m)];
        const float k = (float)kl[l];
        sb[l - m] = make_float2(k * v.x, k * v.y);
    }
    __syncthreads();
    const float *lm = lam + moff[m];
    float2 *Gb = G + (long long)b * nr * (L + 1);
    const int n4 = nrh >> 2;                          // rings in fours: one 16-byte load per l
    for (int q = threadIdx.x; q < n4; q += blockDim.x) {
        float er[4] = {}, ei[4] = {}, orr[4] = {}, oi[4] = {};
        int l = m;
        for (; l + 1 <= L; l += 2) {                 // l - m even (l + m even), then odd
            const float4 w0 = reinterpret_cast<const float4 *>(lm + (long long)(l - m) * nrh)[q];
            const float4 w1 = reinterpret_cast<const float4 *>(lm + (long long)(l + 1 - m) * nrh)[q];
            const float2 b0 = sb[l - m], b1 = sb[l + 1 - m];
            const float a0[4] = {w0.x, w0.y, w0.z, w0.w}, a1[4] = {w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                er[u] = fmaf(a0[u], b0.x, er[u]); ei[u] = fmaf(a0[u], b0.y, ei[u]);
                orr[u] = fmaf(a1[u], b1.x, orr[u]); oi[u] = fmaf(a1[u], b1.y, oi[u]);
            }
        }
        if (l <= L) {
            const float4 w0 = reinterpret_cast<const float4 *>(lm + (long long)(l - m) * nrh)[q];
            const float2 b0 = sb[l - m];
            const float a0[4] = {w0.x, w0.y, w0.z, w0.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) { er[u] = fmaf(a0[u], b0.x, er[u]); ei[u] = fmaf(a0[u], b0.y, ei[u]); }
        }
        // (l + m) has the parity of (l - m): the first of each pair is even
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = 4 * q + u, rs = nr - 1 - r;
            Gb[(long long)r * (L + 1) + m] = make_float2(er[u] + orr[u], ei[u] + oi[u]);
            if (rs != r) Gb[(long long)rs * (L + 1) + m] = make_float2(er[u] - orr[u], ei[u] - oi[u]);
        }
    }
}

// Polar-cap rings: y_j (+)= Re G(0) + 2 Re sum_{m=1}^{L} G(m) e^{i pi m (2j + s) / n}.
__global__ void k_idft_cap(const RingDev *rings, int nside, const float2 *G, int L, int nr, float *y,
                           long long stride, int accumulate, const float2 *twg, const float2 *phg) {
    extern __shared__ float2 sh[];
    const int ncap = nside - 1;
    const int c = blockIdx.x, b = blockIdx.y;
    const int r = c < ncap ? c : nr - 1 - (c - ncap);
    const RingDev R = rings[r];
    const int n = R.n;
    float2 *tw = sh;                                 // e^{+2 pi i k / n}
    float2 *gs = sh + n;                             // G(m) e^{i pi m s / n}, doubled for m >= 1
    const float2 *Gr = G + ((long long)b * nr + r) * (L + 1);
    const int r1 = n / 4;                            // cap ring of 4 r1 pixels (shift 1)
    const float2 *twr = twg + 2LL * r1 * (r1 - 1);
    const float2 *phr = phg + (long long)(r1 - 1) * (L + 1);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const float2 w = twr[k];
        tw[k] = make_float2(w.x, -w.y);              // e^{+2 pi i k / n}
    }
    for (int m = threadIdx.x; m <= L; m += blockDim.x) {
        const float2 p = phr[m];
        float2 v = cmulf(Gr[m], make_float2(p.x, -p.y));   // G(m) e^{+i pi m / n}
        if (m > 0) { v.x *= 2.0f; v.y *= 2.0f; }
        gs[m] = v;
    }
    __syncthreads();
    float *yr = y + (long long)b * stride + R.start;
    // CH pixels per thread, their Horner chains interleaved (one load of g_m each)
    for (int jb = threadIdx.x; jb < n; jb += CH * blockDim.x) {
        // blocks of RESYNC multipoles: S_b = sum_t g_{m0+t} w^t by Horner's rule
        // (w = e^{2 pi i j / n}), y += Re(w^{m0} S_b) with w^{m0} exact
        int step[CH];
        float2 rot[CH];
        float acc[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int j = min(jb + c * (int)blockDim.x, n - 1);
            step[c] = j;
            rot[c] = tw[j];
            acc[c] = 0.0f;
        }
        for (int m0 = 0; m0 <= L; m0 += RESYNC) {
            const int m1 = min(m0 + RESYNC, L + 1);
            float2 h[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) h[c] = gs[m1 - 1];
            for (int m = m1 - 2; m >= m0; --m) {
                const float2 g = gs[m];
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    const float nr = fmaf(h[c].x, rot[c].x, fmaf(-h[c].y, rot[c].y, g.x));
                    h[c].y = fmaf(h[c].x, rot[c].y, fmaf(h[c].y, rot[c].x, g.y));
                    h[c].x = nr;
                }
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const float2 w0 = tw[(int)(((long long)step[c] * m0) % n)];
                acc[c] = fmaf(h[c].x, w0.x, fmaf(-h[c].y, w0.y, acc[c]));
            }
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int j = jb + c * (int)blockDim.x;
            if (j >= n) continue;
            yr[j] = accumulate ? yr[j] + acc[c] : acc[c];
        }
    }
}

// Equatorial zone before the C2R: bins X_r(m) = G_r(m) e^{i pi m s / n} for m <= L, 0 above.
__global__ void k_zone_out(const RingDev *rings, int nside, const float2 *G, int L, int nr, long long b,
                           const float2 *zph, float2 *X) {
    const int zr = blockIdx.x;
    const int r = nside - 1 + zr;
    const int nb = 2 * nside + 1;
    const int s = rings[r].s;
    const float2 *Gr = G + (b * nr + r) * (L + 1);
    for (int m = threadIdx.x; m < nb; m += blockDim.x) {
        float2 v = make_float2(0.0f, 0.0f);
        if (m <= L) {
            v = s ? cmulf(Gr[m], make_float2(zph[m].x, -zph[m].y)) : Gr[m];
            if (m == 0) v.y = 0.0f;
        }
        X[(long long)zr * nb + m] = v;
    }
}

__global__ void k_zone_store(const float *tmp, long long n, float *y, int accumulate) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = accumulate ? y[i] + tmp[i] : tmp[i];
}

// R_l = 2 pi int_0^theta_cut K_lin(theta) P_l(cos theta) sin theta dtheta, l = 0..L:
// Gauss-Legendre with npts points on every node interval (K_lin is linear there),
// one thread per quadrature point, P_l by the Bonnet recurrence, warp sums into
// shared FP64 bins, one global atomic per bin and block.
__device__ __forceinline__ double node_theta(int k, int nt, double tc, int layout) {
    if (layout == 0) return (double)k * tc / (double)(nt - 1);
    const int M = nt / 2;
    const double t1 = tc / 16.0;
    return k <= M ? (double)k * t1 / (double)M : t1 + (double)(k - M) * (tc - t1) / (double)(nt - 1 - M);
}

__global__ void k_response(const double *V, int nt, double tc, int layout, int L, const double *gx,
                           const double *gw, int npts, double *R) {
    extern __shared__ double sR[];
    for (int l = threadIdx.x; l <= L; l += blockDim.x) sR[l] = 0.0;
    __syncthreads();
    const long long nq = (long long)(nt - 1) * npts;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double c = 0.0, x = 1.0;
    if (q < nq) {
        const int k = (int)(q / npts), i = (int)(q % npts);
        const double a = node_theta(k, nt, tc, layout), b = node_theta(k + 1, nt, tc, layout);
        const double t = 0.5 * (b - a) * gx[i] + 0.5 * (a + b);
        const double f = (t - a) / (b - a);
        const double K = V[k] + f * (V[k + 1] - V[k]);
        c = 0.5 * (b - a) * gw[i] * K * sin(t);
        x = cos(t);
    }
    const int lane = threadIdx.x & 31;
    double p0 = 1.0, p1 = x;
    for (int l = 0; l <= L; ++l) {
        double pl;
        if (l == 0) pl = p0;
        else if (l == 1) pl = p1;
        else {
            pl = ((2.0 * l - 1.0) * x * p1 - (l - 1.0) * p0) / (double)l;
            p0 = p1;
            p1 = pl;
        }
        double v = c * pl;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(&sR[l], v);
    }
    __syncthreads();
    for (int l = threadIdx.x; l <= L; l += blockDim.x) atomicAdd(&R[l], 2.0 * SK_PI * sR[l]);
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n from the cosine guesses).
void gauss_legendre(int n, double *x, double *w) {
    for (int i = 0; i < n; ++i) {
        double z = cos(SK_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int l = 2; l <= n; ++l) {
                const double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Response matrix of the hat basis: M[l][k] = 2 pi int hat_k P_l(cos t) sin t dt,
// l = 0..lfit, k = 0..n_u-1 (uniform nodes t_k = k h, h = theta_cut / n_u; the
// node at theta_cut is held at 0).  Half a warp per hat: lanes 0-7 take the 8
// Gauss points of [t_{k-1}, t_k], lanes 8-15 those of [t_k, t_{k+1}].
__global__ void k_hat_response(int n_u, double h, int lfit, const double *gx, const double *gw, double *M) {
    const int hw = (blockIdx.x * blockDim.x + threadIdx.x) >> 4, ln = threadIdx.x & 15;
    const bool live = hw < n_u;
    const int k = live ? hw : 0;
    const int side = ln >> 3, i = ln & 7;             // 0: interval left of node k, 1: right
    double c = 0.0, x = 1.0;
    if (live && !(side == 0 && k == 0)) {
        const double a = (k - 1 + side) * h;          // interval [a, a + h]
        const double t = a + 0.5 * h * (gx[i] + 1.0);
        const double f = (t - a) / h;
        const double hat = side == 0 ? f : 1.0 - f;
        c = 2.0 * SK_PI * 0.5 * h * gw[i] * hat * sin(t);
        x = cos(t);
    }
    double p0 = 1.0, p1 = x;
    for (int l = 0; l <= lfit; ++l) {
        double pl;
        if (l == 0) pl = p0;
        else if (l == 1) pl = p1;
        else {
            pl = ((2.0 * l - 1.0) * x * p1 - (l - 1.0) * p0) / (double)l;
            p0 = p1;
            p1 = pl;
        }
        double v = c * pl;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (live && ln == 0) M[(long long)l * n_u + k] = v;
    }
}

// A[i][j] = sum_l W_l M[l][i] M[l][j]: one thread per entry.
__global__ void k_normal_matrix(const double *M, const double *W, int n_u, int lfit, double *A) {
    const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_u) return;
    double acc = 0.0;
    for (int l = 0; l <= lfit; ++l) acc += W[l] * M[(long long)l * n_u + i] * M[(long long)l * n_u + j];
    A[(long long)i * n_u + j] = acc;
}

void free_harm(sk_harm *h) {
    if (!h) return;
    if (h->plans) { cufftDestroy(h->p_r2c); cufftDestroy(h->p_c2r); }
    cudaFree(h->d_kl); cudaFree(h->d_lam); cudaFree(h->d_moff); cudaFree(h->d_aoff);
    cudaFree(h->d_F); cudaFree(h->d_a); cudaFree(h->d_X); cudaFree(h->d_tmp);
    cudaFree(h->d_tw); cudaFree(h->d_ph); cudaFree(h->d_zph);
    delete h;
}

int cufft_fail(cufftResult r, const char *what) {
    return sk_fail(r == CUFFT_ALLOC_FAILED ? SK_ENOMEM : SK_ECUDA, "%s: cuFFT error %d", what, (int)r);
}

}  // namespace

extern "C" int sk_harmonic_create(sk_ctx *ctx, const sk_geom *g, const double *kl, int lmax, sk_harm **out) {
    if (!ctx || !g || !kl || !out) return sk_fail(SK_EINVAL, "sk_harmonic_create: NULL argument");
    *out = nullptr;
    const long long N = g->nside;
    if (N < 2 || N > SK_HARM_MAX_NSIDE)
        return sk_fail(SK_EUNSUPPORTED, "sk_harmonic_create: nside %lld outside [2, %d]", N, SK_HARM_MAX_NSIDE);
    if (lmax < 0 || lmax > 2 * N - 1)
        return sk_fail(SK_EINVAL, "sk_harmonic_create: lmax %d outside [0, 2 nside - 1]", lmax);
    SK_CU(cudaSetDevice(ctx->device));
    sk_harm *h = new sk_harm();
    h->ctx = ctx;
    h->g = g;
    h->L = lmax;
    h->nrh = (int)(2 * N);
    const int L = lmax, nrh = h->nrh;
    std::vector<long long> moff(L + 1), aoff(L + 1);
    long long tot = 0, atot = 0;
    for (int m = 0; m <= L; ++m) {
        moff[m] = tot; tot += (long long)(L - m + 1) * nrh;
        aoff[m] = atot; atot += L - m + 1;
    }
    h->lam_n = tot;
    h->a_n = atot;
    std::vector<double> lg2c(L + 1);
    {
        double acc = 0.0;                            // log2 prod_{k<=m} (2k-1)/(2k)
        for (int m = 0; m <= L; ++m) {
            if (m > 0) acc += log2((2.0 * m - 1.0) / (2.0 * m));
            lg2c[m] = 0.5 * (log2((2.0 * m + 1.0) / (4.0 * SK_PI)) + acc);
        }
    }
    double *d_lg2c = nullptr;
    const int nb = (int)(2 * N + 1), n4 = (int)(4 * N);
    cudaError_t e = cudaMalloc(&h->d_kl, sizeof(double) * (L + 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_lam, sizeof(float) * tot);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_moff, sizeof(long long) * (L + 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_aoff, sizeof(long long) * (L + 1));
    if (e == cudaSuccess) e = cudaMalloc(&d_lg2c, sizeof(double) * (L + 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_X, sizeof(float2) * (size_t)nb * nb);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_tmp, sizeof(float) * (size_t)nb * n4);
    const long long ntw = 2LL * N * (N - 1), nph = (N - 1) * (long long)(L + 1);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_tw, sizeof(float2) * (size_t)std::max(1LL, ntw));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_ph, sizeof(float2) * (size_t)std::max(1LL, nph));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_zph, sizeof(float2) * (size_t)(L + 1));
    if (e == cudaSuccess) {
        const long long tot = ntw + nph + L + 1;
        k_ring_tables<<<(unsigned)std::min<long long>((tot + HT - 1) / HT, 65535), HT>>>((int)N, L, h->d_tw, h->d_ph,
                                                                                           h->d_zph);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h->d_kl, kl, sizeof(double) * (L + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_moff, moff.data(), sizeof(long long) * (L + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_aoff, aoff.data(), sizeof(long long) * (L + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_lg2c, lg2c.data(), sizeof(double) * (L + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const long long nthr = (long long)(L + 1) * nrh;
        k_lambda<<<(unsigned)((nthr + HT - 1) / HT), HT>>>(g->d_theta, d_lg2c, h->d_moff, L, nrh, h->d_lam);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_lg2c);
    if (e != cudaSuccess) {
        free_harm(h);
        return sk_fail(e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA, "sk_harmonic_create: %s",
                       cudaGetErrorString(e));
    }
    int len[1] = {n4};
    cufftResult cr = cufftPlanMany(&h->p_r2c, 1, len, nullptr, 1, n4, nullptr, 1, nb, CUFFT_R2C, nb);
    if (cr == CUFFT_SUCCESS) cr = cufftPlanMany(&h->p_c2r, 1, len, nullptr, 1, nb, nullptr, 1, n4, CUFFT_C2R, nb);
    if (cr != CUFFT_SUCCESS) { free_harm(h); return cufft_fail(cr, "sk_harmonic_create"); }
    h->plans = true;
    *out = h;
    return SK_OK;
}

extern "C" int sk_harmonic_destroy(sk_harm *h) {
    if (!h) return SK_OK;
    cudaSetDevice(h->ctx->device);
    free_harm(h);
    return SK_OK;
}

extern "C" int sk_harmonic_table_bytes(const sk_harm *h, int64_t *bytes) {
    if (!h || !bytes) return sk_fail(SK_EINVAL, "sk_harmonic_table_bytes: NULL argument");
    *bytes = h->lam_n * (int64_t)sizeof(float);
    return SK_OK;
}

extern "C" int sk_harmonic_apply(sk_ctx *ctx, const sk_harm *hc, const float *d_in, float *d_out, int64_t batch,
                                 int64_t map_stride, int accumulate, void *stream) {
    if (!ctx || !hc || (!d_in && batch > 0) || (!d_out && batch > 0))
        return sk_fail(SK_EINVAL, "sk_harmonic_apply: NULL argument");
    sk_harm *h = const_cast<sk_harm *>(hc);
    const sk_geom *g = h->g;
    if (batch < 0 || map_stride < g->npix) return sk_fail(SK_EINVAL, "sk_harmonic_apply: bad batch or stride");
    if (batch == 0) return SK_OK;
    if (d_in == d_out) return sk_fail(SK_EINVAL, "sk_harmonic_apply: input and output alias");
    if (((uintptr_t)d_in & 15) || ((uintptr_t)d_out & 15) || (map_stride & 3))
        return sk_fail(SK_EINVAL, "sk_harmonic_apply: maps must be 16-byte aligned with a stride multiple of 4");
    SK_CU(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int N = (int)g->nside, nr = g->nr, L = h->L, nrh = h->nrh;
    if (batch > h->cap_batch) {
        cudaFree(h->d_F); h->d_F = nullptr;
        cudaFree(h->d_a); h->d_a = nullptr;
        h->cap_batch = 0;
        SK_CU(cudaMalloc(&h->d_F, sizeof(float2) * (size_t)batch * nr * (L + 1)));
        SK_CU(cudaMalloc(&h->d_a, sizeof(float2) * (size_t)batch * h->a_n));
        h->cap_batch = batch;
    }
    const int nb = 2 * N + 1, n4 = 4 * N;
    const float domega = (float)(4.0 * SK_PI / (double)g->npix);
    const long long zone0 = g->h_rings[N - 1].start;     // first pixel of the equatorial zone
    if (cufftSetStream(h->p_r2c, st) != CUFFT_SUCCESS || cufftSetStream(h->p_c2r, st) != CUFFT_SUCCESS)
        return sk_fail(SK_ECUDA, "sk_harmonic_apply: cufftSetStream failed");
    // ring DFTs
    const int ncap = 2 * (N - 1);
    if (ncap > 0) {
        const size_t sm = sizeof(float2) * 4 * (N - 1) + sizeof(float) * 4 * (N - 1);
        SK_CU(cudaFuncSetAttribute(k_dft_cap, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        // enough threads that one pass of CH chains covers every multipole
        const int thr = std::min(1024, ((L + CH) / CH + 31) / 32 * 32);
        k_dft_cap<<<dim3(ncap, (unsigned)batch), thr, sm, st>>>(g->d_rings, N, d_in, map_stride, L, nr, h->d_tw,
                                                                  h->d_ph, h->d_F);
        SK_CU(cudaGetLastError());
    }
    for (long long b = 0; b < batch; ++b) {
        cufftResult cr = cufftExecR2C(h->p_r2c, const_cast<float *>(d_in) + b * map_stride + zone0,
                                      reinterpret_cast<cufftComplex *>(h->d_X));
        if (cr != CUFFT_SUCCESS) return cufft_fail(cr, "sk_harmonic_apply");
        k_zone_in<<<nb, HT, 0, st>>>(g->d_rings, N, h->d_X, L, nr, b, h->d_zph, h->d_F);
        SK_CU(cudaGetLastError());
    }
    // Legendre analysis and synthesis
    const size_t sm_a = sizeof(float2) * 2 * nrh;
    SK_CU(cudaFuncSetAttribute(k_leg_analysis, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_a));
    k_leg_analysis<<<dim3(L + 1, (unsigned)batch), HT, sm_a, st>>>(h->d_lam, h->d_moff, h->d_aoff, h->d_F, L, nr,
                                                                    nrh, h->a_n, domega, h->d_a);
    SK_CU(cudaGetLastError());
    k_leg_synthesis<<<dim3(L + 1, (unsigned)batch), HT, sizeof(float2) * (L + 1), st>>>(
        h->d_lam, h->d_moff, h->d_aoff, h->d_kl, h->d_a, L, nr, nrh, h->a_n, h->d_F);
    SK_CU(cudaGetLastError());
    // inverse ring DFTs
    if (ncap > 0) {
        const size_t sm = sizeof(float2) * 4 * (N - 1) + sizeof(float2) * (L + 1);
        SK_CU(cudaFuncSetAttribute(k_idft_cap, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_idft_cap<<<dim3(ncap, (unsigned)batch), HT, sm, st>>>(g->d_rings, N, h->d_F, L, nr, d_out, map_stride,
                                                                 accumulate, h->d_tw, h->d_ph);
        SK_CU(cudaGetLastError());
    }
    for (long long b = 0; b < batch; ++b) {
        k_zone_out<<<nb, HT, 0, st>>>(g->d_rings, N, h->d_F, L, nr, b, h->d_zph, h->d_X);
        SK_CU(cudaGetLastError());
        cufftResult cr = cufftExecC2R(h->p_c2r, reinterpret_cast<cufftComplex *>(h->d_X), h->d_tmp);
        if (cr != CUFFT_SUCCESS) return cufft_fail(cr, "sk_harmonic_apply");
        const long long zn = (long long)nb * n4;
        k_zone_store<<<std::min<long long>((zn + HT - 1) / HT, 4096), HT, 0, st>>>(h->d_tmp, zn,
                                                                                 d_out + b * map_stride + zone0,
                                                                                 accumulate);
        SK_CU(cudaGetLastError());
    }
    return SK_OK;
}

extern "C" int sk_kernel_response(sk_ctx *ctx, const sk_kern *k, int lmax, double *h_R) {
    if (!ctx || !k || !h_R) return sk_fail(SK_EINVAL, "sk_kernel_response: NULL argument");
    if (lmax < 0 || lmax > 65535) return sk_fail(SK_EINVAL, "sk_kernel_response: lmax %d outside [0, 65535]", lmax);
    SK_CU(cudaSetDevice(ctx->device));
    constexpr int NP = 8;
    double gx[NP], gw[NP];
    gauss_legendre(NP, gx, gw);
    double *d_g = nullptr, *d_R = nullptr;
    cudaError_t e = cudaMalloc(&d_g, sizeof(double) * 2 * NP);
    if (e == cudaSuccess) e = cudaMalloc(&d_R, sizeof(double) * (lmax + 1));
    if (e == cudaSuccess) e = cudaMemcpy(d_g, gx, sizeof(double) * NP, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_g + NP, gw, sizeof(double) * NP, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d_R, 0, sizeof(double) * (lmax + 1));
    if (e == cudaSuccess) {
        const long long nq = (long long)(k->nt - 1) * NP;
        const size_t sm = sizeof(double) * (lmax + 1);
        e = cudaFuncSetAttribute(k_response, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess) {
            k_response<<<(unsigned)((nq + HT - 1) / HT), HT, sm>>>(k->d_V, k->nt, k->tc, k->layout, lmax, d_g,
                                                                   d_g + NP, NP, d_R);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaMemcpy(h_R, d_R, sizeof(double) * (lmax + 1), cudaMemcpyDeviceToHost);
    cudaFree(d_g);
    cudaFree(d_R);
    if (e != cudaSuccess)
        return sk_fail(e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA, "sk_kernel_response: %s",
                       cudaGetErrorString(e));
    return SK_OK;
}

// Least-squares real-space part (Sec. 3: K^_theta is fit so that its harmonic
// transform matches K_l above l_cut).  See skconv.h.
extern "C" int sk_fit_real_kernel(sk_ctx *ctx, const double *h_kl, int lfit, int lcut, double theta_cut,
                                  int n_basis, int nt_out, double low_weight, double reg, double *h_V,
                                  double *h_sigma_rms) {
    if (!ctx || !h_kl || !h_V) return sk_fail(SK_EINVAL, "sk_fit_real_kernel: NULL argument");
    if (lfit < 1 || lfit > 65535 || lcut < 0 || lcut >= lfit)
        return sk_fail(SK_EINVAL, "sk_fit_real_kernel: need 0 <= lcut < lfit <= 65535");
    if (!(theta_cut > 0.0 && theta_cut <= SK_PI)) return sk_fail(SK_EINVAL, "sk_fit_real_kernel: theta_cut");
    if (n_basis < 3 || n_basis > 4097 || nt_out < n_basis || (nt_out - 1) % (n_basis - 1))
        return sk_fail(SK_EINVAL, "sk_fit_real_kernel: need 3 <= n_basis <= 4097 and (nt_out-1) a multiple of (n_basis-1)");
    if (!(low_weight >= 0.0) || !(reg >= 0.0)) return sk_fail(SK_EINVAL, "sk_fit_real_kernel: negative weight");
    SK_CU(cudaSetDevice(ctx->device));
    const int n_u = n_basis - 1;
    const double h = theta_cut / n_u;
    constexpr int NP = 8;
    double gx[NP], gw[NP];
    gauss_legendre(NP, gx, gw);
    std::vector<double> W(lfit + 1);
    for (int l = 0; l <= lfit; ++l) W[l] = (l > lcut ? 1.0 : low_weight) * (2.0 * l + 1.0);
    double *d_g = nullptr, *d_M = nullptr, *d_W = nullptr, *d_A = nullptr;
    const size_t mbytes = sizeof(double) * (size_t)(lfit + 1) * n_u;
    cudaError_t e = cudaMalloc(&d_g, sizeof(double) * 2 * NP);
    if (e == cudaSuccess) e = cudaMalloc(&d_M, mbytes);
    if (e == cudaSuccess) e = cudaMalloc(&d_W, sizeof(double) * (lfit + 1));
    if (e == cudaSuccess) e = cudaMalloc(&d_A, sizeof(double) * (size_t)n_u * n_u);
    if (e == cudaSuccess) e = cudaMemcpy(d_g, gx, sizeof(double) * NP, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_g + NP, gw, sizeof(double) * NP, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_W, W.data(), sizeof(double) * (lfit + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const long long thr = (long long)n_u * 16;
        k_hat_response<<<(unsigned)((thr + HT - 1) / HT), HT>>>(n_u, h, lfit, d_g, d_g + NP, d_M);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_normal_matrix<<<dim3((n_u + 127) / 128, n_u), 128>>>(d_M, d_W, n_u, lfit, d_A);
        e = cudaGetLastError();
    }
    std::vector<double> M((size_t)(lfit + 1) * n_u), A((size_t)n_u * n_u);
    if (e == cudaSuccess) e = cudaMemcpy(M.data(), d_M, mbytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(A.data(), d_A, sizeof(double) * A.size(), cudaMemcpyDeviceToHost);
    cudaFree(d_g); cudaFree(d_M); cudaFree(d_W); cudaFree(d_A);
    if (e != cudaSuccess)
        return sk_fail(e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA, "sk_fit_real_kernel: %s",
                       cudaGetErrorString(e));
    // right-hand side, Tikhonov term, Cholesky (A is symmetric positive definite with lam > 0)
    std::vector<double> b(n_u, 0.0);
    for (int l = 0; l <= lfit; ++l)
        for (int k = 0; k < n_u; ++k) b[k] += W[l] * h_kl[l] * M[(size_t)l * n_u + k];
    double tr = 0.0;
    for (int k = 0; k < n_u; ++k) tr += A[(size_t)k * n_u + k];
    const double lam = reg * tr / n_u;
    for (int k = 0; k < n_u; ++k) A[(size_t)k * n_u + k] += lam;
    for (int j = 0; j < n_u; ++j) {
        double d = A[(size_t)j * n_u + j];
        for (int q = 0; q < j; ++q) d -= A[(size_t)j * n_u + q] * A[(size_t)j * n_u + q];
        if (!(d > 0.0)) return sk_fail(SK_EINVAL, "sk_fit_real_kernel: normal matrix not positive definite (raise reg)");
        const double ljj = sqrt(d);
        A[(size_t)j * n_u + j] = ljj;
        for (int i = j + 1; i < n_u; ++i) {
            double v = A[(size_t)i * n_u + j];
            for (int q = 0; q < j; ++q) v -= A[(size_t)i * n_u + q] * A[(size_t)j * n_u + q];
            A[(size_t)i * n_u + j] = v / ljj;
        }
    }
    std::vector<double> c(n_u);
    for (int i = 0; i < n_u; ++i) {                  // L z = b
        double v = b[i];
        for (int q = 0; q < i; ++q) v -= A[(size_t)i * n_u + q] * c[q];
        c[i] = v / A[(size_t)i * n_u + i];
    }
    for (int i = n_u - 1; i >= 0; --i) {             // L^T c = z
        double v = c[i];
        for (int q = i + 1; q < n_u; ++q) v -= A[(size_t)q * n_u + i] * c[q];
        c[i] = v / A[(size_t)i * n_u + i];
    }
    // sample the piecewise-linear kernel at the output nodes (the coarse nodes are among them)
    const int q = (nt_out - 1) / n_u;
    for (int i = 0; i < nt_out; ++i) {
        const int k = i / q, r = i % q;
        const double ck = k < n_u ? c[k] : 0.0, ck1 = (k + 1) < n_u ? c[k + 1] : 0.0;
        h_V[i] = r == 0 ? ck : ck + (ck1 - ck) * (double)r / (double)q;
    }
    if (h_sigma_rms) {
        double num = 0.0, den = 0.0;
        for (int l = 0; l <= lfit; ++l) {
            den += (2.0 * l + 1.0) * h_kl[l] * h_kl[l];
            if (l <= lcut) continue;
            double R = 0.0;
            for (int k = 0; k < n_u; ++k) R += M[(size_t)l * n_u + k] * c[k];
            num += (2.0 * l + 1.0) * (R - h_kl[l]) * (R - h_kl[l]);
        }
        *h_sigma_rms = den > 0.0 ? sqrt(num / den) : 0.0;
    }
    return SK_OK;
}
