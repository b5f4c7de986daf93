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
// batched cuFFT R2C / C2R plan straight on the map.  The polar-cap rings (n = 4r
// pixels, r < N, all lengths) go through chirp-z transforms (Bluestein): with
// jk = (j^2 + k^2 - (k-j)^2)/2, X(k) = sum_j x_j W^{jk} (W = e^{-2 pi i/n}) is
// W^{k^2/2} times the convolution of x_j W^{j^2/2} with W^{-t^2/2}, done by FFTs
// of a common length P >= n + K - 1 (K = min(n, L+1) bins: X is n-periodic, so
// F(m) needs X(m mod n) only); the synthesis is the same with W conjugated,
// after folding the m > n aliases onto m mod n.  The rings are grouped by P (a
// power of two or three times one), each group one batched cuFFT plan; the FFTs
// of the chirp filters are made once per handle.  Phases: phi_{r,j} =
// pi (2j + s_r) / n_r, so F_r(m) = e^{-i pi m s_r / n_r} X_r(m) with X_r the plain
// DFT; chirp phases use j^2 mod 2n in integers.
#include <cufft.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "skconv_host.h"

struct sk_harm {
    sk_ctx *ctx = nullptr;
    int device = 0;              // the context's device (the handle may outlive the context)
    const sk_geom *g = nullptr;
    int L = 0;
    int nrh = 0;                 // northern rings and the equator: 0-based rings 0 .. 2N - 1
    double *d_kl = nullptr;      // K^_l, l = 0..L
    float *d_lam = nullptr;      // lambda table [m][l - m][r]
    long long *d_moff = nullptr; // start of block m in d_lam
    long long *d_aoff = nullptr; // start of block m in a (l = m..L)
    long long lam_n = 0, a_n = 0;
    // where the table rows matter: lambda_lm(theta) decays fast towards the pole below the
    // turning point sin(theta) ~ m / (l + 1/2), and values below LAM_EPS are not read --
    // per row (m, l) the first float4 of rings the analysis reads (d_q0, indexed like a_lm),
    // per (m, 32 float4 of rings) the first l the synthesis reads (d_l0w, [m][n4 / 32])
    int *d_q0 = nullptr;
    int *d_l0w = nullptr;
    // per-call buffers (sized for `cap_batch` maps, grown on demand)
    long long cap_batch = 0;
    float2 *d_F = nullptr;       // [batch][nr][L + 1] ring coefficients F, then G
    float2 *d_a = nullptr;       // [batch][a_n]
    // equatorial-zone FFTs (rings N-1 .. 3N-1, 0-based, all 4N pixels)
    cufftHandle p_r2c = 0, p_c2r = 0;
    bool plans = false;
    float2 *d_X = nullptr;       // [(2N+1)][2N+1] bins of one map
    float *d_tmp = nullptr;      // [(2N+1) * 4N] synthesised zone of one map
    float2 *d_zph = nullptr;     // rings of 4N pixels with s = 1: e^{-i pi m / 4N}, m = 0..L
    // chirp-z transforms of the polar-cap rings (see above): classes of rings sharing an FFT
    // length, a row per (ring, hemisphere), the filters' FFTs, a work buffer per map
    struct CzClass { int P, r0, cnt; long long woff; cufftHandle plan; };
    std::vector<CzClass> cz;
    struct CzRow *d_czrow = nullptr;   // [2 (N - 1)] rows of one map
    float2 *d_czf = nullptr;           // per cap ring r: [analysis filter P][synthesis filter P], FFT'd
    long long cz_n = 0;                // complex values of one map's work rows
    long long cz_batch = 0;
    float2 *d_czw = nullptr;           // [batch][cz_n]
};

// A chirp-z row: cap ring r (1-based, 4r pixels), hemisphere h (0 north: ring r - 1,
// 1 south: ring nr - r, 0-based), FFT length P, offset of its work row (one map) and of its
// ring's filters.
struct CzRow {
    int r, h, P;
    int woff;
    long long foff;
};

namespace {

constexpr int HT = 256;

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

// Rows of the table whose leading rings are below LAM_EPS in magnitude: their products
// with the ring coefficients (|F| up to ~sqrt(4 Nside) times the map's rms) sit far below
// the FP32 rounding of the sums, so those rings are not read.  One warp per row (m, l):
// q0 = (first ring with |lambda| >= LAM_EPS) / 4, or n4 when none.
constexpr float LAM_EPS = 1e-12f;
__global__ void k_lam_q0(const float *lam, const long long *moff, const long long *aoff, int L, int nrh,
                         int *q0) {
    const int warp = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    // row index = aoff[m] + (l - m): find m by a scan of aoff (rows of block m: L - m + 1)
    const long long a_n = aoff[L] + 1;
    if (warp >= a_n) return;
    int lo = 0, hi = L;
    while (lo < hi) {                                    // largest m with aoff[m] <= warp
        const int mid = (lo + hi + 1) >> 1;
        if (aoff[mid] <= warp) lo = mid; else hi = mid - 1;
    }
    const int m = lo, l = m + (int)(warp - aoff[m]);
    const float *row = lam + moff[m] + (long long)(l - m) * nrh;
    int first = nrh;
    for (int r0 = 0; r0 < nrh; r0 += 32) {
        const int r = r0 + lane;
        const bool big = r < nrh && fabsf(row[r]) >= LAM_EPS;
        const unsigned bal = __ballot_sync(0xffffffffu, big);
        if (bal) {
            first = r0 + __ffs(bal) - 1;
            break;
        }
    }
    if (lane == 0) q0[warp] = first >> 2;
}

// Per (m, group of 32 float4 of rings): the first l whose row matters to any ring of the
// group, i.e. the smallest l with q0(m, l) <= the group's last float4 (every earlier row is
// negligible on all the group's rings).  One thread per m.
__global__ void k_lam_l0(const int *q0, const long long *aoff, int L, int n4, int *l0w) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > L) return;
    const int nw = (n4 + 31) / 32;
    int *out = l0w + (long long)m * nw;
    int wl = nw;                                         // groups wl .. nw - 1 have their start
    int cur = n4;
    for (int l = m; l <= L && wl > 0; ++l) {
        cur = min(cur, q0[aoff[m] + (l - m)]);
        while (wl > 0 && min(32 * (wl - 1) + 31, n4 - 1) >= cur) out[--wl] = l;
    }
    while (wl > 0) out[--wl] = L + 1;                   // nothing matters: no row is read
}

// Twiddle and phase tables of the ring DFTs (FP64 sincospi, stored FP32).
// Phases of the zone rings with s = 1: e^{-i pi m / 4N}, m = 0..L (FP64, stored FP32).
__global__ void k_zone_phase(int nside, int L, float2 *zph) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > L) return;
    double sn, cs;
    sincospi(-(double)m / (double)(4 * nside), &sn, &cs);
    zph[m] = make_float2((float)cs, (float)sn);
}

// e^{i pi sign q / n} for q = t^2 mod 2n (exact integer reduction).
__device__ __forceinline__ float2 chirp(long long t, int n, float sign) {
    const long long q = (t * t) % (2LL * n);
    float sn, cs;
    sincospif(sign * (float)q / (float)n, &sn, &cs);
    return make_float2(cs, sn);
}

// The chirp filters of cap ring rows (north rows only: the filters depend on n), in the
// time domain at index t mod P: analysis e^{+i pi t^2/n} for t in [-(n-1), K-1],
// synthesis e^{-i pi t^2/n} for t in [-(K-1), n-1]; FP64 phases.
__global__ void k_cz_filters(const CzRow *rows, int L, float2 *f) {
    const CzRow R = rows[blockIdx.x];
    if (R.h != 0) return;
    const int n = 4 * R.r, K = min(n, L + 1), P = R.P;
    const long long none = -(1LL << 40);
    float2 *fa = f + R.foff, *fs = fa + P;
    // index i stands for t = i (the non-negative part) or t = i - P (the negative part);
    // P >= n + K - 1 keeps the two parts apart
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const long long ta = i <= K - 1 ? i : (i >= P - (n - 1) ? (long long)i - P : none);
        const long long ts = i <= n - 1 ? i : (i >= P - (K - 1) ? (long long)i - P : none);
        double sn, cs;
        float2 va = make_float2(0.f, 0.f), vs = make_float2(0.f, 0.f);
        if (ta != none) {
            sincospi((double)((ta * ta) % (2LL * n)) / (double)n, &sn, &cs);
            va = make_float2((float)cs, (float)sn);
        }
        if (ts != none) {
            sincospi(-(double)((ts * ts) % (2LL * n)) / (double)n, &sn, &cs);
            vs = make_float2((float)cs, (float)sn);
        }
        fa[i] = va;
        fs[i] = vs;
    }
}

__device__ __forceinline__ int cz_ring(const CzRow &R, int nr) { return R.h == 0 ? R.r - 1 : nr - R.r; }

// Analysis, before the FFT: a_j = x_j e^{-i pi j^2/n} (j < n), 0 up to P.
__global__ void k_cz_a_pre(const CzRow *rows, const RingDev *rings, int nr, const float *x, long long stride,
                           long long cz_n, float2 *w) {
    const CzRow R = rows[blockIdx.x];
    const int b = blockIdx.y, n = 4 * R.r;
    const float *xr = x + (long long)b * stride + rings[cz_ring(R, nr)].start;
    float2 *wr = w + (long long)b * cz_n + R.woff;
    for (int j = threadIdx.x; j < R.P; j += blockDim.x) {
        float2 v = make_float2(0.f, 0.f);
        if (j < n) {
            const float xv = xr[j];
            const float2 c = chirp(j, n, -1.0f);
            v = make_float2(xv * c.x, xv * c.y);
        }
        wr[j] = v;
    }
}

// Between the FFTs: w *= the row's filter (analysis: which = 0, synthesis: 1).
__global__ void k_cz_mul(const CzRow *rows, const float2 *f, int which, long long cz_n, float2 *w) {
    const CzRow R = rows[blockIdx.x];
    const int b = blockIdx.y;
    const float2 *fr = f + R.foff + (long long)which * R.P;
    float2 *wr = w + (long long)b * cz_n + R.woff;
    for (int k = threadIdx.x; k < R.P; k += blockDim.x) wr[k] = cmulf(wr[k], fr[k]);
}

// Analysis, after the inverse FFT: F(m) = e^{-i pi m/n} X(m mod n), X(k) = e^{-i pi k^2/n} conv(k) / P.
__global__ void k_cz_a_post(const CzRow *rows, int nr, int L, long long cz_n, const float2 *w, float2 *F) {
    const CzRow R = rows[blockIdx.x];
    const int b = blockIdx.y, n = 4 * R.r;
    const float2 *wr = w + (long long)b * cz_n + R.woff;
    float2 *Fr = F + ((long long)b * nr + cz_ring(R, nr)) * (L + 1);
    const float inv = 1.0f / (float)R.P;
    for (int m = threadIdx.x; m <= L; m += blockDim.x) {
        const int k = m % n;
        float2 v = cmulf(wr[k], chirp(k, n, -1.0f));
        float sn, cs;
        sincospif(-(float)(m % (2 * n)) / (float)n, &sn, &cs);
        v = cmulf(v, make_float2(cs, sn));
        Fr[m] = make_float2(v.x * inv, v.y * inv);
    }
}

// Synthesis, before the FFT: c_k = sum_{m = k mod n, m <= L} g_m e^{i pi m/n} (doubled for m >= 1),
// a'_k = c_k e^{i pi k^2/n} for k < K, 0 up to P.
__global__ void k_cz_s_pre(const CzRow *rows, int nr, int L, long long cz_n, const float2 *G, float2 *w) {
    const CzRow R = rows[blockIdx.x];
    const int b = blockIdx.y, n = 4 * R.r, K = min(n, L + 1);
    const float2 *Gr = G + ((long long)b * nr + cz_ring(R, nr)) * (L + 1);
    float2 *wr = w + (long long)b * cz_n + R.woff;
    for (int k = threadIdx.x; k < R.P; k += blockDim.x) {
        float2 c = make_float2(0.f, 0.f);
        if (k < K) {
            for (int m = k; m <= L; m += n) {
                float sn, cs;
                sincospif((float)(m % (2 * n)) / (float)n, &sn, &cs);
                float2 v = cmulf(Gr[m], make_float2(cs, sn));
                if (m > 0) { v.x *= 2.0f; v.y *= 2.0f; }
                c.x += v.x;
                c.y += v.y;
            }
            c = cmulf(c, chirp(k, n, 1.0f));
        }
        wr[k] = c;
    }
}

// Synthesis, after the inverse FFT: y_j (+)= Re(e^{i pi j^2/n} conv(j)) / P, j < n.
__global__ void k_cz_s_post(const CzRow *rows, const RingDev *rings, int nr, long long cz_n, const float2 *w,
                            float *y, long long stride, int accumulate) {
    const CzRow R = rows[blockIdx.x];
    const int b = blockIdx.y, n = 4 * R.r;
    const float2 *wr = w + (long long)b * cz_n + R.woff;
    float *yr = y + (long long)b * stride + rings[cz_ring(R, nr)].start;
    const float inv = 1.0f / (float)R.P;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const float2 c = chirp(j, n, 1.0f), v = wr[j];
        const float val = (v.x * c.x - v.y * c.y) * inv;
        yr[j] = accumulate ? yr[j] + val : val;
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
__global__ void k_leg_analysis(const float *lam, const long long *moff, const long long *aoff, const int *q0s,
                               const float2 *F, int L, int nr, int nrh, long long a_n, float domega, float2 *a) {
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
        int q = q0s[aoff[m] + (l - m)] + lane;       // the row's leading rings are negligible
#pragma unroll 2
        for (; q + 32 < n4; q += 64) {               // four 16-byte loads in flight per lane (unrolled
                                                     // twice: 3.86 -> 3.74 ms at Nside 2048; four times 3.91)
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
__global__ void k_leg_synthesis(const float *lam, const long long *moff, const long long *aoff, const int *l0w,
                                const double *kl, const float2 *a, int L, int nr, int nrh, long long a_n,
                                float2 *G) {
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
        // the rows before the group's first one that matters are skipped (the start is
        // rounded down to an even l - m, keeping the pairs' parity)
        const int l0 = l0w[(long long)m * ((n4 + 31) / 32) + (q >> 5)];
        int l = m + ((max(l0, m) - m) & ~1);
#pragma unroll 4
        for (; l + 1 <= L; l += 2) {                 // l - m even (l + m even), then odd (4 pairs of
                                                     // rows in flight: 3.90 -> 3.86 ms at Nside 2048)
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
    cudaFree(h->d_zph);
    cudaFree(h->d_q0); cudaFree(h->d_l0w);
    for (auto &c : h->cz)
        if (c.plan) cufftDestroy(c.plan);
    cudaFree(h->d_czrow); cudaFree(h->d_czf); cudaFree(h->d_czw);
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
    h->device = ctx->device;
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
    if (e == cudaSuccess) e = cudaMalloc(&h->d_zph, sizeof(float2) * (size_t)(L + 1));
    if (e == cudaSuccess) {
        k_zone_phase<<<(L + HT) / HT, HT>>>((int)N, L, h->d_zph);
        e = cudaGetLastError();
    }
    // chirp-z classes of the cap rings r = 1 .. N-1: FFT length P = the smallest 2^a or 3 2^a
    // that holds n + K - 1 (n = 4r, K = min(n, L+1)), but at least 2048 (or the largest
    // ring's P when that is smaller): the small rings then share one class, one batched FFT
    // each way instead of a dozen launches of a few microseconds; rows north then south per
    // class
    std::vector<CzRow> rows;
    if (e == cudaSuccess && N > 1) {
        auto fft_len = [](long long need) {
            long long p = 1;
            while (p < need) p <<= 1;
            const long long p3 = 3 * (p >> 2);           // 3 2^(a-2) between p/2 and p
            return (int)(p3 >= need ? p3 : p);
        };
        const int nlast = 4 * ((int)N - 1);
        const int pmin = std::min(2048, fft_len(nlast + std::min(nlast, L + 1) - 1));
        auto ring_len = [&](int r) { return std::max(pmin, fft_len(4 * r + std::min(4 * r, L + 1) - 1)); };
        long long woff = 0, foff = 0;
        for (int r = 1; r < N;) {
            const int P = ring_len(r);
            int r1 = r;
            while (r1 + 1 < N && ring_len(r1 + 1) == P) ++r1;
            sk_harm::CzClass c{P, r, r1 - r + 1, woff, 0};
            for (int hh = 0; hh < 2; ++hh)
                for (int i = 0; i < c.cnt; ++i)
                    rows.push_back(CzRow{r + i, hh, P, (int)(woff + ((long long)hh * c.cnt + i) * P),
                                         foff + 2LL * i * P});
            woff += 2LL * c.cnt * P;
            foff += 2LL * c.cnt * P;
            h->cz.push_back(c);
            r = r1 + 1;
        }
        h->cz_n = woff;
        if (woff >= (1LL << 31)) e = cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = cudaMalloc(&h->d_czrow, sizeof(CzRow) * rows.size());
        if (e == cudaSuccess) e = cudaMemcpy(h->d_czrow, rows.data(), sizeof(CzRow) * rows.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&h->d_czf, sizeof(float2) * (size_t)foff);
        if (e == cudaSuccess) {
            k_cz_filters<<<(unsigned)rows.size(), HT>>>(h->d_czrow, L, h->d_czf);
            e = cudaGetLastError();
        }
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
    // where the rows matter (rings in float4 groups of four: nq of them)
    const int nq = nrh / 4;
    if (e == cudaSuccess) e = cudaMalloc(&h->d_q0, sizeof(int) * (size_t)atot);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_l0w, sizeof(int) * (size_t)(L + 1) * ((nq + 31) / 32));
    if (e == cudaSuccess) {
        const long long threads = 32LL * atot;
        k_lam_q0<<<(unsigned)((threads + HT - 1) / HT), HT>>>(h->d_lam, h->d_moff, h->d_aoff, L, nrh, h->d_q0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_lam_l0<<<(L + HT) / HT, HT>>>(h->d_q0, h->d_aoff, L, nq, h->d_l0w);
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
    // one C2C plan per chirp-z class (2 cnt rows of length P: one map's rows, or the class's
    // filter pairs, which have the same layout); the filters go to the frequency domain now
    for (auto &c : h->cz) {
        int plen[1] = {c.P};
        cr = cufftPlanMany(&c.plan, 1, plen, nullptr, 1, c.P, nullptr, 1, c.P, CUFFT_C2C, 2 * c.cnt);
        if (cr != CUFFT_SUCCESS) { free_harm(h); return cufft_fail(cr, "sk_harmonic_create"); }
        cufftComplex *fz = reinterpret_cast<cufftComplex *>(h->d_czf + c.woff);
        cr = cufftExecC2C(c.plan, fz, fz, CUFFT_FORWARD);
        if (cr != CUFFT_SUCCESS) { free_harm(h); return cufft_fail(cr, "sk_harmonic_create"); }
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { free_harm(h); return sk_fail(SK_ECUDA, "sk_harmonic_create: %s", cudaGetErrorString(e)); }
    *out = h;
    return SK_OK;
}

extern "C" int sk_harmonic_destroy(sk_harm *h) {
    if (!h) return SK_OK;
    cudaSetDevice(h->device);
    free_harm(h);
    return SK_OK;
}

extern "C" int sk_harmonic_table_bytes(const sk_harm *h, int64_t *bytes) {
    if (!h || !bytes) return sk_fail(SK_EINVAL, "sk_harmonic_table_bytes: NULL argument");
    *bytes = h->lam_n * (int64_t)sizeof(float);
    return SK_OK;
}

// The chirp-z FFTs (in place) of every class for `batch` maps.
static int cz_fft(sk_harm *h, long long batch, int dir) {
    for (long long b = 0; b < batch; ++b)
        for (auto &c : h->cz) {
            cufftComplex *w = reinterpret_cast<cufftComplex *>(h->d_czw + b * h->cz_n + c.woff);
            cufftResult cr = cufftExecC2C(c.plan, w, w, dir);
            if (cr != CUFFT_SUCCESS) return cufft_fail(cr, "sk_harmonic_apply");
        }
    return SK_OK;
}

// The analysis half of the transform: ring DFTs of `batch` maps into h->d_F and the
// Legendre analysis into h->d_a (a_lm, m = 0..L, l = m..L; per map a_n float2).
static int harm_analysis(sk_ctx *ctx, sk_harm *h, const float *d_in, int64_t batch, int64_t map_stride,
                         cudaStream_t st) {
    const sk_geom *g = h->g;
    const int N = (int)g->nside, nr = g->nr, L = h->L, nrh = h->nrh;
    if (batch > h->cap_batch) {
        cudaFree(h->d_F); h->d_F = nullptr;
        cudaFree(h->d_a); h->d_a = nullptr;
        h->cap_batch = 0;
        SK_CU(cudaMalloc(&h->d_F, sizeof(float2) * (size_t)batch * nr * (L + 1)));
        SK_CU(cudaMalloc(&h->d_a, sizeof(float2) * (size_t)batch * h->a_n));
        h->cap_batch = batch;
    }
    const int nb = 2 * N + 1;
    const float domega = (float)(4.0 * SK_PI / (double)g->npix);
    const long long zone0 = g->h_rings[N - 1].start;     // first pixel of the equatorial zone
    (void)ctx;
    if (cufftSetStream(h->p_r2c, st) != CUFFT_SUCCESS || cufftSetStream(h->p_c2r, st) != CUFFT_SUCCESS)
        return sk_fail(SK_ECUDA, "sk_harmonic_apply: cufftSetStream failed");
    // ring DFTs: the cap rings by chirp-z transforms, the zone by one R2C per map
    const int ncap = 2 * (N - 1);
    if (ncap > 0) {
        if (batch > h->cz_batch) {
            cudaFree(h->d_czw); h->d_czw = nullptr;
            h->cz_batch = 0;
            SK_CU(cudaMalloc(&h->d_czw, sizeof(float2) * (size_t)batch * h->cz_n));
            h->cz_batch = batch;
        }
        for (auto &c : h->cz)
            if (cufftSetStream(c.plan, st) != CUFFT_SUCCESS)
                return sk_fail(SK_ECUDA, "sk_harmonic_apply: cufftSetStream failed");
        const dim3 grid(ncap, (unsigned)batch);
        k_cz_a_pre<<<grid, HT, 0, st>>>(h->d_czrow, g->d_rings, nr, d_in, map_stride, h->cz_n, h->d_czw);
        SK_CU(cudaGetLastError());
        if (int rc = cz_fft(h, batch, CUFFT_FORWARD)) return rc;
        k_cz_mul<<<grid, HT, 0, st>>>(h->d_czrow, h->d_czf, 0, h->cz_n, h->d_czw);
        SK_CU(cudaGetLastError());
        if (int rc = cz_fft(h, batch, CUFFT_INVERSE)) return rc;
        k_cz_a_post<<<grid, HT, 0, st>>>(h->d_czrow, nr, L, h->cz_n, h->d_czw, h->d_F);
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
    k_leg_analysis<<<dim3(L + 1, (unsigned)batch), HT, sm_a, st>>>(h->d_lam, h->d_moff, h->d_aoff, h->d_q0, h->d_F,
                                                                    L, nr, nrh, h->a_n, domega, h->d_a);
    SK_CU(cudaGetLastError());
    return SK_OK;
}

// The synthesis half: y (+)= sum_lm K^_l a_lm Y_lm from h->d_a.
static int harm_synthesis(sk_ctx *ctx, sk_harm *h, float *d_out, int64_t batch, int64_t map_stride, int accumulate,
                          cudaStream_t st) {
    const sk_geom *g = h->g;
    const int N = (int)g->nside, nr = g->nr, L = h->L, nrh = h->nrh;
    const int nb = 2 * N + 1, n4 = 4 * N;
    const long long zone0 = g->h_rings[N - 1].start;
    const int ncap = 2 * (N - 1);
    (void)ctx;
    k_leg_synthesis<<<dim3(L + 1, (unsigned)batch), HT, sizeof(float2) * (L + 1), st>>>(
        h->d_lam, h->d_moff, h->d_aoff, h->d_l0w, h->d_kl, h->d_a, L, nr, nrh, h->a_n, h->d_F);
    SK_CU(cudaGetLastError());
    // inverse ring DFTs
    if (ncap > 0) {
        const dim3 grid(ncap, (unsigned)batch);
        k_cz_s_pre<<<grid, HT, 0, st>>>(h->d_czrow, nr, L, h->cz_n, h->d_F, h->d_czw);
        SK_CU(cudaGetLastError());
        if (int rc = cz_fft(h, batch, CUFFT_FORWARD)) return rc;
        k_cz_mul<<<grid, HT, 0, st>>>(h->d_czrow, h->d_czf, 1, h->cz_n, h->d_czw);
        SK_CU(cudaGetLastError());
        if (int rc = cz_fft(h, batch, CUFFT_INVERSE)) return rc;
        k_cz_s_post<<<grid, HT, 0, st>>>(h->d_czrow, g->d_rings, nr, h->cz_n, h->d_czw, d_out, map_stride,
                                         accumulate);
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

static int check_harm_maps(const char *who, const sk_harm *h, const float *in, const float *out, int64_t batch,
                           int64_t map_stride) {
    if (batch < 0 || map_stride < h->g->npix) return sk_fail(SK_EINVAL, "%s: bad batch or stride", who);
    if (batch > 0 && (!in || (out && in == out))) return sk_fail(SK_EINVAL, "%s: NULL or aliasing maps", who);
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15) || (map_stride & 3))
        return sk_fail(SK_EINVAL, "%s: maps must be 16-byte aligned with a stride multiple of 4", who);
    return SK_OK;
}

extern "C" int sk_harmonic_apply(sk_ctx *ctx, const sk_harm *hc, const float *d_in, float *d_out, int64_t batch,
                                 int64_t map_stride, int accumulate, void *stream) {
    if (!ctx || !hc || (!d_in && batch > 0) || (!d_out && batch > 0))
        return sk_fail(SK_EINVAL, "sk_harmonic_apply: NULL argument");
    sk_harm *h = const_cast<sk_harm *>(hc);
    if (int rc = check_harm_maps("sk_harmonic_apply", h, d_in, d_out, batch, map_stride)) return rc;
    if (batch == 0) return SK_OK;
    SK_CU(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = harm_analysis(ctx, h, d_in, batch, map_stride, st)) return rc;
    return harm_synthesis(ctx, h, d_out, batch, map_stride, accumulate, st);
}

// C_l = (|a_l0|^2 + 2 sum_{m>=1} |a_lm|^2) / (2l + 1), in FP64, one thread per (l, map).
__global__ void k_spectrum(const float2 *a, const long long *aoff, int L, long long a_n, int batch, double *cl) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (l > L || b >= batch) return;
    const float2 *ab = a + (long long)b * a_n;
    double s = 0.0;
    for (int m = 0; m <= l; ++m) {
        const float2 v = ab[aoff[m] + (l - m)];
        s += (m == 0 ? 1.0 : 2.0) * ((double)v.x * v.x + (double)v.y * v.y);
    }
    cl[(long long)b * (L + 1) + l] = s / (2.0 * l + 1.0);
}

extern "C" int sk_harmonic_spectrum(sk_ctx *ctx, const sk_harm *hc, const float *d_in, int64_t batch,
                                    int64_t map_stride, double *d_cl, void *stream) {
    if (!ctx || !hc || (batch > 0 && (!d_in || !d_cl))) return sk_fail(SK_EINVAL, "sk_harmonic_spectrum: NULL argument");
    sk_harm *h = const_cast<sk_harm *>(hc);
    if (int rc = check_harm_maps("sk_harmonic_spectrum", h, d_in, nullptr, batch, map_stride)) return rc;
    if (batch == 0) return SK_OK;
    SK_CU(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = harm_analysis(ctx, h, d_in, batch, map_stride, st)) return rc;
    k_spectrum<<<dim3((h->L + HT) / HT, (unsigned)batch), HT, 0, st>>>(h->d_a, h->d_aoff, h->L, h->a_n, (int)batch,
                                                                       d_cl);
    SK_CU(cudaGetLastError());
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
