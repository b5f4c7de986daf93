// fourier.cu -- ring-pair Fourier form of the belt sums, for wide theta_cut.
//
// In the equatorial zone every ring has n = 4 Nside pixels, and for output pixel
// j of ring o and input pixel j + e of ring i the phi difference is
// pi (2e + s_i - s_o) / n: the real-space convolution (Sec. 2, Eq. 1 with the
// tabulated kernel of Sec. 3) restricted to one ring pair is a circular
// correlation along the ring,
//     y_o[j] += sum_e w_oi(e) x_i[(j + e) mod n],
// and a correlation is diagonal in the ring's Fourier modes:
//     Y_o(m) = sum_i W_oi(m) X_i(m),   X_i(m) = sum_k x_i[k] e^{-2 pi i m k / n},
//     W_oi(m) = sum_e w_oi(e) e^{+2 pi i m e / n}.
// The weight depends on the phi difference only through cos, so with
// delta = (s_i - s_o) / 2 in {0, +-1/2}, w_oi(e) = f(e + delta) for an even f and
// W_oi(m) = e^{-2 pi i m delta / n} G_oi(m) with G_oi real.  In the zone s
// alternates from ring to ring: even ring offsets have delta = 0, odd ones the
// same delta, so
//     Y_o(m) = sum_{d even} G X  +  e^{-2 pi i m delta_o / n} sum_{d odd} G X.
// Cost per map: one FFT per ring each way and (2H+1) complex FMAs per output
// mode, linear in theta_cut, where the direct sums grow with its square (the
// paper's Eq. 3 cost model is linear in theta_cut).
//
// G is built once per handle: each weight row w_oi(e) over the whole ring,
// evaluated in FP64 (exact-integer half-angle, FP64 chord, asin and lerp of the
// FP64 node values) and scaled by dOmega / n (the inverse FFT's 1/n), goes
// through a batched FP32 R2C FFT; G_oi(m) = Re(e^{2 pi i m delta / n} conj(R(m))).
// Per call: R2C of the input rings straight from the map, the mode mix (FP32,
// partial sums over blocks of 32 ring offsets), C2R straight into the output
// rings.  The rings this form does not cover (the caps and the rings whose
// window leaves the zone) run through the direct paths with the kernel's own
// plan.
#include <cufft.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "skconv_host.h"

struct sk_fourier {
    sk_ctx *ctx = nullptr;
    int device = 0;                 // the context's device (the handle may outlive the context)
    const sk_kern *k = nullptr;
    int n = 0, M = 0;               // ring length 4 Nside, modes 0 .. n/2
    int f_lo = 0, f_nb = 0;         // output rings [f_lo, f_lo + f_nb) (0-based)
    int in_lo = 0, in_n = 0;        // input rings [in_lo, in_lo + in_n)
    int H = 0;                      // ring offsets -H .. H
    float *d_G = nullptr;           // [f_nb][2H + 1][M]
    size_t g_bytes = 0;
    cufftHandle p_r2c = 0, p_c2r = 0;
    bool plans = false;
    float2 *d_X = nullptr;          // [in_n][M] modes of one map's input rings
    float2 *d_Y = nullptr;          // [f_nb][M] modes of its output rings
    // the other rings: cap items and per-pair items, as a subset of the kernel's work
    int4 *d_items = nullptr;
    SkItems rest;
};

namespace {

int cufft_fail(cufftResult r, const char *what) { return sk_fail(SK_ECUDA, "%s: cuFFT error %d", what, (int)r); }

// Rows rho0 .. rho0 + gridDim.x - 1 of the weight table: row rho = (output ring
// f_lo + rho / (2H+1), offset d = rho % (2H+1) - H), e = 0 .. n-1 (offsets taken
// mod n, signed for the half-angle).  Zero where the ring pair has no window.
__global__ void k_fw_rows(const RingDev *rings, const int *pair_off, const PairInfo *pairs, const double2 *ab64,
                          const double *V, KernParams kp, KernParams64 kd, double scale, int f_lo, int H, int n,
                          long long rho0, float *rows) {
    const long long rho = rho0 + blockIdx.x;
    const int o = f_lo + (int)(rho / (2 * H + 1)), d = (int)(rho % (2 * H + 1)) - H;
    const int i = o + d;
    float *row = rows + (size_t)blockIdx.x * n;
    const int p0 = pair_off[o], cnt = pair_off[o + 1] - p0;
    const int rel = cnt > 0 ? i - pairs[p0].ri : -1;
    if (rel < 0 || rel >= cnt) {
        for (int e = threadIdx.x; e < n; e += blockDim.x) row[e] = 0.0f;
        return;
    }
    const double2 ab = ab64[p0 + rel];
    const int ds = rings[i].s - rings[o].s;
    const double c0 = SK_PI / (2.0 * (double)n);
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int es = e <= n / 2 ? e : e - n;
        int k;
        float fr;
        double w = 0.0;
        if (pair_kf64((double)(2 * es + ds) * c0, ab.x, ab.y, kp, kd, k, fr))
            w = scale * fma((double)fr, V[k + 1] - V[k], V[k]);
        row[e] = (float)w;
    }
}

// G[rho][m] = Re(e^{2 pi i m delta / n} conj(R[rho][m])), delta = (s_i - s_o) / 2.
__global__ void k_fw_finish(const RingDev *rings, const float2 *R, int f_lo, int H, int n, int M, long long rho0,
                            int rows, float *G) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)rows * M) return;
    const int rr = (int)(idx / M), m = (int)(idx % M);
    const long long rho = rho0 + rr;
    const int o = f_lo + (int)(rho / (2 * H + 1)), d = (int)(rho % (2 * H + 1)) - H;
    const int ds = (d & 1) ? 1 - 2 * rings[o].s : 0;     // 2 delta: s alternates in the zone
    const float2 r = R[(size_t)rr * M + m];
    double g = r.x;
    if (ds != 0) {
        double sn, cs;
        sincospi((double)m / (double)n, &sn, &cs);        // e^{i pi m / n}
        g = cs * r.x + (double)ds * sn * r.y;            // Re((cs + i ds sn)(r.x - i r.y))
    }
    G[rho * M + m] = (float)g;
}

// Y[o][m] = sum_{d even} G X + e^{-2 pi i m delta_o / n} sum_{d odd} G X, one thread
// per (output ring, mode), reading G once (coalesced along m); offsets whose input
// ring lies outside the buffer (their G rows are zero) are skipped by the loop
// bounds.  Partial sums over blocks of 32 offsets, two offsets per step.
__global__ void k_fmix(const RingDev *rings, const float *__restrict__ G, const float2 *__restrict__ X, int f_lo,
                       int f_nb, int in_lo, int in_n, int H, int n, int M, float2 *Y) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int oi = blockIdx.y;
    if (m >= M || oi >= f_nb) return;
    const int o = f_lo + oi;
    const int dlo = max(0, in_lo - (o - H)), dhi = min(2 * H, in_lo + in_n - 1 - (o - H));
    const float *g = G + (size_t)oi * (2 * H + 1) * M + m;
    const float2 *x = X + (ptrdiff_t)(o - H - in_lo) * M + m;
    // accumulators a0 (offsets dlo, dlo + 2, ...) and a1 (dlo + 1, ...); even ring offsets
    // d = dd - H are a0 when dlo - H is even
    float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
    for (int d0 = dlo; d0 <= dhi; d0 += 32) {
        const int d1 = min(d0 + 31, dhi);
        float2 b0 = make_float2(0.f, 0.f), b1 = make_float2(0.f, 0.f);
        int dd = d0;
#pragma unroll 8
        for (; dd + 1 <= d1; dd += 2) {
            const float g0 = g[(size_t)dd * M], g1 = g[(size_t)(dd + 1) * M];
            const float2 x0 = x[(size_t)dd * M], x1 = x[(size_t)(dd + 1) * M];
            b0.x = fmaf(g0, x0.x, b0.x); b0.y = fmaf(g0, x0.y, b0.y);
            b1.x = fmaf(g1, x1.x, b1.x); b1.y = fmaf(g1, x1.y, b1.y);
        }
        if (dd == d1) {
            const float g0 = g[(size_t)dd * M];
            const float2 x0 = x[(size_t)dd * M];
            b0.x = fmaf(g0, x0.x, b0.x); b0.y = fmaf(g0, x0.y, b0.y);
        }
        a0.x += b0.x; a0.y += b0.y;
        a1.x += b1.x; a1.y += b1.y;
    }
    const bool swap = ((dlo - H) & 1) != 0;
    const float2 ev = swap ? a1 : a0, od = swap ? a0 : a1;
    // odd offsets: s_i = 1 - s_o in the zone, 2 delta_o = 1 - 2 s_o; phase e^{-i pi m (1 - 2 s_o) / n}
    const int ds = 1 - 2 * rings[o].s;
    float sn, cs;
    sincospif((float)m / (float)n, &sn, &cs);
    const float ps = -(float)ds * sn;                     // e^{-i pi m ds / n} = cs + i ps
    Y[(size_t)oi * M + m] = make_float2(ev.x + cs * od.x - ps * od.y, ev.y + cs * od.y + ps * od.x);
}

void free_fourier(sk_fourier *f) {
    if (!f) return;
    if (f->plans) { cufftDestroy(f->p_r2c); cufftDestroy(f->p_c2r); }
    cudaFree(f->d_G);
    cudaFree(f->d_X);
    cudaFree(f->d_Y);
    cudaFree(f->d_items);
    delete f;
}

}  // namespace

extern "C" int sk_fourier_create(sk_ctx *ctx, const sk_kern *k, sk_fourier **out) {
    if (!out) return sk_fail(SK_EINVAL, "sk_fourier_create: NULL out");
    *out = nullptr;
    if (!ctx || !k) return sk_fail(SK_EINVAL, "sk_fourier_create: NULL argument");
    SK_CU(cudaSetDevice(ctx->device));
    const sk_geom *g = k->g;
    const int nr = g->nr, N = (int)g->nside;
    const int z0 = N - 1, z1 = 3 * N - 1;                 // rings of 4N pixels (0-based)
    sk_fourier *f = new sk_fourier();
    f->ctx = ctx;
    f->device = ctx->device;
    f->k = k;
    f->n = 4 * N;
    f->M = 2 * N + 1;
    // output rings whose whole window lies in the zone (a contiguous range)
    int lo = -1, hi = -2;
    for (int r = z0; r <= z1; ++r)
        if (k->h_lo[r] >= z0 && k->h_hi[r] <= z1 && k->h_pair_off[r + 1] > k->h_pair_off[r]) {
            if (lo < 0) lo = r;
            hi = r;
        }
    if (lo >= 0 && N >= 2) {
        f->f_lo = lo;
        f->f_nb = hi - lo + 1;
        int ilo = z1, ihi = z0;
        for (int r = lo; r <= hi; ++r) {
            f->H = std::max(f->H, std::max(r - k->h_lo[r], k->h_hi[r] - r));
            ilo = std::min(ilo, k->h_lo[r]);
            ihi = std::max(ihi, k->h_hi[r]);
        }
        // the mode mix reads X for every offset -H .. H of every output ring
        ilo = std::min(ilo, lo - f->H);
        ihi = std::max(ihi, hi + f->H);
        f->in_lo = std::max(ilo, z0);
        f->in_n = std::min(ihi, z1) - f->in_lo + 1;
    }
    int rc = SK_OK;
    auto fail = [&](int code) { free_fourier(f); return code; };
    if (f->f_nb > 0) {
        const int n = f->n, M = f->M, R2 = 2 * f->H + 1;
        const long long rows = (long long)f->f_nb * R2;
        f->g_bytes = (size_t)rows * M * sizeof(float);
        cudaError_t e = cudaMalloc(&f->d_G, f->g_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&f->d_X, sizeof(float2) * (size_t)f->in_n * M);
        if (e == cudaSuccess) e = cudaMalloc(&f->d_Y, sizeof(float2) * (size_t)f->f_nb * M);
        if (e != cudaSuccess) return fail(sk_fail(SK_ENOMEM, "sk_fourier_create: %s", cudaGetErrorString(e)));
        // per-call plans: the input rings and the output rings of one map
        int len[1] = {n};
        int inem[1] = {n}, onem[1] = {M};
        cufftResult cr = cufftPlanMany(&f->p_r2c, 1, len, inem, 1, n, onem, 1, M, CUFFT_R2C, f->in_n);
        if (cr == CUFFT_SUCCESS) cr = cufftPlanMany(&f->p_c2r, 1, len, onem, 1, M, inem, 1, n, CUFFT_C2R, f->f_nb);
        if (cr != CUFFT_SUCCESS) return fail(cufft_fail(cr, "sk_fourier_create"));
        f->plans = true;
        // the weight table, in chunks of rows
        const long long chunk = std::max(1LL, std::min(rows, (long long)((256LL << 20) / ((long long)n * 4))));
        float *d_rows = nullptr;
        float2 *d_R = nullptr;
        cufftHandle p_w = 0;
        e = cudaMalloc(&d_rows, sizeof(float) * (size_t)chunk * n);
        if (e == cudaSuccess) e = cudaMalloc(&d_R, sizeof(float2) * (size_t)chunk * M);
        if (e != cudaSuccess) {
            cudaFree(d_rows);
            return fail(sk_fail(SK_ENOMEM, "sk_fourier_create: %s", cudaGetErrorString(e)));
        }
        const double scale = 4.0 * SK_PI / (double)g->npix / (double)n;
        for (long long r0 = 0; r0 < rows && rc == SK_OK; r0 += chunk) {
            const int nrow = (int)std::min(chunk, rows - r0);
            cr = cufftPlanMany(&p_w, 1, len, inem, 1, n, onem, 1, M, CUFFT_R2C, nrow);
            if (cr != CUFFT_SUCCESS) { rc = cufft_fail(cr, "sk_fourier_create"); break; }
            k_fw_rows<<<nrow, 256>>>(g->d_rings, k->d_pair_off, k->d_pairs, k->d_ab64, k->d_V, k->kp, k->kd, scale,
                                     f->f_lo, f->H, n, r0, d_rows);
            cr = cufftExecR2C(p_w, d_rows, reinterpret_cast<cufftComplex *>(d_R));
            if (cr != CUFFT_SUCCESS) rc = cufft_fail(cr, "sk_fourier_create");
            const long long tot = (long long)nrow * M;
            if (rc == SK_OK)
                k_fw_finish<<<(unsigned)((tot + 255) / 256), 256>>>(g->d_rings, d_R, f->f_lo, f->H, n, M, r0, nrow,
                                                                    f->d_G);
            cufftDestroy(p_w);
            e = cudaGetLastError();
            if (rc == SK_OK && e != cudaSuccess) rc = sk_fail(SK_ECUDA, "sk_fourier_create: %s", cudaGetErrorString(e));
        }
        e = cudaDeviceSynchronize();
        cudaFree(d_rows);
        cudaFree(d_R);
        if (rc) return fail(rc);
        if (e != cudaSuccess) return fail(sk_fail(SK_ECUDA, "sk_fourier_create: %s", cudaGetErrorString(e)));
    }
    // the other rings: the kernel's cap items outside the Fourier range, per-pair items
    // for every ring neither covers
    {
        auto fourier = [&](int r) { return f->f_nb > 0 && r >= f->f_lo && r < f->f_lo + f->f_nb; };
        std::vector<int4> all;
        std::vector<unsigned char> covered(nr, 0);
        for (int r = 0; r < nr; ++r) covered[r] = fourier(r);
        size_t off_cap[SK_CAP_LS_CLASSES][2], n_cap[SK_CAP_LS_CLASSES][2];
        for (int c = 0; c < SK_CAP_LS_CLASSES; ++c)
            for (int v = 0; v < 2; ++v) {
                off_cap[c][v] = all.size();
                if (k->plan_ok)
                    for (const int4 &it : k->h_items_cap[c][v])
                        if (!fourier(it.x) && !fourier(nr - 1 - it.x)) {
                            all.push_back(it);
                            covered[it.x] = covered[nr - 1 - it.x] = 1;
                        }
                n_cap[c][v] = all.size() - off_cap[c][v];
            }
        const size_t off_gen = all.size();
        const auto &R = g->h_rings;
        for (int r = 0; r < nr; ++r)
            if (!covered[r])
                for (int j = 0; j < R[r].n; j += 128) all.push_back(make_int4(r, j, 0, 0));
        const size_t n_gen = all.size() - off_gen;
        if (!all.empty()) {
            cudaError_t e = cudaMalloc(&f->d_items, sizeof(int4) * all.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(f->d_items, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return fail(sk_fail(SK_ENOMEM, "sk_fourier_create: %s", cudaGetErrorString(e)));
        }
        for (int c = 0; c < SK_CAP_LS_CLASSES; ++c)
            for (int v = 0; v < 2; ++v) {
                f->rest.cap[c][v] = n_cap[c][v] ? f->d_items + off_cap[c][v] : nullptr;
                f->rest.n_cap[c][v] = (int)n_cap[c][v];
            }
        f->rest.gen = n_gen ? f->d_items + off_gen : nullptr;
        f->rest.n_gen = (int)n_gen;
        f->rest.sym[0][0] = 0;
        f->rest.sym[0][1] = k->sym_hi;
    }
    *out = f;
    return SK_OK;
}

extern "C" int sk_fourier_destroy(sk_fourier *f) {
    if (!f) return SK_OK;
    cudaSetDevice(f->device);
    free_fourier(f);
    return SK_OK;
}

extern "C" int sk_fourier_info(const sk_fourier *f, int64_t *out4) {
    if (!f || !out4) return sk_fail(SK_EINVAL, "sk_fourier_info: NULL argument");
    out4[0] = f->f_lo;
    out4[1] = f->f_nb;
    out4[2] = f->H;
    out4[3] = (int64_t)f->g_bytes;
    return SK_OK;
}

extern "C" int sk_fourier_apply(sk_ctx *ctx, const sk_fourier *f, const float *d_in, float *d_out, int64_t batch,
                                int64_t map_stride, void *stream) {
    if (!ctx || !f) return sk_fail(SK_EINVAL, "sk_fourier_apply: NULL argument");
    int rc = sk_check_maps("sk_fourier_apply", f->k, d_in, d_out, batch, map_stride);
    if (rc || batch == 0) return rc;
    SK_CU(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const sk_kern *k = f->k;
    // the rings outside the Fourier range, through the kernel's direct paths
    SkJob jb{k, d_in, d_out, batch, map_stride};
    jb.sub = &f->rest;
    jb.weights = false;
    void *ws = nullptr;
    if ((rc = sk_ctx_workspace(ctx, sk_jobs_workspace_bytes(&jb, 1), &ws))) return rc;
    if ((rc = sk_run_jobs(ctx, &jb, 1, SK_PATH_AUTO, ws, st))) return rc;
    if (f->f_nb == 0) return SK_OK;
    if (cufftSetStream(f->p_r2c, st) != CUFFT_SUCCESS || cufftSetStream(f->p_c2r, st) != CUFFT_SUCCESS)
        return sk_fail(SK_ECUDA, "sk_fourier_apply: cufftSetStream failed");
    const auto &R = k->g->h_rings;
    for (int64_t b = 0; b < batch; ++b) {
        const float *xin = d_in + b * map_stride + R[f->in_lo].start;
        float *yout = d_out + b * map_stride + R[f->f_lo].start;
        cudaEvent_t ev = sk_prof_begin(ctx, st);
        cufftResult cr = cufftExecR2C(f->p_r2c, const_cast<float *>(xin), reinterpret_cast<cufftComplex *>(f->d_X));
        if (cr != CUFFT_SUCCESS) return cufft_fail(cr, "sk_fourier_apply");
        sk_prof_end(ctx, "fourier_fft", ev, st);
        ev = sk_prof_begin(ctx, st);
        dim3 grid((f->M + 127) / 128, f->f_nb);
        k_fmix<<<grid, 128, 0, st>>>(k->g->d_rings, f->d_G, f->d_X, f->f_lo, f->f_nb, f->in_lo, f->in_n, f->H, f->n,
                                     f->M, f->d_Y);
        SK_CU(cudaGetLastError());
        sk_prof_end(ctx, "fourier_mix", ev, st);
        ev = sk_prof_begin(ctx, st);
        cr = cufftExecC2R(f->p_c2r, reinterpret_cast<cufftComplex *>(f->d_Y), yout);
        if (cr != CUFFT_SUCCESS) return cufft_fail(cr, "sk_fourier_apply");
        sk_prof_end(ctx, "fourier_fft", ev, st);
    }
    return SK_OK;
}
