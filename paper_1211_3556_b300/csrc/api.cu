// api.cu -- the C ABI (include/skconv.h): handles, set-up and argument checks.
// Launch sequences live in plan.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "skconv_host.h"

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------

static thread_local std::string g_last_error;

int sk_fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

extern "C" const char *sk_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

int sk_ctx_workspace(sk_ctx *ctx, size_t bytes, void **out) {
    if (bytes > ctx->ws_bytes && ctx->ws_limit && bytes > ctx->ws_limit)
        return sk_fail(SK_ENOMEM, "workspace of %zu bytes over the context's limit of %zu bytes", bytes,
                       ctx->ws_limit);
    if (bytes > ctx->ws_bytes) {
        if (ctx->ws) cudaFree(ctx->ws);          // cudaFree waits for work using it
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
        size_t b = std::max(bytes, (size_t)1 << 20);
        if (ctx->ws_limit) b = std::min(b, std::max(bytes, ctx->ws_limit));
        SK_CU(cudaMalloc(&ctx->ws, b));
        ctx->ws_bytes = b;
    }
    *out = ctx->ws;
    return SK_OK;
}

extern "C" int sk_set_workspace_limit(sk_ctx *ctx, int64_t bytes) {
    if (!ctx) return sk_fail(SK_EINVAL, "sk_set_workspace_limit: NULL context");
    if (bytes < 0) return sk_fail(SK_EINVAL, "sk_set_workspace_limit: bytes %lld < 0", (long long)bytes);
    ctx->ws_limit = (size_t)bytes;
    return SK_OK;
}

extern "C" int sk_create(sk_ctx **out, int device) {
    if (!out) return sk_fail(SK_EINVAL, "sk_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    SK_CU(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return sk_fail(SK_EINVAL, "sk_create: device %d of %d", device, ndev);
    SK_CU(cudaSetDevice(device));
    sk_ctx *c = new sk_ctx();
    c->device = device;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_queue, sizeof(int) * sk_ctx::NQUEUE);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_sym, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaFree(c->d_status);
        cudaFree(c->d_queue);
        if (c->aux) cudaStreamDestroy(c->aux);
        if (c->ev_fork) cudaEventDestroy(c->ev_fork);
        if (c->ev_join) cudaEventDestroy(c->ev_join);
        if (c->ev_sym) cudaEventDestroy(c->ev_sym);
        delete c;
        return sk_fail(SK_ECUDA, "sk_create: %s", cudaGetErrorString(e));
    }
    c->num_sms = prop.multiProcessorCount;
    *out = c;
    return SK_OK;
}

extern "C" int sk_destroy(sk_ctx *ctx) {
    if (!ctx) return SK_OK;
    cudaSetDevice(ctx->device);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->d_queue) cudaFree(ctx->d_queue);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    if (ctx->h2d) cudaStreamDestroy(ctx->h2d);
    if (ctx->d2h) cudaStreamDestroy(ctx->d2h);
    for (int b = 0; b < SK_HOST_BANDS; ++b) {
        if (ctx->ev_in[b]) cudaEventDestroy(ctx->ev_in[b]);
        if (ctx->ev_out[b]) cudaEventDestroy(ctx->ev_out[b]);
    }
    if (ctx->ev_done) cudaEventDestroy(ctx->ev_done);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ev_sym) cudaEventDestroy(ctx->ev_sym);
    delete ctx;
    return SK_OK;
}

cudaEvent_t sk_prof_begin(sk_ctx *ctx, cudaStream_t st) {
    if (!ctx->prof) return nullptr;
    cudaEvent_t a = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess) return nullptr;
    cudaEventRecord(a, st);
    return a;
}

void sk_prof_end(sk_ctx *ctx, const char *name, cudaEvent_t a, cudaStream_t st) {
    if (!ctx->prof || !a) return;
    cudaEvent_t b = nullptr;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
    cudaEventRecord(b, st);
    ctx->prof_recs.push_back({name, a, b});
}

extern "C" int sk_profile_enable(sk_ctx *ctx, int on) {
    if (!ctx) return sk_fail(SK_EINVAL, "sk_profile_enable: NULL context");
    ctx->prof = on != 0;
    return SK_OK;
}

extern "C" int sk_profile_read(sk_ctx *ctx, int max_kernels, char *names, double *ms, int *launches,
                               int *n_kernels) {
    if (!ctx || !n_kernels) return sk_fail(SK_EINVAL, "sk_profile_read: NULL argument");
    SK_CU(cudaSetDevice(ctx->device));
    std::vector<std::string> nm;
    std::vector<double> tot;
    std::vector<int> cnt;
    int rc = SK_OK;
    for (auto &r : ctx->prof_recs) {
        float t = 0.0f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
            rc = sk_fail(SK_ECUDA, "sk_profile_read: event failed");
        size_t i = 0;
        while (i < nm.size() && nm[i] != r.name) ++i;
        if (i == nm.size()) { nm.push_back(r.name); tot.push_back(0.0); cnt.push_back(0); }
        tot[i] += t;
        cnt[i] += 1;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    ctx->prof_recs.clear();
    int n = (int)nm.size();
    *n_kernels = n;
    for (int i = 0; i < n && i < max_kernels; ++i) {
        if (names) { strncpy(names + 32 * i, nm[i].c_str(), 31); names[32 * i + 31] = 0; }
        if (ms) ms[i] = tot[i];
        if (launches) launches[i] = cnt[i];
    }
    return rc;
}

extern "C" int sk_get_status(sk_ctx *ctx, void *stream) {
    if (!ctx) return sk_fail(SK_EINVAL, "sk_get_status: NULL context");
    SK_CU(cudaSetDevice(ctx->device));
    SK_CU(cudaStreamSynchronize((cudaStream_t)stream));
    int st = 0;
    SK_CU(cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    SK_CU(cudaMemset(ctx->d_status, 0, sizeof(int)));
    if (st != 0) return sk_fail(st, "device status word: %d", st);
    return SK_OK;
}

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------

static bool valid_nside(int64_t n) { return n >= 1 && n <= 8192 && (n & (n - 1)) == 0; }

extern "C" int64_t sk_npix(int64_t nside) { return valid_nside(nside) ? 12 * nside * nside : -1; }

extern "C" int sk_geometry_destroy(sk_geom *g) {
    if (!g) return SK_OK;
    cudaSetDevice(g->device);
    cudaFree(g->d_rings); cudaFree(g->d_z); cudaFree(g->d_rho); cudaFree(g->d_theta);
    delete g;
    return SK_OK;
}

extern "C" int sk_geometry_create(sk_ctx *ctx, int64_t nside, sk_geom **out) {
    if (!ctx || !out) return sk_fail(SK_EINVAL, "sk_geometry_create: NULL argument");
    *out = nullptr;
    if (!valid_nside(nside)) return sk_fail(SK_EINVAL, "nside %lld is not a power of two in [1, 8192]", (long long)nside);
    SK_CU(cudaSetDevice(ctx->device));
    sk_geom *g = new sk_geom();
    g->ctx = ctx;
    g->device = ctx->device;
    g->nside = nside;
    g->npix = 12 * nside * nside;
    g->nr = (int)(4 * nside - 1);
    const int nr = g->nr;
    cudaError_t e = cudaMalloc(&g->d_rings, sizeof(RingDev) * nr);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_z, sizeof(double) * nr);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_rho, sizeof(double) * nr);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_theta, sizeof(double) * nr);
    if (e == cudaSuccess) e = sk_launch_ring_geom(nside, g->d_rings, g->d_z, g->d_rho, g->d_theta, 0);
    if (e == cudaSuccess) {
        g->h_rings.resize(nr);
        e = cudaMemcpy(g->h_rings.data(), g->d_rings, sizeof(RingDev) * nr, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) {
        sk_geometry_destroy(g);
        return sk_fail(e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA, "sk_geometry_create: %s",
                       cudaGetErrorString(e));
    }
    *out = g;
    return SK_OK;
}

extern "C" int sk_geometry_rings(const sk_geom *g, int32_t *h_n, int64_t *h_start, int32_t *h_shift,
                                 double *h_z, double *h_sinth) {
    if (!g) return sk_fail(SK_EINVAL, "sk_geometry_rings: NULL geometry");
    SK_CU(cudaSetDevice(g->ctx->device));
    for (int r = 0; r < g->nr; ++r) {
        if (h_n) h_n[r] = g->h_rings[r].n;
        if (h_start) h_start[r] = g->h_rings[r].start;
        if (h_shift) h_shift[r] = g->h_rings[r].s;
    }
    if (h_z) SK_CU(cudaMemcpy(h_z, g->d_z, sizeof(double) * g->nr, cudaMemcpyDeviceToHost));
    if (h_sinth) SK_CU(cudaMemcpy(h_sinth, g->d_rho, sizeof(double) * g->nr, cudaMemcpyDeviceToHost));
    return SK_OK;
}

// ---------------------------------------------------------------------------
// kernel (operator) handles
// ---------------------------------------------------------------------------

static void free_kern(sk_kern *k) {
    if (!k) return;
    cudaFree(k->d_changed);
    cudaFree(k->d_V); cudaFree(k->d_tab); cudaFree(k->d_pair_off); cudaFree(k->d_pairs);
    cudaFree(k->d_dphimax); cudaFree(k->d_items_all); cudaFree(k->d_ab64);
    sk_plan_free(k);
    delete k;
}

extern "C" int sk_kernel_destroy(sk_kern *k) {
    if (!k) return SK_OK;
    cudaSetDevice(k->device);
    free_kern(k);
    return SK_OK;
}

static int check_table_args(int64_t n_nodes, double tc, int layout) {
    if (layout != SK_NODES_UNIFORM && layout != SK_NODES_BIASED)
        return sk_fail(SK_EINVAL, "unknown node layout %d", layout);
    if (n_nodes < 2 || (layout == SK_NODES_BIASED && n_nodes < 4))
        return sk_fail(SK_EINVAL, "n_nodes %lld too small for layout %d", (long long)n_nodes, layout);
    if (n_nodes > SK_MAX_NODES)
        return sk_fail(SK_EUNSUPPORTED, "n_nodes %lld > %d", (long long)n_nodes, SK_MAX_NODES);
    if (!(tc > 0.0) || tc > SK_PI) return sk_fail(SK_EINVAL, "theta_cut %g outside (0, pi]", tc);
    return SK_OK;
}

// Builds everything else from node values already on the device (k->d_V).
static int finish_kernel(sk_kern *k) {
    const sk_geom *g = k->g;
    const int nr = g->nr;
    const double tc = k->tc;
    const int nt = k->nt;

    SK_CU(cudaMalloc(&k->d_tab, sizeof(float2) * nt));
    SK_CU(sk_launch_make_table(k->d_V, nt, 4.0 * SK_PI / (double)g->npix, k->d_tab, 0));

    KernParams &kp = k->kp;
    kp.nt = nt;
    kp.layout = k->layout;
    const double sh = sin(0.5 * tc);
    kp.tcut = (float)(4.0 * sh * sh);
    if (k->layout == SK_NODES_UNIFORM) {
        kp.inv_h = (float)((double)(nt - 1) / tc);
        kp.t1 = 0.0f; kp.inv_h2 = 0.0f; kp.Mf = 0.0f;
    } else {
        const int M = nt / 2;
        const double t1 = tc / 16.0;
        kp.inv_h = (float)((double)M / t1);
        kp.t1 = (float)t1;
        kp.inv_h2 = (float)((double)(nt - 1 - M) / (tc - t1));
        kp.Mf = (float)M;
    }
    // the FP32 asin series to t^2 holds to 8e-9 relative up to theta_cut = 0.15
    kp.small_angle = tc <= 0.15 ? 1 : 0;
    {
        const double coef[5] = {1.0, 1.0 / 24.0, 3.0 / 640.0, 0.0, 0.0};
        const double ih = (double)(nt - 1) / tc;       // uniform layout only
        for (int i = 0; i < 5; ++i) kp.sa[i] = (float)(ih * coef[i]);
        kp.umax = (float)(nt - 1) - 1.0f / 256.0f;
        kp.umax_pad = (float)nt + 0.25f;
    }
    KernParams64 &kd = k->kd;
    kd.tcut = 4.0 * sh * sh;
    if (k->layout == SK_NODES_UNIFORM) {
        kd.inv_h = (double)(nt - 1) / tc;
        kd.t1 = 0.0; kd.inv_h2 = 0.0; kd.Mf = 0.0;
    } else {
        const int M = nt / 2;
        kd.t1 = tc / 16.0;
        kd.inv_h = (double)M / kd.t1;
        kd.inv_h2 = (double)(nt - 1 - M) / (tc - kd.t1);
        kd.Mf = (double)M;
    }

    int *d_lo = nullptr, *d_hi = nullptr;
    SK_CU(cudaMalloc(&d_lo, sizeof(int) * nr));
    cudaError_t e = cudaMalloc(&d_hi, sizeof(int) * nr);
    if (e == cudaSuccess) e = sk_launch_pair_ranges(nr, g->d_theta, tc, d_lo, d_hi, 0);
    k->h_lo.resize(nr);
    k->h_hi.resize(nr);
    if (e == cudaSuccess) e = cudaMemcpy(k->h_lo.data(), d_lo, sizeof(int) * nr, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(k->h_hi.data(), d_hi, sizeof(int) * nr, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
        k->h_pair_off.assign(nr + 1, 0);
        for (int r = 0; r < nr; ++r) k->h_pair_off[r + 1] = k->h_pair_off[r] + (k->h_hi[r] - k->h_lo[r] + 1);
        k->n_pairs = k->h_pair_off[nr];
        e = cudaMalloc(&k->d_pair_off, sizeof(int) * (nr + 1));
    }
    if (e == cudaSuccess) e = cudaMalloc(&k->d_pairs, sizeof(PairInfo) * k->n_pairs);
    if (e == cudaSuccess) e = cudaMalloc(&k->d_dphimax, sizeof(double) * k->n_pairs);
    if (e == cudaSuccess) e = cudaMalloc(&k->d_ab64, sizeof(double2) * k->n_pairs);
    if (e == cudaSuccess) e = cudaMemcpy(k->d_pair_off, k->h_pair_off.data(), sizeof(int) * (nr + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = sk_launch_pair_info(nr, g->d_rings, g->d_z, g->d_rho, g->d_theta, k->d_pair_off, d_lo, tc,
                                k->d_pairs, k->d_dphimax, k->d_ab64, 0);
    if (e == cudaSuccess) {
        k->h_pairs.resize(k->n_pairs);
        e = cudaMemcpy(k->h_pairs.data(), k->d_pairs, sizeof(PairInfo) * k->n_pairs, cudaMemcpyDeviceToHost);
    }
    cudaFree(d_lo);
    cudaFree(d_hi);
    if (e != cudaSuccess)
        return sk_fail(e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA, "pair tables: %s", cudaGetErrorString(e));

    std::vector<int4> items;
    for (int r = 0; r < nr; ++r)
        for (int j = 0; j < g->h_rings[r].n; j += 128) items.push_back(make_int4(r, j, 0, 0));
    k->n_items_all = (int)items.size();
    SK_CU(cudaMalloc(&k->d_items_all, sizeof(int4) * items.size()));
    SK_CU(cudaMemcpy(k->d_items_all, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));

    int rc = sk_plan_build(k);
    if (rc) return rc;
    rc = sk_capw_build(k);
    if (rc) return rc;
    rc = sk_beltw_build(k);
    if (rc) return rc;
    SK_CU(cudaDeviceSynchronize());
    return SK_OK;
}

static sk_kern *new_kernel(sk_ctx *ctx, const sk_geom *g, int64_t n_nodes, double tc, int layout) {
    sk_kern *k = new sk_kern();
    k->ctx = ctx;
    k->device = ctx->device;
    k->g = g;
    k->nt = (int)n_nodes;
    k->tc = tc;
    k->layout = layout;
    return k;
}

extern "C" int sk_kernel_create(sk_ctx *ctx, const sk_geom *g, const double *h_values, int64_t n_nodes,
                                double theta_cut, int layout, sk_kern **out) {
    if (!ctx || !g || !h_values || !out) return sk_fail(SK_EINVAL, "sk_kernel_create: NULL argument");
    *out = nullptr;
    int rc = check_table_args(n_nodes, theta_cut, layout);
    if (rc) return rc;
    SK_CU(cudaSetDevice(ctx->device));
    sk_kern *k = new_kernel(ctx, g, n_nodes, theta_cut, layout);
    cudaError_t e = cudaMalloc(&k->d_V, sizeof(double) * n_nodes);
    if (e == cudaSuccess) e = cudaMemcpy(k->d_V, h_values, sizeof(double) * n_nodes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_kern(k);
        return sk_fail(e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA, "sk_kernel_create: %s", cudaGetErrorString(e));
    }
    rc = finish_kernel(k);
    if (rc) { free_kern(k); return rc; }
    *out = k;
    return SK_OK;
}

extern "C" int sk_kernel_from_legendre(sk_ctx *ctx, const sk_geom *g, const double *h_kl, int64_t lmin,
                                       int64_t lmax, int64_t n_nodes, double theta_cut, int layout,
                                       double taper_start, double *h_values_out, sk_kern **out) {
    if (!ctx || !g || !h_kl) return sk_fail(SK_EINVAL, "sk_kernel_from_legendre: NULL argument");
    if (out) *out = nullptr;
    if (lmax < 0 || lmin < 0 || lmin > lmax || lmax > 1000000)
        return sk_fail(SK_EINVAL, "bad l range [%lld, %lld]", (long long)lmin, (long long)lmax);
    int rc = check_table_args(n_nodes, theta_cut, layout);
    if (rc) return rc;
    SK_CU(cudaSetDevice(ctx->device));
    double *d_kl = nullptr, *d_V = nullptr;
    SK_CU(cudaMalloc(&d_kl, sizeof(double) * (lmax + 1)));
    cudaError_t e = cudaMalloc(&d_V, sizeof(double) * n_nodes);
    if (e == cudaSuccess) e = cudaMemcpy(d_kl, h_kl, sizeof(double) * (lmax + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = sk_launch_tabulate(d_kl, (int)lmin, (int)lmax, (int)n_nodes, theta_cut, layout, taper_start, d_V, 0);
    if (e == cudaSuccess && h_values_out)
        e = cudaMemcpy(h_values_out, d_V, sizeof(double) * n_nodes, cudaMemcpyDeviceToHost);
    cudaFree(d_kl);
    if (e != cudaSuccess) {
        cudaFree(d_V);
        return sk_fail(e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA, "tabulation: %s", cudaGetErrorString(e));
    }
    if (!out) { cudaFree(d_V); return SK_OK; }
    sk_kern *k = new_kernel(ctx, g, n_nodes, theta_cut, layout);
    k->d_V = d_V;
    rc = finish_kernel(k);
    if (rc) { free_kern(k); return rc; }
    *out = k;
    return SK_OK;
}

extern "C" int sk_kernel_update_values(sk_kern *k, const double *h_values) {
    if (!k || !h_values) return sk_fail(SK_EINVAL, "sk_kernel_update_values: NULL argument");
    SK_CU(cudaSetDevice(k->ctx->device));
    SK_CU(cudaDeviceSynchronize());                 // no launch may still read the old table
    SK_CU(cudaMemcpy(k->d_V, h_values, sizeof(double) * k->nt, cudaMemcpyHostToDevice));
    SK_CU(sk_launch_make_table(k->d_V, k->nt, 4.0 * SK_PI / (double)k->g->npix, k->d_tab, 0));
    if (k->d_capw) {
        int rc = sk_capw_build(k);                  // the stored cap weights follow the table
        if (rc) return rc;
    }
    if (k->d_beltw) {
        int rc = sk_beltw_build(k);                 // and the stored belt rows
        if (rc) return rc;
    }
    for (int f = 0; f < 2; ++f)
        if (k->tcp[f].d_A) {
            int rc = sk_tca_build(k, f);            // and the tensor-core belt's tiles
            if (rc) return rc;
        }
    SK_CU(cudaDeviceSynchronize());
    return SK_OK;
}

extern "C" int sk_kernel_update_values_async(sk_kern *k, const double *d_values, void *stream) {
    if (!k || !d_values) return sk_fail(SK_EINVAL, "sk_kernel_update_values_async: NULL argument");
    SK_CU(cudaSetDevice(k->ctx->device));
    if (!k->d_changed) SK_CU(cudaMalloc(&k->d_changed, sizeof(int)));
    cudaStream_t st = (cudaStream_t)stream;
    SK_CU(sk_launch_update_values(d_values, k->d_V, k->nt, k->d_changed, st));
    SK_CU(sk_launch_make_table(k->d_V, k->nt, 4.0 * SK_PI / (double)k->g->npix, k->d_tab, st, k->d_changed));
    if (k->d_beltw) {
        int rc = sk_beltw_build(k, st, k->d_changed);
        if (rc) return rc;
    }
    for (int f = 0; f < 2; ++f)
        if (k->tcp[f].d_A) {
            int rc = sk_tca_build(k, f, st, k->d_changed);
            if (rc) return rc;
        }
    if (k->d_capw) return sk_capw_build(k, false, st, k->d_changed);
    return SK_OK;
}

extern "C" int sk_kernel_set_cap_weights(sk_kern *k, int stored) {
    if (!k || (stored != 0 && stored != 1)) return sk_fail(SK_EINVAL, "sk_kernel_set_cap_weights: bad argument");
    SK_CU(cudaSetDevice(k->ctx->device));
    SK_CU(cudaDeviceSynchronize());                 // no launch may still read the weights
    k->capw_wanted = stored != 0;
    if (!stored) {
        sk_capw_free(k);
        return SK_OK;
    }
    if (k->d_capw) return SK_OK;
    int rc = sk_capw_build(k, true);
    if (rc) return rc;
    SK_CU(cudaDeviceSynchronize());
    if (!k->d_capw && k->capw_len > 0)
        return sk_fail(SK_ENOMEM, "sk_kernel_set_cap_weights: %lld bytes of weights do not fit",
                       (long long)k->capw_len * 16);
    return SK_OK;
}

extern "C" int sk_kernel_set_belt_form(sk_kern *k, int form) {
    if (!k || (form != SK_BELT_FP32 && form != SK_BELT_TENSOR && form != SK_BELT_BF16X3))
        return sk_fail(SK_EINVAL, "sk_kernel_set_belt_form: bad argument");
    if (form == SK_BELT_FP32) {
        k->belt_form = form;
        return SK_OK;
    }
    const int f = form == SK_BELT_BF16X3 ? 1 : 0;
    TcPlan &T = k->tcp[f];
    if (!T.ok) return sk_fail(SK_EINVAL, "sk_kernel_set_belt_form: the operator has no such tensor belt form");
    SK_CU(cudaSetDevice(k->ctx->device));
    if (!T.d_A) {
        int rc = sk_tca_build(k, f);
        if (rc) return rc;
        SK_CU(cudaDeviceSynchronize());
        if (!T.d_A)
            return sk_fail(SK_ENOMEM, "sk_kernel_set_belt_form: %lld KB of weight tiles do not fit", (long long)T.kb);
    }
    k->belt_form = form;
    return SK_OK;
}

extern "C" int sk_kernel_get_config(const sk_kern *k, int64_t *out4) {
    if (!k || !out4) return sk_fail(SK_EINVAL, "sk_kernel_get_config: NULL argument");
    out4[0] = k->belt_P;
    out4[1] = k->belt_form;
    out4[2] = k->d_capw ? 1 : 0;
    out4[3] = (k->tcp[0].ok ? 1 : 0) | (k->tcp[1].ok ? 2 : 0);
    return SK_OK;
}

extern "C" int sk_kernel_cap_weight_bytes(const sk_kern *k, int64_t *bytes) {
    if (!k || !bytes) return sk_fail(SK_EINVAL, "sk_kernel_cap_weight_bytes: NULL argument");
    *bytes = k->d_capw ? (int64_t)k->capw_len * 16 : 0;
    return SK_OK;
}

extern "C" int sk_count_pairs(sk_ctx *ctx, const sk_kern *k, int64_t *out) {
    if (!ctx || !k || !out) return sk_fail(SK_EINVAL, "sk_count_pairs: NULL argument");
    SK_CU(cudaSetDevice(ctx->device));
    unsigned long long *d_total = nullptr;
    SK_CU(cudaMalloc(&d_total, sizeof(unsigned long long)));
    cudaError_t e = cudaMemset(d_total, 0, sizeof(unsigned long long));
    if (e == cudaSuccess)
        e = sk_launch_count_pairs(k->g->nr, (int)(4 * k->g->nside), k->g->d_rings, k->d_pair_off, k->d_pairs,
                                  k->d_dphimax, nullptr, d_total, 0);
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d_total, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d_total);
    if (e != cudaSuccess) return sk_fail(SK_ECUDA, "sk_count_pairs: %s", cudaGetErrorString(e));
    *out = (int64_t)h;
    return SK_OK;
}

extern "C" int sk_count_pairs_by_ring(sk_ctx *ctx, const sk_kern *k, int64_t *out, uint8_t *path) {
    if (!ctx || !k || !out) return sk_fail(SK_EINVAL, "sk_count_pairs_by_ring: NULL argument");
    const int nr = k->g->nr;
    if (path) {
        if (!k->plan_ok) return sk_fail(SK_EUNSUPPORTED, "sk_count_pairs_by_ring: no plan");
        for (int r = 0; r < nr; ++r) path[r] = k->h_ring_path[r];
    }
    SK_CU(cudaSetDevice(ctx->device));
    unsigned long long *d_c = nullptr;
    SK_CU(cudaMalloc(&d_c, sizeof(unsigned long long) * nr));
    cudaError_t e = cudaMemset(d_c, 0, sizeof(unsigned long long) * nr);
    if (e == cudaSuccess)
        e = sk_launch_count_pairs(nr, (int)(4 * k->g->nside), k->g->d_rings, k->d_pair_off, k->d_pairs, k->d_dphimax,
                                  nullptr, d_c, 0, true);
    std::vector<unsigned long long> h(nr);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), d_c, sizeof(unsigned long long) * nr, cudaMemcpyDeviceToHost);
    cudaFree(d_c);
    if (e != cudaSuccess) return sk_fail(SK_ECUDA, "sk_count_pairs_by_ring: %s", cudaGetErrorString(e));
    for (int r = 0; r < nr; ++r) out[r] = (int64_t)h[r];
    return SK_OK;
}

extern "C" int sk_count_pairs_by_launch(sk_ctx *ctx, const sk_kern *k, int64_t *out4) {
    if (!ctx || !k || !out4) return sk_fail(SK_EINVAL, "sk_count_pairs_by_launch: NULL argument");
    if (!k->plan_ok) return sk_fail(SK_EUNSUPPORTED, "operator has no plan");
    SK_CU(cudaSetDevice(ctx->device));
    unsigned long long *d_total = nullptr;
    SK_CU(cudaMalloc(&d_total, 4 * sizeof(unsigned long long)));
    cudaError_t e = cudaMemset(d_total, 0, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess)
        e = sk_launch_count_pairs(k->g->nr, (int)(4 * k->g->nside), k->g->d_rings, k->d_pair_off, k->d_pairs,
                                  k->d_dphimax, k->d_ring_path, d_total, 0);
    unsigned long long h[4] = {0, 0, 0, 0};        // by ring class: belt, narrow caps, general, wide caps
    if (e == cudaSuccess) e = cudaMemcpy(h, d_total, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d_total);
    if (e != cudaSuccess) return sk_fail(SK_ECUDA, "sk_count_pairs_by_launch: %s", cudaGetErrorString(e));
    out4[0] = (int64_t)h[0];
    out4[1] = (int64_t)h[1];
    out4[2] = (int64_t)h[3];
    out4[3] = (int64_t)h[2];
    return SK_OK;
}

extern "C" int sk_count_pairs_by_path(sk_ctx *ctx, const sk_kern *k, int64_t *out3) {
    if (!out3) return sk_fail(SK_EINVAL, "sk_count_pairs_by_path: NULL argument");
    int64_t c[4];
    int rc = sk_count_pairs_by_launch(ctx, k, c);
    if (rc) return rc;
    out3[0] = c[0];
    out3[1] = c[1] + c[2];
    out3[2] = c[3];
    return SK_OK;
}

extern "C" int sk_kernel_set_tiles(sk_kern *k, int belt_p, int cap_t) {
    if (!k) return sk_fail(SK_EINVAL, "sk_kernel_set_tiles: NULL operator");
    if (belt_p != 0 && (belt_p < 5 || belt_p > 17 || belt_p % 2 == 0))
        return sk_fail(SK_EINVAL, "belt_p %d not an odd value in [5, 17]", belt_p);
    if (cap_t != 0 && cap_t != 128) return sk_fail(SK_EINVAL, "cap_t %d unsupported (128)", cap_t);
    if (belt_p != 0 && belt_p != k->belt_P) {
        SK_CU(cudaSetDevice(k->ctx->device));
        SK_CU(cudaDeviceSynchronize());
        k->belt_P = belt_p;
        int rc = sk_plan_rebuild_belt_items(k);
        if (rc) return rc;
    }
    return SK_OK;
}

extern "C" int sk_kernel_get_tiles(const sk_kern *k, int *belt_p, int *cap_t) {
    if (!k) return sk_fail(SK_EINVAL, "sk_kernel_get_tiles: NULL operator");
    if (belt_p) *belt_p = k->belt_P;
    if (cap_t) *cap_t = 128;
    return SK_OK;
}

// ---------------------------------------------------------------------------
// convolution
// ---------------------------------------------------------------------------

int sk_check_maps(const char *who, const sk_kern *k, const void *in, const void *out, int64_t batch,
                  int64_t stride, bool disjoint) {
    if (!k) return sk_fail(SK_EINVAL, "%s: NULL operator", who);
    if (batch < 0) return sk_fail(SK_EINVAL, "%s: batch %lld < 0", who, (long long)batch);
    if (batch == 0) return SK_OK;
    if (batch > (1LL << 20)) return sk_fail(SK_EINVAL, "%s: batch %lld too large", who, (long long)batch);
    if (!in || !out) return sk_fail(SK_EINVAL, "%s: NULL map pointer", who);
    if (stride < k->g->npix)
        return sk_fail(SK_EINVAL, "%s: map_stride %lld < npix %lld", who, (long long)stride, (long long)k->g->npix);
    if (stride % 4) return sk_fail(SK_EINVAL, "%s: map_stride %lld not a multiple of 4", who, (long long)stride);
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15))
        return sk_fail(SK_EINVAL, "%s: map pointers must be 16-byte aligned", who);
    const char *a0 = (const char *)in, *a1 = a0 + (size_t)batch * stride * 4;
    const char *b0 = (const char *)out, *b1 = b0 + (size_t)batch * stride * 4;
    if (disjoint && a0 < b1 && b0 < a1) return sk_fail(SK_EINVAL, "%s: input and output overlap", who);
    return SK_OK;
}

extern "C" int sk_convolve_path(sk_ctx *ctx, const sk_kern *k, const float *d_in, float *d_out, int64_t batch,
                                int64_t map_stride, int path, void *stream) {
    if (!ctx) return sk_fail(SK_EINVAL, "sk_convolve: NULL context");
    int rc = sk_check_maps("sk_convolve", k, d_in, d_out, batch, map_stride);
    if (rc) return rc;
    if (path != SK_PATH_AUTO && path != SK_PATH_GENERAL && path != SK_PATH_TENSOR && path != SK_PATH_FP32 &&
        path != SK_PATH_BF16X3)
        return sk_fail(SK_EINVAL, "unknown path %d", path);
    if (batch == 0) return SK_OK;
    SK_CU(cudaSetDevice(ctx->device));
    SkJob jb{k, d_in, d_out, batch, map_stride};
    void *ws = nullptr;
    size_t need = path != SK_PATH_GENERAL ? sk_jobs_workspace_bytes(&jb, 1, path) : 0;
    if (need && (rc = sk_ctx_workspace(ctx, need, &ws))) return rc;
    return sk_run_jobs(ctx, &jb, 1, path, ws, (cudaStream_t)stream);
}

static int convolve_ring_subset(const char *who, sk_ctx *ctx, const sk_kern *k, const float *d_in, float *d_out,
                                int64_t batch, int64_t map_stride, int ring_lo, int ring_hi, bool sym, void *stream) {
    if (!ctx) return sk_fail(SK_EINVAL, "%s: NULL context", who);
    int rc = sk_check_maps(who, k, d_in, d_out, batch, map_stride);
    if (rc) return rc;
    if (ring_lo < 0 || ring_hi > k->g->nr || ring_lo > ring_hi)
        return sk_fail(SK_EINVAL, "%s: ring range [%d, %d) outside [0, %d)", who, ring_lo, ring_hi, k->g->nr);
    if (batch == 0 || ring_lo == ring_hi) return SK_OK;
    SK_CU(cudaSetDevice(ctx->device));
    const SkItems *sub = nullptr;
    if ((rc = sk_plan_ring_subset(const_cast<sk_kern *>(k), ring_lo, ring_hi, sym, &sub))) return rc;
    SkJob jb{k, d_in, d_out, batch, map_stride};
    jb.sub = sub;
    void *ws = nullptr;
    if ((rc = sk_ctx_workspace(ctx, sk_jobs_workspace_bytes(&jb, 1), &ws))) return rc;
    return sk_run_jobs(ctx, &jb, 1, SK_PATH_AUTO, ws, (cudaStream_t)stream);
}

extern "C" int sk_convolve_rings(sk_ctx *ctx, const sk_kern *k, const float *d_in, float *d_out, int64_t batch,
                                 int64_t map_stride, int ring_lo, int ring_hi, void *stream) {
    return convolve_ring_subset("sk_convolve_rings", ctx, k, d_in, d_out, batch, map_stride, ring_lo, ring_hi,
                                false, stream);
}

extern "C" int sk_convolve_rings_sym(sk_ctx *ctx, const sk_kern *k, const float *d_in, float *d_out, int64_t batch,
                                     int64_t map_stride, int ring_lo, int ring_hi, void *stream) {
    return convolve_ring_subset("sk_convolve_rings_sym", ctx, k, d_in, d_out, batch, map_stride, ring_lo, ring_hi,
                                true, stream);
}

extern "C" int sk_convolve(sk_ctx *ctx, const sk_kern *k, const float *d_in, float *d_out, int64_t batch,
                           int64_t map_stride, void *stream) {
    return sk_convolve_path(ctx, k, d_in, d_out, batch, map_stride, SK_PATH_AUTO, stream);
}

extern "C" int sk_convolve_adjoint(sk_ctx *ctx, const sk_kern *k, const float *d_gy, float *d_gx, int64_t batch,
                                   int64_t map_stride, void *stream) {
    // A_oi = dOmega K_lin(gamma(o,i)) and gamma(o,i) = gamma(i,o): A^T = A, and
    // gathering A^T ybar over the inputs of each output is the forward gather.
    return sk_convolve_path(ctx, k, d_gy, d_gx, batch, map_stride, SK_PATH_AUTO, stream);
}

extern "C" int sk_grad_table(sk_ctx *ctx, const sk_kern *k, const float *d_x, const float *d_gy, int64_t batch,
                             int64_t map_stride, float *d_gtable, void *stream) {
    if (!ctx || !k || !d_gtable) return sk_fail(SK_EINVAL, "sk_grad_table: NULL argument");
    int rc = sk_check_maps("sk_grad_table", k, d_x, d_gy, batch, map_stride, false);
    if (rc) return rc;
    SK_CU(cudaSetDevice(ctx->device));
    void *ws = nullptr;
    if ((rc = sk_ctx_workspace(ctx, sk_grad_workspace_bytes(k, batch, ctx->num_sms), &ws))) return rc;
    return sk_run_grad(ctx, k, d_x, d_gy, batch, map_stride, d_gtable, (double *)ws, (cudaStream_t)stream);
}

// Host buffers: the map goes up in ring bands ordered by distance from the poles
// (northern and southern rings of a band together), the sums of a band start once
// every band its windows reach has arrived, and its outputs go back while later
// bands are still copied or summed: host-to-device copies, sums and device-to-host
// copies overlap on three streams.  Page-locked host memory is needed for the
// copies to be asynchronous (pageable memory still gives the right result).
static int host_streams(sk_ctx *ctx) {
    if (ctx->h2d) return SK_OK;
    SK_CU(cudaStreamCreateWithFlags(&ctx->h2d, cudaStreamNonBlocking));
    SK_CU(cudaStreamCreateWithFlags(&ctx->d2h, cudaStreamNonBlocking));
    for (int b = 0; b < SK_HOST_BANDS; ++b) {
        SK_CU(cudaEventCreateWithFlags(&ctx->ev_in[b], cudaEventDisableTiming));
        SK_CU(cudaEventCreateWithFlags(&ctx->ev_out[b], cudaEventDisableTiming));
    }
    SK_CU(cudaEventCreateWithFlags(&ctx->ev_done, cudaEventDisableTiming));
    return SK_OK;
}

extern "C" int sk_convolve_host(sk_ctx *ctx, const sk_kern *k, const float *h_in, float *h_out, int64_t batch,
                                int64_t map_stride, void *stream) {
    if (!ctx || !k) return sk_fail(SK_EINVAL, "sk_convolve_host: NULL argument");
    if (batch < 0) return sk_fail(SK_EINVAL, "sk_convolve_host: batch < 0");
    if (batch == 0) return SK_OK;
    if (!h_in || !h_out) return sk_fail(SK_EINVAL, "sk_convolve_host: NULL map pointer");
    if (map_stride < k->g->npix || map_stride % 4) return sk_fail(SK_EINVAL, "sk_convolve_host: bad map_stride");
    SK_CU(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)batch * map_stride * sizeof(float);
    const size_t half = (bytes + 255) & ~(size_t)255;
    SkJob jb{k, nullptr, nullptr, batch, map_stride};
    // the band runs below convolve one map at a time: their workspace is that of one map
    SkJob one = jb;
    one.batch = 1;
    void *ws = nullptr;
    int rc = sk_ctx_workspace(ctx, 2 * half + sk_jobs_workspace_bytes(&one, 1, SK_PATH_FP32), &ws);
    if (rc) return rc;
    float *d_in = (float *)ws, *d_out = (float *)((char *)ws + half);
    void *wsj = (char *)ws + 2 * half;
    if (k->bands.empty()) {                      // no plan (general path only): one block of work
        jb.x = d_in;
        jb.y = d_out;
        SK_CU(cudaMemcpyAsync(d_in, h_in, bytes, cudaMemcpyHostToDevice, st));
        if ((rc = sk_run_jobs(ctx, &jb, 1, SK_PATH_FP32, wsj, st))) return rc;
        SK_CU(cudaMemcpyAsync(h_out, d_out, bytes, cudaMemcpyDeviceToHost, st));
        SK_CU(cudaStreamSynchronize(st));
        return SK_OK;
    }
    if ((rc = host_streams(ctx))) return rc;
    const auto &R = k->g->h_rings;
    const long long npix = k->g->npix;
    auto pix = [&](int r) { return r >= k->g->nr ? npix : R[r].start; };
    // the copies wait for whatever the caller queued on its stream before this call
    SK_CU(cudaEventRecord(ctx->ev_done, st));
    SK_CU(cudaStreamWaitEvent(ctx->h2d, ctx->ev_done, 0));
    for (long long m = 0; m < batch; ++m) {
        const long long mo = m * map_stride;
        for (size_t b = 0; b < k->bands.size(); ++b) {
            const sk_kern::Band &B = k->bands[b];
            const long long n0 = pix(B.n_lo), n1 = pix(B.n_hi), s0 = pix(B.s_lo), s1 = pix(B.s_hi);
            if (n1 > n0)
                SK_CU(cudaMemcpyAsync(d_in + mo + n0, h_in + mo + n0, sizeof(float) * (n1 - n0),
                                      cudaMemcpyHostToDevice, ctx->h2d));
            if (s1 > s0)
                SK_CU(cudaMemcpyAsync(d_in + mo + s0, h_in + mo + s0, sizeof(float) * (s1 - s0),
                                      cudaMemcpyHostToDevice, ctx->h2d));
            SK_CU(cudaEventRecord(ctx->ev_in[b], ctx->h2d));
        }
        for (size_t b = 0; b < k->bands.size(); ++b) {
            const sk_kern::Band &B = k->bands[b];
            SK_CU(cudaStreamWaitEvent(st, ctx->ev_in[B.need], 0));
            SkJob j{k, d_in + mo, d_out + mo, 1, map_stride};
            j.sub = &B.items;
            j.weights = (m == 0 && b == 0);      // the belt weight rows stay in the workspace
            // the FP32 belt: a band's few ring groups underfill the tensor-core form's one-CTA-
            // per-SM launch, and the sums hide behind the copies either way
            if ((rc = sk_run_jobs(ctx, &j, 1, SK_PATH_FP32, wsj, st))) return rc;
            SK_CU(cudaEventRecord(ctx->ev_out[b], st));
            SK_CU(cudaStreamWaitEvent(ctx->d2h, ctx->ev_out[b], 0));
            // every band whose outputs are complete once this band's sums are done
            for (size_t o = 0; o < k->bands.size(); ++o) {
                const sk_kern::Band &O = k->bands[o];
                if (O.ready != (int)b) continue;
                const long long n0 = pix(O.n_lo), n1 = pix(O.n_hi), s0 = pix(O.s_lo), s1 = pix(O.s_hi);
                if (n1 > n0)
                    SK_CU(cudaMemcpyAsync(h_out + mo + n0, d_out + mo + n0, sizeof(float) * (n1 - n0),
                                          cudaMemcpyDeviceToHost, ctx->d2h));
                if (s1 > s0)
                    SK_CU(cudaMemcpyAsync(h_out + mo + s0, d_out + mo + s0, sizeof(float) * (s1 - s0),
                                          cudaMemcpyDeviceToHost, ctx->d2h));
            }
        }
    }
    SK_CU(cudaEventRecord(ctx->ev_done, ctx->d2h));
    SK_CU(cudaStreamWaitEvent(st, ctx->ev_done, 0));
    SK_CU(cudaStreamSynchronize(st));
    return SK_OK;
}

// ---------------------------------------------------------------------------
// jobs and graphs
// ---------------------------------------------------------------------------

static int convert_jobs(const sk_job *jobs, int n, std::vector<SkJob> &out) {
    if (n < 0 || (n > 0 && !jobs)) return sk_fail(SK_EINVAL, "bad job list");
    out.resize(n);
    for (int i = 0; i < n; ++i) {
        int rc = sk_check_maps("sk_convolve_jobs", jobs[i].k, jobs[i].d_in, jobs[i].d_out, jobs[i].batch,
                            jobs[i].map_stride);
        if (rc) return rc;
        out[i] = SkJob{jobs[i].k, jobs[i].d_in, jobs[i].d_out, jobs[i].batch, jobs[i].map_stride};
    }
    return SK_OK;
}

extern "C" int sk_convolve_jobs(sk_ctx *ctx, const sk_job *jobs, int n_jobs, int flags, void *stream) {
    if (!ctx) return sk_fail(SK_EINVAL, "sk_convolve_jobs: NULL context");
    if (flags != SK_PATH_AUTO && flags != SK_PATH_GENERAL && flags != SK_PATH_TENSOR && flags != SK_PATH_FP32 &&
        flags != SK_PATH_BF16X3)
        return sk_fail(SK_EINVAL, "unknown flags %d", flags);
    std::vector<SkJob> js;
    int rc = convert_jobs(jobs, n_jobs, js);
    if (rc) return rc;
    SK_CU(cudaSetDevice(ctx->device));
    void *ws = nullptr;
    size_t need = flags != SK_PATH_GENERAL ? sk_jobs_workspace_bytes(js.data(), n_jobs, flags) : 0;
    if (need && (rc = sk_ctx_workspace(ctx, need, &ws))) return rc;
    return sk_run_jobs(ctx, js.data(), n_jobs, flags, ws, (cudaStream_t)stream);
}

struct sk_graph {
    cudaGraphExec_t exec = nullptr;
    void *ws = nullptr;        // belt weight rows the graph writes and reads
    int device = 0;
};

extern "C" int sk_graph_capture(sk_ctx *ctx, const sk_job *jobs, int n_jobs, int flags, void *stream,
                                void **graph_exec) {
    if (!ctx || !graph_exec) return sk_fail(SK_EINVAL, "sk_graph_capture: NULL argument");
    *graph_exec = nullptr;
    if (flags != SK_PATH_AUTO && flags != SK_PATH_GENERAL && flags != SK_PATH_TENSOR && flags != SK_PATH_FP32 &&
        flags != SK_PATH_BF16X3)
        return sk_fail(SK_EINVAL, "unknown flags %d", flags);
    if (!stream) return sk_fail(SK_EINVAL, "sk_graph_capture: capture needs a non-default stream");
    std::vector<SkJob> js;
    int rc = convert_jobs(jobs, n_jobs, js);
    if (rc) return rc;
    SK_CU(cudaSetDevice(ctx->device));
    sk_graph *g = new sk_graph();
    g->device = ctx->device;
    size_t need = flags != SK_PATH_GENERAL ? sk_jobs_workspace_bytes(js.data(), n_jobs, flags) : 0;
    if (need) {
        cudaError_t e = cudaMalloc(&g->ws, need);
        if (e != cudaSuccess) { delete g; return sk_fail(SK_ENOMEM, "graph workspace: %s", cudaGetErrorString(e)); }
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaFree(g->ws); delete g; return sk_fail(SK_ECUDA, "begin capture: %s", cudaGetErrorString(e)); }
    rc = sk_run_jobs(ctx, js.data(), n_jobs, flags, g->ws, st);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(st, &graph);
    if (rc == SK_OK && e != cudaSuccess) rc = sk_fail(SK_ECUDA, "end capture: %s", cudaGetErrorString(e));
    if (rc == SK_OK) {
        e = cudaGraphInstantiate(&g->exec, graph, 0);
        if (e != cudaSuccess) rc = sk_fail(SK_ECUDA, "instantiate: %s", cudaGetErrorString(e));
    }
    if (graph) cudaGraphDestroy(graph);
    if (rc) { cudaFree(g->ws); delete g; return rc; }
    *graph_exec = g;
    return SK_OK;
}

extern "C" int sk_graph_launch(void *graph_exec, void *stream) {
    sk_graph *g = (sk_graph *)graph_exec;
    if (!g || !g->exec) return sk_fail(SK_EINVAL, "sk_graph_launch: NULL graph");
    SK_CU(cudaSetDevice(g->device));
    SK_CU(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return SK_OK;
}

extern "C" int sk_graph_destroy(void *graph_exec) {
    sk_graph *g = (sk_graph *)graph_exec;
    if (!g) return SK_OK;
    cudaSetDevice(g->device);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    cudaFree(g->ws);
    delete g;
    return SK_OK;
}
