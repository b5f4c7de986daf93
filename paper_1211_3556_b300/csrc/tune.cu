// tune.cu -- autotuner of the belt tile width and the bounded-wait self-test.
//
// The belt kernel's tile width P (outputs per thread along a ring) trades the
// per-chunk strip reloads (P + 3 values per 4P FFMAs) against the tail of the
// last segment of each ring (rings have 4 Nside pixels, a segment 32 P).  The
// planner starts from a cost model; sk_kernel_autotune times every candidate on
// the caller's maps and keeps the fastest, optionally remembering the choice in
// a small text cache keyed by GPU name, Nside, cut, node count and batch.
#include <stdio.h>
#include <string.h>

#include <string>

#include "skconv_host.h"

namespace {

std::string cache_key(const sk_ctx *ctx, const sk_kern *k, long long batch) {
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, ctx->device);
    char buf[512];
    snprintf(buf, sizeof buf, "%s|nside=%lld|tc=%.9e|nt=%d|layout=%d|batch=%lld", p.name, k->g->nside, k->tc,
             k->nt, k->layout, batch);
    for (char *c = buf; *c; ++c)
        if (*c == ' ') *c = '_';
    return buf;
}

int cache_lookup(const char *path, const std::string &key) {
    FILE *f = fopen(path, "r");
    if (!f) return 0;
    char line[768];
    int found = 0;
    while (fgets(line, sizeof line, f)) {
        char key_in[640];
        int p = 0;
        if (sscanf(line, "%639s %d", key_in, &p) == 2 && key == key_in) found = p;
    }
    fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, int p) {
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d\n", key.c_str(), p);
    fclose(f);
}

// Bounded wait on an mbarrier phase that nothing completes: returns after
// `limit_ns` of %globaltimer and records SK_ETIMEOUT.  Used only by the self-test.
__global__ void k_wait_timeout(int *status, unsigned long long limit_ns) {
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(1));
    __syncthreads();
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok) : "r"(a), "r"(0) : "memory");
        if (ok) return;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) {
            if (threadIdx.x == 0) atomicCAS(status, 0, SK_ETIMEOUT);
            return;
        }
    }
}

}  // namespace

extern "C" int sk_kernel_autotune(sk_ctx *ctx, sk_kern *k, const float *d_in, float *d_out, int64_t batch,
                                  int64_t map_stride, const char *cache_path, void *stream, int *chosen) {
    if (!ctx || !k || !chosen) return sk_fail(SK_EINVAL, "sk_kernel_autotune: NULL argument");
    *chosen = k->belt_P;
    if (!k->plan_ok || k->nb == 0) return SK_OK;              // no belt: nothing to tune
    SK_CU(cudaSetDevice(ctx->device));
    const std::string key = cache_key(ctx, k, batch);
    if (cache_path) {
        int p = cache_lookup(cache_path, key);
        if (p) {
            int rc = sk_kernel_set_tiles(k, p, 0);
            if (rc == SK_OK) { *chosen = p; return SK_OK; }
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    SK_CU(cudaEventCreate(&e0));
    SK_CU(cudaEventCreate(&e1));
    const int Ps[] = {5, 7, 9, 11, 13, 15, 17};
    int best = k->belt_P;
    float best_ms = 1e30f;
    int rc = SK_OK;
    for (int P : Ps) {
        if ((rc = sk_kernel_set_tiles(k, P, 0))) break;
        if ((rc = sk_convolve(ctx, k, d_in, d_out, batch, map_stride, stream))) break;   // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && rc == SK_OK; ++r) rc = sk_convolve(ctx, k, d_in, d_out, batch, map_stride, stream);
        cudaEventRecord(e1, st);
        if (rc) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = sk_fail(SK_ECUDA, "autotune: event"); break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best = P; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if ((rc = sk_kernel_set_tiles(k, best, 0))) return rc;
    if (cache_path) cache_store(cache_path, key, best);
    *chosen = best;
    return SK_OK;
}

extern "C" int sk_selftest_wait_timeout(sk_ctx *ctx, double seconds, void *stream) {
    if (!ctx) return sk_fail(SK_EINVAL, "sk_selftest_wait_timeout: NULL context");
    if (!(seconds > 0.0) || seconds > 2.0) return sk_fail(SK_EINVAL, "sk_selftest_wait_timeout: limit in (0, 2] s");
    SK_CU(cudaSetDevice(ctx->device));
    k_wait_timeout<<<1, 32, 0, (cudaStream_t)stream>>>(ctx->d_status, (unsigned long long)(seconds * 1e9));
    SK_CU(cudaGetLastError());
    return SK_OK;
}
