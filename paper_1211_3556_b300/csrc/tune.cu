// tune.cu -- autotuner of an operator's launch settings and the bounded-wait
// self-test.
//
// Settings: the belt form (the FP32 kernel, whose tile width P -- outputs per
// thread along a ring -- trades the per-chunk strip reloads, P + 3 values per 4P
// FFMAs, against the tail of the last segment of each ring, 4 Nside pixels in
// segments of 32 P; or the 3xTF32 tensor-core kernel, whose extra work is the
// padding of its weight tiles and the split of the maps' rows in each stage) and whether
// the caps stream stored weights or evaluate them.  The planner starts from a
// cost model; sk_kernel_autotune times the candidates on the caller's maps and
// keeps the fastest, optionally remembering the choice in a small text cache
// keyed by GPU name, Nside, cut, node count, layout and batch.
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

struct Choice {
    int P = 0, form = SK_BELT_FP32, capw = 1;
};

// The last line of the cache with this key: "key P [form [capw]]".
bool cache_lookup(const char *path, const std::string &key, Choice *out) {
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[768];
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        char key_in[640];
        Choice c;
        const int n = sscanf(line, "%639s %d %d %d", key_in, &c.P, &c.form, &c.capw);
        if (n >= 2 && key == key_in) {
            if (n < 3) c.form = SK_BELT_FP32;
            if (n < 4) c.capw = 1;
            *out = c;
            found = true;
        }
    }
    fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, const Choice &c) {
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d\n", key.c_str(), c.P, c.form, c.capw);
    fclose(f);
}

// Apply a choice (a tensor form the operator cannot take falls back to FP32).
int apply(sk_kern *k, const Choice &c) {
    int rc = sk_kernel_set_tiles(k, c.P, 0);
    if (rc) return rc;
    if (c.form == SK_BELT_TENSOR && k->tcp[0].ok) {
        if (sk_kernel_set_belt_form(k, SK_BELT_TENSOR) != SK_OK) k->belt_form = SK_BELT_FP32;
    } else {
        k->belt_form = SK_BELT_FP32;
    }
    if (!c.capw && k->d_capw) return sk_kernel_set_cap_weights(k, 0);
    if (c.capw && !k->d_capw && k->capw_len > 0) sk_kernel_set_cap_weights(k, 1);   // if it fits
    return SK_OK;
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
        Choice c;
        if (cache_lookup(cache_path, key, &c) && apply(k, c) == SK_OK) {
            *chosen = k->belt_P;
            return SK_OK;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    SK_CU(cudaEventCreate(&e0));
    SK_CU(cudaEventCreate(&e1));
    // one warm-up call (it also builds what a setting evaluates on first use), then
    // three timed calls of the whole operator
    auto time_it = [&](float *ms) -> int {
        int rc = sk_convolve(ctx, k, d_in, d_out, batch, map_stride, stream);
        if (rc) return rc;
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && rc == SK_OK; ++r) rc = sk_convolve(ctx, k, d_in, d_out, batch, map_stride, stream);
        cudaEventRecord(e1, st);
        if (rc) return rc;
        if (cudaEventSynchronize(e1) != cudaSuccess) return sk_fail(SK_ECUDA, "autotune: event");
        cudaEventElapsedTime(ms, e0, e1);
        return SK_OK;
    };
    const int Ps[] = {5, 7, 9, 11, 13, 15, 17};
    Choice best;
    best.P = k->belt_P;
    best.capw = k->d_capw ? 1 : 0;
    float best_ms = 1e30f, ms = 0.0f;
    int rc = SK_OK;
    k->belt_form = SK_BELT_FP32;
    for (int P : Ps) {
        if ((rc = sk_kernel_set_tiles(k, P, 0)) || (rc = time_it(&ms))) break;
        if (ms < best_ms) { best_ms = ms; best.P = P; }
    }
    if (rc == SK_OK) rc = sk_kernel_set_tiles(k, best.P, 0);
    // (the BF16x3 form is outside the accuracy bound and never a candidate)
    if (rc == SK_OK && k->tcp[0].ok && sk_kernel_set_belt_form(k, SK_BELT_TENSOR) == SK_OK) {
        if ((rc = time_it(&ms)) == SK_OK && ms < best_ms) {
            best_ms = ms;
            best.form = SK_BELT_TENSOR;
        }
        k->belt_form = best.form;
    }
    // (operators with wide windows keep their stored weights: those are evaluated in FP64
    // and summed ring by ring, the evaluating kernel is neither)
    if (rc == SK_OK && k->d_capw && !k->blocked) {
        if ((rc = sk_kernel_set_cap_weights(k, 0)) == SK_OK && (rc = time_it(&ms)) == SK_OK && ms < best_ms) {
            best_ms = ms;
            best.capw = 0;
        }
        if (rc == SK_OK && best.capw) rc = sk_kernel_set_cap_weights(k, 1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if ((rc = apply(k, best))) return rc;
    if (cache_path) cache_store(cache_path, key, best);
    *chosen = best.P;
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
