// noalloc.cu -- the table gradient for callers that cannot allocate device memory.
//
// sk_grad_table accumulates its bins in FP64 in the context's workspace, which
// the library grows with cudaMalloc on demand.  Some callers cannot let a
// library allocate: hosts whose device memory is owned by their own allocator
// or budget, and latency-critical loops where a cudaMalloc or cudaFree would
// synchronise the device.  sk_grad_table_noalloc computes the same gradient
// with the FP64 accumulator in a fixed array compiled into this library instead.
// It uses only the per-pixel gradient kernel (one FP64 node coordinate per pair,
// on every output ring): the belt's ring-pair correlations and the caps'
// symmetric base pairs need workspace (their FP32 sums and the symmetric copy of
// the maps), so it is several times slower than sk_grad_table at large sizes.
//
// The array lives for as long as the library is loaded, on every GPU that
// loads it (SK_NOALLOC_MAX_NODES doubles = 128 KiB each).  All calls on a
// device share it: each call clears it before use, and two calls whose work
// overlaps on the GPU (different streams, no ordering) race on it.
#include <string.h>

#include <algorithm>
#include <mutex>

#include "skconv_host.h"

namespace {

constexpr int SK_NOALLOC_MAX_NODES = 16384;
constexpr int SK_NOALLOC_MAX_DEVICES = 64;

// The accumulator.  In host code this name is only a stand-in for the device
// symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_grad_scratch[SK_NOALLOC_MAX_NODES];

std::mutex g_mu;
double *g_scratch_addr[SK_NOALLOC_MAX_DEVICES] = {};

// Device address of the accumulator on `device`, looked up once per device with
// that device current (the first call on a device does this).
int scratch_on(int device, double **out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (device < 0 || device >= SK_NOALLOC_MAX_DEVICES)
        return sk_fail(SK_EUNSUPPORTED, "sk_grad_table_noalloc: device %d out of range", device);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_grad_scratch);
        if (e != cudaSuccess)
            return sk_fail(SK_ECUDA, "sk_grad_table_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_addr[device] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[device];
    return SK_OK;
}

}  // namespace

extern "C" int sk_grad_table_noalloc(sk_ctx *ctx, const sk_kern *k, const float *d_x, const float *d_gy,
                                     int64_t batch, int64_t map_stride, float *d_gtable, void *stream) {
    if (!ctx || !k || !d_gtable) return sk_fail(SK_EINVAL, "sk_grad_table_noalloc: NULL argument");
    if (k->nt > SK_NOALLOC_MAX_NODES)
        return sk_fail(SK_EINVAL, "sk_grad_table_noalloc: %d table nodes exceed the fixed accumulator of %d",
                       k->nt, SK_NOALLOC_MAX_NODES);
    if (batch < 0 || batch > (1LL << 20)) return sk_fail(SK_EINVAL, "sk_grad_table_noalloc: bad batch %lld", (long long)batch);
    if (batch > 0) {
        if (!d_x || !d_gy) return sk_fail(SK_EINVAL, "sk_grad_table_noalloc: NULL map pointer");
        if (map_stride < k->g->npix || map_stride % 4)
            return sk_fail(SK_EINVAL, "sk_grad_table_noalloc: bad map_stride %lld", (long long)map_stride);
        if (((uintptr_t)d_x & 15) || ((uintptr_t)d_gy & 15))
            return sk_fail(SK_EINVAL, "sk_grad_table_noalloc: map pointers must be 16-byte aligned");
    }
    SK_CU(cudaSetDevice(ctx->device));
    double *acc = nullptr;
    int rc = scratch_on(ctx->device, &acc);
    if (rc) return rc;
    // Clear the shared accumulator on the stream, run the gradient kernel over every
    // output ring and the FP64 -> FP32 finish kernel.  Nothing here allocates.
    cudaStream_t st = (cudaStream_t)stream;
    SK_CU(cudaMemsetAsync(acc, 0, sizeof(double) * k->nt, st));
    if (batch > 0) {
        JobsArg a;
        memset(&a, 0, sizeof a);
        JobDesc &d = a.j[0];
        d.rings = k->g->d_rings;
        d.pair_off = k->d_pair_off;
        d.pairs = k->d_pairs;
        d.tab = k->d_tab;
        d.kp = k->kp;
        d.kd = k->kd;
        d.ab64 = k->d_ab64;
        d.nr = k->g->nr;
        d.x = d_x;
        d.stride = map_stride;
        d.batch = (int)batch;
        d.items = k->d_items_all;
        d.n_items = k->n_items_all;
        d.flat_base = 0;
        a.n_jobs = 1;
        a.total = k->n_items_all * (int)batch;
        a.status = ctx->d_status;
        const int grid = std::max(1, std::min(a.total, 8 * ctx->num_sms));
        SK_CU(sk_launch_grad_general(a, d_gy, acc, grid, st));
    }
    SK_CU(sk_launch_grad_finish(acc, k->nt, 4.0 * SK_PI / (double)k->g->npix, d_gtable, st));
    return SK_OK;
}
