// peaks.cu -- measured arithmetic peaks of the device, the denominators of the
// roofline fractions the benchmark reports for the FP32 sums and the TF32
// tensor-core form.
//
//  * FP32: persistent blocks run independent FMA chains (scalar fma.rn.f32, or
//    the paired fma.rn.f32x2) in registers, 16 chains per thread so that the
//    FMA latency is covered by one warp's own work; 2 flop per FMA.
//  * TF32: one block per SM issues tcgen05.mma.kind::tf32 of 128 x 256 x 8
//    (the largest single-CTA shape) back to back from shared-memory operands
//    into a 256-column tensor-memory accumulator; 2 x 128 x 256 x 8 flop per
//    MMA.  A chunk of MMAs is committed to an mbarrier and the issuing thread
//    waits (bounded) for the chunk before the previous one, so that at least
//    one chunk is always queued on the tensor pipe.
// Every launch runs a fixed amount of work; the host repeats launches until the
// requested time has passed and divides the flops by the CUDA-event time.
#include <algorithm>

#include "skconv_host.h"
#include "tc.cuh"

namespace {

constexpr int FMA_CHAINS = 16;       // independent accumulators per thread
constexpr int FMA_UNROLL = 8;        // chain steps per loop trip
constexpr int PEAK_THREADS = 256;
constexpr int TC_N = 256;            // MMA N (columns of the accumulator)
constexpr int TC_CHUNK = 64;         // MMAs per commit
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;

__global__ void __launch_bounds__(PEAK_THREADS)
k_peak_ffma(int iters, float *out) {
    float a[FMA_CHAINS];
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) a[c] = 1e-3f * (float)(threadIdx.x + c);
    const float m = 0.9999999f, s = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < FMA_UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < FMA_CHAINS; ++c) a[c] = fmaf(a[c], m, s);
    }
    float r = 0.0f;
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) r += a[c];
    if (r == 1234.5f) out[blockIdx.x] = r;      // never true; keeps the chains live
}

__global__ void __launch_bounds__(PEAK_THREADS)
k_peak_ffma2(int iters, float *out) {
    float2 a[FMA_CHAINS / 2];
#pragma unroll
    for (int c = 0; c < FMA_CHAINS / 2; ++c) a[c] = make_float2(1e-3f * (float)(threadIdx.x + c), 2e-3f * (float)c);
    const float2 m = make_float2(0.9999999f, 0.9999998f), s = make_float2(1e-7f, 2e-7f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 2 * FMA_UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < FMA_CHAINS / 2; ++c) a[c] = __ffma2_rn(a[c], m, s);
    }
    float r = 0.0f;
#pragma unroll
    for (int c = 0; c < FMA_CHAINS / 2; ++c) r += a[c].x + a[c].y;
    if (r == 1234.5f) out[blockIdx.x] = r;
}

// One block of 128 threads per SM; thread 0 issues the MMAs.  Shared memory: A
// (128 rows x 32 TF32 columns, one 128-byte swizzled atom, 16 KB) and B (256 rows,
// 32 KB), filled with hashed values in [-1, 1) so that the tensor pipe works on
// ordinary operands.
__global__ void __launch_bounds__(128)
k_peak_tf32(int chunks, int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *a = base;
    unsigned char *b = a + 128 * 128;
    __shared__ __align__(8) uint64_t bars[3];    // two for the chunks, one for the final drain
    __shared__ uint32_t tslot;
    const int t = threadIdx.x, warp = t >> 5;
    if (warp == 0) tc::tmem_alloc(&tslot, TC_N);
    if (t == 0) {
        for (int i = 0; i < 3; ++i) tc::mbar_init(tc::smem_u32(&bars[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = t; i < (128 + TC_N) * 32; i += 128) {
        uint32_t h = (uint32_t)i * 2654435761u + 12345u;
        h ^= h >> 15;
        *reinterpret_cast<float *>(base + 4 * i) = tc::rna_tf32((float)(h & 0xFFFF) / 32768.0f - 1.0f);
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;
    if (t == 0) {
        const uint32_t idesc = tc::idesc_tf32(128, TC_N);
        const uint32_t sa = tc::smem_u32(a), sb = tc::smem_u32(b);
        bool ok = true;
        for (int c = 0; c < chunks && ok; ++c) {
            for (int m = 0; m < TC_CHUNK; ++m) {
                const int kk = m & 3;       // the four K steps of the atom
                tc::mma_tf32(taddr, tc::sw128_desc(sa + kk * 32), tc::sw128_desc(sb + kk * 32), idesc,
                             (c | m) != 0);
            }
            // chunk c completes phase c >> 1 of bars[c & 1]; chunk c - 1 must be done before
            // chunk c + 1 is issued
            tc::mma_commit(tc::smem_u32(&bars[c & 1]));
            if (c >= 1) ok = tc::mbar_wait(tc::smem_u32(&bars[(c - 1) & 1]), ((c - 1) >> 1) & 1, TC_WAIT_NS);
        }
        // drain: the first phase of the third barrier completes once every MMA issued so
        // far is done (also after a timeout, before the block frees the tensor memory)
        tc::mma_commit(tc::smem_u32(&bars[2]));
        const bool drained = tc::mbar_wait(tc::smem_u32(&bars[2]), 0, TC_WAIT_NS);
        if (!ok || !drained) sk_record_error(status, SK_ETIMEOUT);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(taddr, TC_N);
    }
}

}  // namespace

extern "C" int sk_device_info(sk_ctx *ctx, int64_t *out4) {
    if (!ctx || !out4) return sk_fail(SK_EINVAL, "sk_device_info: NULL argument");
    SK_CU(cudaSetDevice(ctx->device));
    int sms = 0, khz = 0, smem = 0, l2 = 0;
    SK_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    SK_CU(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device));
    SK_CU(cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    SK_CU(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device));
    out4[0] = sms;
    out4[1] = khz;
    out4[2] = smem;
    out4[3] = l2;
    return SK_OK;
}

extern "C" int sk_measure_peak(sk_ctx *ctx, int kind, double seconds, double *tflops, void *stream) {
    if (!ctx || !tflops) return sk_fail(SK_EINVAL, "sk_measure_peak: NULL argument");
    if (kind < SK_PEAK_FFMA || kind > SK_PEAK_TF32)
        return sk_fail(SK_EINVAL, "sk_measure_peak: kind %d is not SK_PEAK_FFMA, SK_PEAK_FFMA2 or SK_PEAK_TF32", kind);
    if (!(seconds > 0.0 && seconds <= 60.0)) return sk_fail(SK_EINVAL, "sk_measure_peak: seconds in (0, 60]");
    SK_CU(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = ctx->num_sms;
    float *sink = nullptr;
    SK_CU(cudaMalloc(&sink, sizeof(float) * 8 * sms));
    const size_t tc_smem = 1024 + (size_t)(128 + TC_N) * 128;
    if (kind == SK_PEAK_TF32) {
        cudaError_t e = cudaFuncSetAttribute(k_peak_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem);
        if (e != cudaSuccess) { cudaFree(sink); SK_CU(e); }
    }
    // work per launch: FP32 8 blocks per SM; TF32 one block per SM
    const int fma_iters = 1 << 14, tc_chunks = 1 << 10;
    double flop_launch;
    auto launch = [&]() -> cudaError_t {
        if (kind == SK_PEAK_FFMA) k_peak_ffma<<<8 * sms, PEAK_THREADS, 0, st>>>(fma_iters, sink);
        else if (kind == SK_PEAK_FFMA2) k_peak_ffma2<<<8 * sms, PEAK_THREADS, 0, st>>>(fma_iters, sink);
        else k_peak_tf32<<<sms, 128, tc_smem, st>>>(tc_chunks, ctx->d_status);
        return cudaGetLastError();
    };
    // FMAs per thread and loop trip: FMA_UNROLL x FMA_CHAINS scalar ones, or 2 FMA_UNROLL x
    // FMA_CHAINS / 2 paired instructions of two FMAs each
    if (kind == SK_PEAK_TF32) flop_launch = (double)sms * tc_chunks * TC_CHUNK * 2.0 * 128 * TC_N * 8;
    else flop_launch = 8.0 * sms * PEAK_THREADS * (double)fma_iters * FMA_UNROLL * FMA_CHAINS * 2.0 *
                       (kind == SK_PEAK_FFMA2 ? 2.0 : 1.0);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SK_OK;
    auto fail = [&](cudaError_t e) {
        rc = sk_fail(SK_ECUDA, "sk_measure_peak: %s", cudaGetErrorString(e));
    };
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // one warm-up launch, timed, to size the run
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms1 = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms1, e0, e1);
    if (e != cudaSuccess) {
        fail(e);
    } else {
        const int n = (int)std::max(1.0, std::min(1e5, seconds * 1e3 / std::max(1e-3, (double)ms1)));
        e = cudaEventRecord(e0, st);
        for (int i = 0; i < n && e == cudaSuccess; ++i) e = launch();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) fail(e);
        else *tflops = flop_launch * n / (ms * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
}
