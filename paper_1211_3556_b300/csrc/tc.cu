// tc.cu -- self-test of the tcgen05 building blocks of the tensor-core path.
//
// One block computes D = A B^T for A (128 x K) and B (N x K) given in global
// memory, with the operands split into TF32 hi/lo pieces in shared memory
// (128-byte swizzled K-major atoms) and either one product (hi hi) or the
// three products hi hi + hi lo + lo hi accumulated in tensor memory; D is read
// back with tcgen05.ld.  It checks the descriptor and layout conventions the
// batched belt kernel relies on against a host reference.
//
// A second block checks the no-swizzle K-major form the tensor-core belt uses:
// the weights (A, 128 x K) as 4-column chunks 2048 bytes apart, and a B operand
// that is a vector read in sliding rows, B_q[s][t] = x[8 s + 8 q + t + off]
// (k-step q, t < 8, off 0 or 4), staged as three planes of 16-byte rows
// (x[8m .. 8m+3], x[8m+4 .. 8m+7], x[8m+8 .. 8m+11]) so that every k-step of
// either offset is a start address 16 q bytes into the planes.
#include "skconv_host.h"
#include "tc.cuh"

namespace {

__global__ void __launch_bounds__(128)
k_tc_gemm(const float *__restrict__ a, const float *__restrict__ b, float *__restrict__ d, int N, int K, int passes,
          int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte align the operand region
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int KA = K / 32;
    unsigned char *a_hi = base;
    unsigned char *a_lo = a_hi + KA * 128 * 128;
    unsigned char *b_hi = a_lo + KA * 128 * 128;
    unsigned char *b_lo = b_hi + KA * N * 128;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int t = threadIdx.x, warp = t >> 5;

    if (warp == 0) tc::tmem_alloc(&tslot, 256);
    if (t == 0) {
        tc::mbar_init(tc::smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // operands: element (r, k) of atom k/32
    for (int i = t; i < 128 * K; i += 128) {
        const int r = i / K, k = i % K;
        float hi, lo;
        tc::split_tf32(a[i], hi, lo);
        const uint32_t off = (uint32_t)(k >> 5) * 128 * 128 + tc::sw128_offset(r, k);
        *reinterpret_cast<float *>(a_hi + off) = hi;
        *reinterpret_cast<float *>(a_lo + off) = lo;
    }
    for (int i = t; i < N * K; i += 128) {
        const int r = i / K, k = i % K;
        float hi, lo;
        tc::split_tf32(b[i], hi, lo);
        const uint32_t off = (uint32_t)(k >> 5) * N * 128 + tc::sw128_offset(r, k);
        *reinterpret_cast<float *>(b_hi + off) = hi;
        *reinterpret_cast<float *>(b_lo + off) = lo;
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;

    if (t == 0) {
        const uint32_t idesc = tc::idesc_tf32(128, N);
        int acc = 0;
        for (int s = 0; s < K / 8; ++s) {
            const int ka = s >> 2, kk = s & 3;
            const uint32_t ao = (uint32_t)ka * 128 * 128 + kk * 32, bo = (uint32_t)ka * N * 128 + kk * 32;
            tc::mma_tf32(taddr, tc::sw128_desc(tc::smem_u32(a_hi + ao)), tc::sw128_desc(tc::smem_u32(b_hi + bo)),
                         idesc, acc);
            acc = 1;
            if (passes == 3) {
                tc::mma_tf32(taddr, tc::sw128_desc(tc::smem_u32(a_hi + ao)),
                             tc::sw128_desc(tc::smem_u32(b_lo + bo)), idesc, 1);
                tc::mma_tf32(taddr, tc::sw128_desc(tc::smem_u32(a_lo + ao)),
                             tc::sw128_desc(tc::smem_u32(b_hi + bo)), idesc, 1);
            }
        }
        tc::mma_commit(tc::smem_u32(&bar));
    }
    const bool ok = tc::mbar_wait(tc::smem_u32(&bar), 0, 1000000000ull);
    if (!ok && t == 0) atomicCAS(status, 0, SK_ETIMEOUT);
    tc::fence_after_sync();
    if (ok) {
        const int row = warp * 32 + (t & 31);
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) d[row * N + c0 + j] = v[j];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(taddr, 256);
    }
}

__global__ void __launch_bounds__(128)
k_tc_sliding(const float *__restrict__ a, const float *__restrict__ x, float *__restrict__ d, int N, int K, int off,
             int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int R = N + K / 8;                           // rows of each plane
    const uint32_t slot = (uint32_t)R * 16;
    unsigned char *b_hi = base, *b_lo = base + 3 * slot;
    unsigned char *a_hi = base + ((6 * slot + 1023) & ~1023u);
    unsigned char *a_lo = a_hi + (uint32_t)K * 512;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int t = threadIdx.x, warp = t >> 5;

    if (warp == 0) tc::tmem_alloc(&tslot, 512);
    if (t == 0) {
        tc::mbar_init(tc::smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = t; i < 128 * K; i += 128) {
        const int r = i / K, k = i % K;
        float hi, lo;
        tc::split_tf32(a[i], hi, lo);
        *reinterpret_cast<float *>(a_hi + tc::kmajor128_offset(r, k)) = hi;
        *reinterpret_cast<float *>(a_lo + tc::kmajor128_offset(r, k)) = lo;
    }
    for (int i = t; i < 3 * R * 4; i += 128) {
        const int p = i / (4 * R), m = (i / 4) % R, c = i & 3;
        const int px = 8 * m + 4 * p + c;              // plane 2 is plane 0 one row on
        float hi, lo;
        tc::split_tf32(x[px], hi, lo);
        *reinterpret_cast<float *>(b_hi + p * slot + 16 * m + 4 * c) = hi;
        *reinterpret_cast<float *>(b_lo + p * slot + 16 * m + 4 * c) = lo;
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;

    if (t == 0) {
        const uint32_t idesc = tc::idesc_tf32(128, N);
        const uint32_t b0 = off ? slot : 0u;           // first plane of the k-step's two
        for (int q = 0; q < K / 8; ++q) {
            const uint64_t ah = tc::kmajor_desc(tc::smem_u32(a_hi + 4096 * q), 2048, 128);
            const uint64_t al = tc::kmajor_desc(tc::smem_u32(a_lo + 4096 * q), 2048, 128);
            const uint64_t bh = tc::kmajor_desc(tc::smem_u32(b_hi + b0 + 16 * q), slot, 128);
            const uint64_t bl = tc::kmajor_desc(tc::smem_u32(b_lo + b0 + 16 * q), slot, 128);
            tc::mma_tf32(taddr, ah, bh, idesc, q > 0);
            tc::mma_tf32(taddr + 256u, ah, bl, idesc, q > 0);
            tc::mma_tf32(taddr + 256u, al, bh, idesc, 1);
        }
        tc::mma_commit(tc::smem_u32(&bar));
    }
    const bool ok = tc::mbar_wait(tc::smem_u32(&bar), 0, 1000000000ull);
    if (!ok && t == 0) atomicCAS(status, 0, SK_ETIMEOUT);
    tc::fence_after_sync();
    if (ok) {
        const int row = warp * 32 + (t & 31);
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16], w[16];
            tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + 256u + (uint32_t)c0, w);
#pragma unroll
            for (int j = 0; j < 16; ++j) d[row * N + c0 + j] = v[j] + w[j];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(taddr, 512);
    }
}

// BF16 form: A (128 x K) as 8-column chunks 2048 bytes apart; x in one plane of 16-byte
// rows of 8 values (x[8m .. 8m+7]); k-step q (16 columns) of B_q[s][t] = x[8 s + 16 q + t]
// is rows s + 2q (t < 8) and s + 2q + 1 (t >= 8): a start address 32 q bytes into the
// plane, 16 bytes between the two core matrices along K.  3 passes, two accumulators.
__global__ void __launch_bounds__(128)
k_tc_sliding_bf16(const float *__restrict__ a, const float *__restrict__ x, float *__restrict__ d, int N, int K,
                  int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int R = N + K / 8;                           // rows of the plane
    const uint32_t slot = (uint32_t)R * 16;
    unsigned char *b_hi = base, *b_lo = base + slot;
    unsigned char *a_hi = base + ((2 * slot + 1023) & ~1023u);
    unsigned char *a_lo = a_hi + (uint32_t)K * 256;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int t = threadIdx.x, warp = t >> 5;

    if (warp == 0) tc::tmem_alloc(&tslot, 512);
    if (t == 0) {
        tc::mbar_init(tc::smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = t; i < 128 * K; i += 128) {
        const int r = i / K, k = i % K;
        uint16_t hi, lo;
        tc::split_bf16(a[i], hi, lo);
        *reinterpret_cast<uint16_t *>(a_hi + tc::kmajor128_offset_bf16(r, k)) = hi;
        *reinterpret_cast<uint16_t *>(a_lo + tc::kmajor128_offset_bf16(r, k)) = lo;
    }
    for (int i = t; i < 8 * R; i += 128) {
        uint16_t hi, lo;
        tc::split_bf16(x[i], hi, lo);
        *reinterpret_cast<uint16_t *>(b_hi + 2 * i) = hi;
        *reinterpret_cast<uint16_t *>(b_lo + 2 * i) = lo;
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;

    if (t == 0) {
        const uint32_t idesc = tc::idesc_bf16(128, N);
        for (int q = 0; q < K / 16; ++q) {
            const uint64_t ah = tc::kmajor_desc(tc::smem_u32(a_hi + 4096 * q), 2048, 128);
            const uint64_t al = tc::kmajor_desc(tc::smem_u32(a_lo + 4096 * q), 2048, 128);
            const uint64_t bh = tc::kmajor_desc(tc::smem_u32(b_hi + 32 * q), 16, 128);
            const uint64_t bl = tc::kmajor_desc(tc::smem_u32(b_lo + 32 * q), 16, 128);
            tc::mma_bf16(taddr, ah, bh, idesc, q > 0);
            tc::mma_bf16(taddr + 256u, ah, bl, idesc, q > 0);
            tc::mma_bf16(taddr + 256u, al, bh, idesc, 1);
        }
        tc::mma_commit(tc::smem_u32(&bar));
    }
    const bool ok = tc::mbar_wait(tc::smem_u32(&bar), 0, 1000000000ull);
    if (!ok && t == 0) atomicCAS(status, 0, SK_ETIMEOUT);
    tc::fence_after_sync();
    if (ok) {
        const int row = warp * 32 + (t & 31);
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16], w[16];
            tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + 256u + (uint32_t)c0, w);
#pragma unroll
            for (int j = 0; j < 16; ++j) d[row * N + c0 + j] = v[j] + w[j];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(taddr, 512);
    }
}

}  // namespace

extern "C" int sk_selftest_tc_sliding_bf16(sk_ctx *ctx, const float *d_a, const float *d_x, float *d_d, int n, int k,
                                           void *stream) {
    if (!ctx || !d_a || !d_x || !d_d) return sk_fail(SK_EINVAL, "sk_selftest_tc_sliding_bf16: NULL argument");
    if (n < 16 || n > 256 || n % 16 || k < 16 || k > 64 || k % 16)
        return sk_fail(SK_EINVAL, "sk_selftest_tc_sliding_bf16: N in 16..256 (x16), K in 16..64 (x16)");
    // a fixed 200 KB: every operand read stays inside the block's shared memory
    const size_t smem = 200 * 1024;
    SK_CU(cudaSetDevice(ctx->device));
    SK_CU(cudaFuncSetAttribute(k_tc_sliding_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_tc_sliding_bf16<<<1, 128, smem, (cudaStream_t)stream>>>(d_a, d_x, d_d, n, k, ctx->d_status);
    SK_CU(cudaGetLastError());
    return SK_OK;
}

extern "C" int sk_selftest_tc_sliding(sk_ctx *ctx, const float *d_a, const float *d_x, float *d_d, int n, int k,
                                      int off, void *stream) {
    if (!ctx || !d_a || !d_x || !d_d) return sk_fail(SK_EINVAL, "sk_selftest_tc_sliding: NULL argument");
    if (n < 16 || n > 256 || n % 16 || k < 8 || k > 64 || k % 8 || (off != 0 && off != 4))
        return sk_fail(SK_EINVAL, "sk_selftest_tc_sliding: N in 16..256 (x16), K in 8..64 (x8), off 0 or 4");
    // a fixed 200 KB: every operand read stays inside the block's shared memory
    const size_t smem = 200 * 1024;
    SK_CU(cudaSetDevice(ctx->device));
    SK_CU(cudaFuncSetAttribute(k_tc_sliding, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_tc_sliding<<<1, 128, smem, (cudaStream_t)stream>>>(d_a, d_x, d_d, n, k, off, ctx->d_status);
    SK_CU(cudaGetLastError());
    return SK_OK;
}

extern "C" int sk_selftest_tc_gemm(sk_ctx *ctx, const float *d_a, const float *d_b, float *d_d, int n, int k,
                                   int passes, void *stream) {
    if (!ctx || !d_a || !d_b || !d_d) return sk_fail(SK_EINVAL, "sk_selftest_tc_gemm: NULL argument");
    if (n < 16 || n > 256 || n % 16 || k < 32 || k > 128 || k % 32 || (passes != 1 && passes != 3))
        return sk_fail(SK_EINVAL, "sk_selftest_tc_gemm: N in 16..256 (x16), K in 32..128 (x32), passes 1 or 3");
    const size_t smem = 1024 + (size_t)2 * (k / 32) * 128 * 128 + (size_t)2 * (k / 32) * n * 128;
    if (smem > 200 * 1024) return sk_fail(SK_EINVAL, "sk_selftest_tc_gemm: operands exceed shared memory");
    SK_CU(cudaSetDevice(ctx->device));
    SK_CU(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_tc_gemm<<<1, 128, smem, (cudaStream_t)stream>>>(d_a, d_b, d_d, n, k, passes, ctx->d_status);
    SK_CU(cudaGetLastError());
    return SK_OK;
}
