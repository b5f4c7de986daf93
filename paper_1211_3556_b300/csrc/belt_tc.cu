// belt_tc.cu -- tensor-core form of the belt path (tcgen05, 3xTF32).
//
// Same operator as the FP32 belt (the real-space convolution of Sec. 2, Eq. 1
// with the tabulated kernel of Sec. 3); only the order of work differs.  In the
// belt every ring has n = 4 Nside pixels and the weight of output pixel j of ring
// o against input pixel j + e of ring i depends on (o, i, e) only.  For a group of
// SK_BELT_G = 16 output rings and one input ring i:
//   y_o[j0 + 8 s + n] += sum_k A_i[(o, n)][k] x_i[j0 + E0 + 8 s + k]
//   A_i[(o, n)][k] = w(o, i, e = k - n + E0)
// a dense product with rows (o, n) = 16 rings x 8 pixels (M = 128), columns
// s = the item's 8-pixel segments (N = nn <= 256) and k < K_i, where E0 is the
// first offset of the union of the group's windows against ring i rounded down
// to a multiple of 4 and K_i covers the union plus the 7 extra columns of the
// 8 output pixels (a multiple of 8).  For k-step q the B operand is
// B_q[s][t] = x_i[j0 + E0 + 8 (s + q) + t]: the input ring read in sliding rows.
// Staged as two slots of 16-byte rows -- the 4-pixel rows v = 0, 2, 4, .. and
// v = 1, 3, 5, .. of the ring from the tile's first column on (pixels j0 + E0 + 4 v
// .. + 3, wrapped around the ring) -- every k-step of both operands is a start
// address in shared memory (no-swizzle K-major, rows 16 bytes apart, the second slot
// one slot further), so nothing is rebuilt inside the loop:
//  * A (TF32 hi and lo parts) is stored per (group, input ring) with the
//    operator (k_tc_tiles) and rebuilt with its table;
//  * the map rows are read as they are: one producer thread bulk-copies (1-D TMA)
//    each tile's A and the raw pixels of its input ring into a pipeline stage, and
//    two converter warps split the pixels into TF32 hi and lo parts and write them
//    into the stage's operand slots.
// 3xTF32 (hi*hi + hi*lo + lo*hi, FP32 accumulation): the tiles of a group are
// taken in chunks of consecutive input rings with at least SK_TC_CHUNK_KSTEPS
// k-steps; each chunk is accumulated by the tensor cores in a fresh
// tensor-memory accumulator, two of them in turn (256 columns each), and the
// epilogue warps add the chunks' partial sums into registers with FP32
// round-to-nearest additions while the next chunk is multiplied.  The tensor
// cores' own accumulation then spans a few tens of MMAs: summing a whole item
// (about 40 tiles, 500 MMAs) in tensor memory measured an rms relative error
// near 1.1e-6 against the FP32 path at Nside 2048, per-tile partial sums 3.6e-7.
// A chunk also keeps each hand-over of an accumulator longer than its round trip
// (single tiles at the window's edge are one k-step).
// The BF16x3 form (SK_BELT_BF16X3) is the same pipeline with BF16 hi/lo parts and
// kind::f16 MMAs of K = 16: half the MMAs, about 1e-5 relative error (16 significant
// bits per operand), outside the 1e-6 bound -- reported beside 3xTF32, never chosen by
// the autotuner.
// Warp roles: 0 producer (bulk copies), 1 MMA issuer, 2..9 epilogue (tensor
// memory -> registers -> outputs), 10..11 converters (raw pixels -> operand
// slots).  The producer takes items (group, map, pixel block) from an atomic
// queue and hands their indices to the other roles through a small ring of
// shared-memory slots (items differ in tile count: against a fixed share per
// CTA, 0.387 -> 0.382 ms at Nside 2048, 4.63 -> 4.47 ms for 64 maps at Nside
// 1024).  Every wait is bounded and records SK_ETIMEOUT.
#include <string.h>

#include <algorithm>

#include "skconv_host.h"
#include "tc.cuh"

namespace {

constexpr int RG = SK_BELT_G;          // output rings per item
constexpr int SO = 128 / RG;           // output pixels per ring per segment
static_assert(RG * SO == 128, "M must be 128");
constexpr int NEPI = 8;                // epilogue warps
constexpr int NCONV = 2;               // converter warps
constexpr int NT = 32 * (2 + NEPI + NCONV);
constexpr unsigned long long LIMIT = 2000000000ull;

// One pipeline stage: A (hi then lo, K x 512 bytes each for TF32, K x 256 for BF16,
// room for kmax), then the operand slots of `slot` bytes (nn + kmax/8 rows of 16
// bytes): two hi and two lo for 3xTF32, one hi and one lo for BF16x3; then the raw
// pixels the slots are made from (8 (nn + kmax/8) floats).
struct Stage {
    uint32_t a_bytes, slot, raw, bytes;
};
__host__ __device__ inline Stage stage_of(int kmax, int nn, bool bf) {
    Stage s;
    s.a_bytes = 2u * (uint32_t)kmax * (bf ? 256u : 512u);
    s.slot = (uint32_t)(nn + kmax / 8) * 16u;
    s.raw = (uint32_t)(nn + kmax / 8) * 32u;
    // no-swizzle operands and bulk copies need 16-byte alignment; stages on 128 bytes
    s.bytes = (s.a_bytes + (bf ? 2u : 4u) * s.slot + s.raw + 127u) & ~127u;
    return s;
}

// Ring group of the gi-th group a launch runs (two ranges, the second possibly empty).
__device__ __forceinline__ int group_of(const TcArgs &T, int gi) {
    const int na = T.ga1 - T.ga0;
    return gi < na ? T.ga0 + gi : T.gb0 + (gi - na);
}

__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *status) {
    if (*abort_flag) return false;
    if (tc::mbar_wait(bar, parity, LIMIT)) return true;
    *abort_flag = 1;
    atomicCAS(status, 0, SK_ETIMEOUT);
    return false;
}

// Items: the producer takes each from the launch's queue (an atomic counter, so CTAs that
// start late -- beside another launch -- take fewer) and writes it to slot ic mod NITEM;
// every other role reads the slots in the same order.  take_item: the ic-th item (T.total
// when there are none left or after an abort); `arrive` for one thread of each reading unit
// (the MMA thread, each epilogue and converter warp), after its lanes have read the slot.
constexpr int NITEM = 4;
__device__ __forceinline__ int take_item(const int *sitem, uint64_t *ifull, uint64_t *iempty, uint32_t ic,
                                         volatile int *abort_flag, int *status, bool arrive) {
    const int si = (int)(ic % NITEM);
    int f = 1 << 30;
    if (wait_or_abort(tc::smem_u32(&ifull[si]), (ic / NITEM) & 1, abort_flag, status)) f = sitem[si];
    __syncwarp(__activemask());
    if (arrive) tc::mbar_arrive1(tc::smem_u32(&iempty[si]));
    return f;
}

// BF: the BF16x3 form -- BF16 hi/lo parts, K = 16 per MMA (kind::f16), one slot of
// 8-pixel rows per part: B_q[s][t] = rows s + 2q and s + 2q + 1 of the slot, a start
// address 32 q bytes in with 16 bytes between the two core matrices along K.
template <bool BF>
__global__ void __launch_bounds__(NT, 1) k_belt_tc(const __grid_constant__ TcArgs T) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    __shared__ __align__(8) uint64_t full_bar[SK_TC_MAX_STAGES];    // copies of a stage landed
    __shared__ __align__(8) uint64_t conv_bar[SK_TC_MAX_STAGES];    // its operand slots written
    __shared__ __align__(8) uint64_t empty_bar[SK_TC_MAX_STAGES];   // MMAs reading a stage done
    __shared__ __align__(8) uint64_t tfull_bar[2];                  // a tile's partial sums complete
    __shared__ __align__(8) uint64_t tempty_bar[2];                 // the epilogue has read them
    __shared__ __align__(8) uint64_t drain_bar;                     // teardown
    __shared__ int4 stile[SK_TC_MAX_STAGES];                        // the tile each stage holds
    // the items the producer takes from the launch's queue, handed to the other roles
    __shared__ int sitem[NITEM];
    __shared__ __align__(8) uint64_t ifull_bar[NITEM];              // an item index written
    __shared__ __align__(8) uint64_t iempty_bar[NITEM];             // every role has read it
    __shared__ uint32_t tslot;
    __shared__ int abort_s;
    volatile int *abort_flag = &abort_s;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int S = T.nstages;
    const Stage L = stage_of(T.kmax, T.nn, BF);
    const int per_g = T.batch * T.nblk;
    constexpr int NPL = BF ? 2 : 4;                 // operand slots per stage
    constexpr uint32_t APART = BF ? 256u : 512u;    // bytes of one part of A per column

    if (warp == 0) tc::tmem_alloc(&tslot, 512);
    if (t == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(tc::smem_u32(&full_bar[s]), 1);
            tc::mbar_init(tc::smem_u32(&conv_bar[s]), NCONV);
            tc::mbar_init(tc::smem_u32(&empty_bar[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(tc::smem_u32(&tfull_bar[a]), 1);
            tc::mbar_init(tc::smem_u32(&tempty_bar[a]), NEPI);
        }
        for (int i = 0; i < NITEM; ++i) {
            tc::mbar_init(tc::smem_u32(&ifull_bar[i]), 1);
            tc::mbar_init(tc::smem_u32(&iempty_bar[i]), 1 + NEPI + NCONV);
        }
        tc::mbar_init(tc::smem_u32(&drain_bar), 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;

    if (warp == 0) {
        // ---------------- producer ----------------
        if (lane == 0) {
            uint32_t cnt = 0;
            for (uint32_t ic = 0;; ++ic) {
                // the next item from the queue (T.total: none left), handed to the other roles
                const int f = *abort_flag ? T.total : min(atomicAdd(T.queue, 1), T.total);
                const int si = (int)(ic % NITEM);
                if (ic >= NITEM && !wait_or_abort(tc::smem_u32(&iempty_bar[si]), ((ic / NITEM) - 1) & 1,
                                                  abort_flag, T.status))
                    break;
                sitem[si] = f;
                tc::mbar_arrive1(tc::smem_u32(&ifull_bar[si]));
                if (f >= T.total) break;
                const int gi = f / per_g, rem = f - gi * per_g, b = rem / T.nblk, pb = rem - b * T.nblk;
                const int j0 = pb * 8 * T.nn;
                const int4 tr = T.trng[group_of(T, gi)];
                const float *xb = T.x + (long long)b * T.stride;
                for (int u = 0; u < tr.y; ++u, ++cnt) {
                    const int4 tl = T.tiles[tr.x + u];            // (input ring, E0, K | flags, A offset in KB)
                    const int s = (int)(cnt % (uint32_t)S);
                    if (cnt >= (uint32_t)S &&
                        !wait_or_abort(tc::smem_u32(&empty_bar[s]), ((cnt / S) - 1) & 1, abort_flag, T.status))
                        break;
                    const int K = tl.z & SK_TC_K_MASK;
                    const int npix = 8 * (T.nn + K / 8 - 1);      // pixels j0 + E0 .. of the input ring
                    unsigned char *sb = base + (size_t)s * L.bytes;
                    const uint32_t bar = tc::smem_u32(&full_bar[s]);
                    const uint32_t abytes = 2u * (uint32_t)K * APART;
                    stile[s] = tl;                                // read after the barrier
                    tc::mbar_expect_tx(bar, abytes + 4u * (uint32_t)npix);
                    tc::bulk_g2s(tc::smem_u32(sb), T.A + (size_t)tl.w * 1024, abytes, bar);
                    // the raw pixels, wrapped around the ring: pieces start on 4-pixel
                    // boundaries (E0, j0 and the ring length are multiples of 4)
                    const float *xr = xb + T.rings[tl.x].start;
                    int p = (j0 + tl.y) % T.n4;
                    if (p < 0) p += T.n4;
                    uint32_t dst = tc::smem_u32(sb + L.a_bytes + NPL * L.slot);
                    for (int rem = npix; rem > 0;) {
                        const int c = min(rem, T.n4 - p);
                        tc::bulk_g2s(dst, xr + p, 4u * (uint32_t)c, bar);
                        dst += 4u * (uint32_t)c;
                        rem -= c;
                        p = 0;
                    }
                }
            }
            // copies still in flight land before the block exits (bounded)
            for (uint32_t c = cnt > (uint32_t)S ? cnt - S : 0; c < cnt; ++c)
                tc::mbar_wait(tc::smem_u32(&full_bar[c % S]), (c / S) & 1, LIMIT);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            uint32_t cnt = 0, ccnt = 0;                           // tiles, chunks
            const uint32_t idesc = BF ? tc::idesc_bf16(128, T.nn) : tc::idesc_tf32(128, T.nn);
            bool need_empty = false;                              // the next tile opens a chunk
            for (uint32_t ic = 0;; ++ic) {
                const int f = take_item(sitem, ifull_bar, iempty_bar, ic, abort_flag, T.status, true);
                if (f >= T.total) break;
                const int ntile = T.trng[group_of(T, f / per_g)].y;
                for (int u = 0; u < ntile; ++u, ++cnt) {
                    const int s = (int)(cnt % (uint32_t)S);
                    const int ab = (int)(ccnt & 1);               // accumulator of this chunk
                    // a chunk starts at the group's first tile or after a chunk's last one:
                    // its accumulator must have been read by the epilogue (two chunks ago)
                    if ((u == 0 || need_empty) && ccnt >= 2 &&
                        !wait_or_abort(tc::smem_u32(&tempty_bar[ab]), ((ccnt >> 1) - 1) & 1, abort_flag, T.status))
                        break;
                    if (!wait_or_abort(tc::smem_u32(&full_bar[s]), (cnt / S) & 1, abort_flag, T.status)) break;
                    if (!wait_or_abort(tc::smem_u32(&conv_bar[s]), (cnt / S) & 1, abort_flag, T.status)) break;
                    tc::fence_after_sync();
                    const int4 tl = stile[s];
                    const bool first = (tl.z & SK_TC_FIRST) != 0, last = (tl.z & SK_TC_LAST) != 0;
                    need_empty = last;
                    const int K = tl.z & SK_TC_K_MASK;
                    const uint32_t sb = tc::smem_u32(base + (size_t)s * L.bytes);
                    const uint32_t a_hi = sb, a_lo = sb + (uint32_t)K * APART;
                    const uint32_t d = taddr + 256u * (uint32_t)ab;
                    // descriptors of the k-step's operands: the start address is their low
                    // field (16-byte units), so a k-step is an add (4096 bytes in A, 32 or 16
                    // bytes in B); addresses stay below 256 KB, so the field never carries
                    const uint32_t b_hi = sb + L.a_bytes, b_lo = b_hi + (BF ? 1u : 2u) * L.slot;
                    uint64_t ah = tc::kmajor_desc(a_hi, 2048, 128), al = tc::kmajor_desc(a_lo, 2048, 128);
                    uint64_t bh = tc::kmajor_desc(b_hi, BF ? 16u : L.slot, 128);
                    uint64_t bl = tc::kmajor_desc(b_lo, BF ? 16u : L.slot, 128);
                    constexpr uint64_t DA = 4096u >> 4, DB = (BF ? 32u : 16u) >> 4;
                    const int nq = K / (BF ? 16 : 8);
                    for (int q = 0; q < nq; ++q) {
                        if constexpr (BF) {
                            tc::mma_bf16(d, ah, bh, idesc, (first && q == 0) ? 0 : 1);
                            tc::mma_bf16(d, ah, bl, idesc, 1);
                            tc::mma_bf16(d, al, bh, idesc, 1);
                        } else {
                            tc::mma_tf32(d, ah, bh, idesc, (first && q == 0) ? 0 : 1);
                            tc::mma_tf32(d, ah, bl, idesc, 1);
                            tc::mma_tf32(d, al, bh, idesc, 1);
                        }
                        ah += DA; al += DA; bh += DB; bl += DB;
                    }
                    tc::mma_commit(tc::smem_u32(&empty_bar[s]));
                    if (last) {
                        tc::mma_commit(tc::smem_u32(&tfull_bar[ab]));
                        ++ccnt;
                    }
                }
            }
            // every MMA this thread issued has completed before tensor memory is released
            tc::mma_commit(tc::smem_u32(&drain_bar));
            tc::mbar_wait(tc::smem_u32(&drain_bar), 0, LIMIT);
        }
    } else if (warp < 2 + NEPI) {
        // ---------------- epilogue ----------------
        // warp w reads lane quadrant w % 4 (rows 32 (w % 4) ..) and the 16-column chunks
        // 16 half, 16 half + 32, ...: up to eight chunks of partial sums held in registers
        constexpr int CH = 8;
        const int quad = warp & 3, half = (warp - 2) >> 2;
        const int row = quad * 32 + lane, r = row / SO, n = row - r * SO;
        const int nch = (T.nn - 16 * half + 31) / 32;
        uint32_t ccnt = 0;
        for (uint32_t ic = 0;; ++ic) {
            const int f = take_item(sitem, ifull_bar, iempty_bar, ic, abort_flag, T.status, lane == 0);
            if (f >= T.total) break;
            const int gi = f / per_g, rem = f - gi * per_g, b = rem / T.nblk, pb = rem - b * T.nblk;
            const int g = group_of(T, gi);
            const int j0 = pb * 8 * T.nn;
            const int nchunk = T.trng[g].z;
            float acc[CH][16];
#pragma unroll
            for (int c = 0; c < CH; ++c)
#pragma unroll
                for (int m = 0; m < 16; ++m) acc[c][m] = 0.0f;
            bool ok = true;
            for (int u = 0; u < nchunk; ++u) {
                const int ab = (int)(ccnt & 1);
                if (!wait_or_abort(tc::smem_u32(&tfull_bar[ab]), (ccnt >> 1) & 1, abort_flag, T.status)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t lane_base = taddr + ((uint32_t)(quad * 32) << 16) + 256u * (uint32_t)ab;
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    if (c < nch) {
                        float v[16];
                        tc::tmem_ld16(lane_base + (uint32_t)(16 * half + 32 * c), v);
#pragma unroll
                        for (int m = 0; m < 16; ++m) acc[c][m] += v[m];
                    }
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive1(tc::smem_u32(&tempty_bar[ab]));
                ++ccnt;
            }
            if (!ok) break;
            const int rb = g * RG + r;
            if (rb < T.nb) {
                float *yr = T.y + (long long)b * T.stride + T.rings[T.b_lo + rb].start;
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    if (c < nch) {
#pragma unroll
                        for (int m = 0; m < 16; ++m) {
                            const int j = j0 + SO * (16 * half + 32 * c + m) + n;
                            if (j < T.n4) yr[j] = acc[c][m];
                        }
                    }
                }
            }
        }
    } else {
        // ---------------- converters ----------------
        // the stage's raw pixels into its operand slots: 3xTF32 4-pixel row v to slot
        // v & 1 (row v >> 1) of the hi and lo parts, BF16x3 8-pixel row v to row v of
        // the hi and lo slots; then the writes are made visible to the tensor cores
        const int c = warp - 2 - NEPI;
        uint32_t cnt = 0;
        for (uint32_t ic = 0;; ++ic) {
            const int f = __shfl_sync(0xffffffffu, take_item(sitem, ifull_bar, iempty_bar, ic, abort_flag,
                                                             T.status, lane == 0), 0);
            if (f >= T.total || __shfl_sync(0xffffffffu, *abort_flag, 0)) break;   // the same in every lane
            const int ntile = T.trng[group_of(T, f / per_g)].y;
            bool ok = true;
            for (int u = 0; u < ntile; ++u, ++cnt) {
                const int s = (int)(cnt % (uint32_t)S);
                ok = wait_or_abort(tc::smem_u32(&full_bar[s]), (cnt / S) & 1, abort_flag, T.status);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                const int4 tl = stile[s];
                const int R = T.nn + (tl.z & SK_TC_K_MASK) / 8 - 1;     // rows per slot
                unsigned char *sb = base + (size_t)s * L.bytes;
                const float4 *raw = reinterpret_cast<const float4 *>(sb + L.a_bytes + NPL * L.slot);
                if constexpr (BF) {
                    uint4 *hs = reinterpret_cast<uint4 *>(sb + L.a_bytes);
                    uint4 *ls = reinterpret_cast<uint4 *>(sb + L.a_bytes + L.slot);
                    for (int v = 32 * c + lane; v < R; v += 32 * NCONV) {
                        const float4 x0 = raw[2 * v], x1 = raw[2 * v + 1];
                        const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                        uint32_t h[4], l[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            uint16_t h0, l0, h1, l1;
                            tc::split_bf16(xv[2 * e], h0, l0);
                            tc::split_bf16(xv[2 * e + 1], h1, l1);
                            h[e] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                            l[e] = (uint32_t)l0 | ((uint32_t)l1 << 16);
                        }
                        hs[v] = make_uint4(h[0], h[1], h[2], h[3]);
                        ls[v] = make_uint4(l[0], l[1], l[2], l[3]);
                    }
                } else {
                    for (int v = 32 * c + lane; v < 2 * R; v += 32 * NCONV) {
                        const float4 xv = raw[v];
                        float4 h, l;
                        tc::split_tf32(xv.x, h.x, l.x);
                        tc::split_tf32(xv.y, h.y, l.y);
                        tc::split_tf32(xv.z, h.z, l.z);
                        tc::split_tf32(xv.w, h.w, l.w);
                        const uint32_t o = (uint32_t)(v & 1) * L.slot + 16u * (uint32_t)(v >> 1);
                        *reinterpret_cast<float4 *>(sb + L.a_bytes + o) = h;
                        *reinterpret_cast<float4 *>(sb + L.a_bytes + 2u * L.slot + o) = l;
                    }
                }
                tc::fence_smem_to_async();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive1(tc::smem_u32(&conv_bar[s]));
            }
            if (!ok) break;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(taddr, 512);
    }
}

// One block per tile: A_i[(o, n)][k] = w(o, i, k - n + E0) for the group's rings,
// zero outside each ring's window, split into TF32 (or BF16) hi and lo parts and
// written in the no-swizzle K-major image the MMA reads (kmajor128_offset(_bf16); lo
// K x 512 (256) bytes after hi).  The weight is the FP32 belt's (pair_weight of the
// same half-angle).
__global__ void k_tc_tiles(const __grid_constant__ TcTileArgs T, const int *gate) {
    if (gate && !*gate) return;                      // table unchanged: the tiles stand
    const int tile = blockIdx.x;
    const int4 tl = T.tiles[tile];
    const int g = T.tile_group[tile];
    const int K = tl.z & SK_TC_K_MASK;
    unsigned char *hi = T.A + (size_t)tl.w * 1024, *lo = hi + (size_t)K * (T.bf16 ? 256 : 512);
    const double half_step = SK_PI / (2.0 * (double)T.n4);
    for (int idx = threadIdx.x; idx < 128 * K; idx += blockDim.x) {
        const int row = idx / K, k = idx - row * K;
        const int r = row / SO, n = row - r * SO;
        const int rb = g * RG + r, e = k - n + tl.y;
        float v = 0.0f;
        if (rb < T.nb) {
            const int ro = T.b_lo + rb;
            const int p0 = T.pair_off[ro], p1 = T.pair_off[ro + 1];
            const int p = p0 + (tl.x - T.pairs[p0].ri);
            if (p >= p0 && p < p1) {
                const PairInfo P = T.pairs[p];
                const int s_o = T.rings[ro].s;
                const int ec = (s_o + 1 - P.s_i) >> 1;
                if (e >= ec - P.W && e <= ec + P.W) {
                    const float x = (float)((double)(2 * e + P.s_i - s_o) * half_step);
                    v = pair_weight(x, P.A, P.B, T.kp, T.tab);
                }
            }
        }
        if (T.bf16) {
            uint16_t h, l;
            tc::split_bf16(v, h, l);
            *reinterpret_cast<uint16_t *>(hi + tc::kmajor128_offset_bf16(row, k)) = h;
            *reinterpret_cast<uint16_t *>(lo + tc::kmajor128_offset_bf16(row, k)) = l;
        } else {
            float h, l;
            tc::split_tf32(v, h, l);
            *reinterpret_cast<float *>(hi + tc::kmajor128_offset(row, k)) = h;
            *reinterpret_cast<float *>(lo + tc::kmajor128_offset(row, k)) = l;
        }
    }
}

}  // namespace

int sk_tc_stages(int kmax, int nn, bool bf16, size_t *smem) {
    const Stage L = stage_of(kmax, nn, bf16);
    // the opt-in maximum of dynamic shared memory per block (227 KB) less the static
    // barriers and the base alignment
    const size_t avail = (size_t)227 * 1024 - 1024 - 128;
    int S = (int)std::min<size_t>(SK_TC_MAX_STAGES, avail / L.bytes);
    if (S < 2) return 0;
    // at least 120 KB so that one block holds an SM (it allocates all 512 tensor-memory columns)
    if (smem) *smem = std::max((size_t)128 + (size_t)S * L.bytes, (size_t)120 * 1024);
    return S;
}

cudaError_t sk_launch_belt_tc(const TcArgs &a, int grid, cudaStream_t st) {
    if (a.total <= 0) return cudaSuccess;
    size_t smem = 0;
    if (sk_tc_stages(a.kmax, a.nn, a.bf16 != 0, &smem) != a.nstages) return cudaErrorInvalidValue;
    if (a.bf16) {
        cudaError_t e = cudaFuncSetAttribute(k_belt_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_belt_tc<true><<<grid, NT, smem, st>>>(a);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_belt_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_belt_tc<false><<<grid, NT, smem, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t sk_launch_tc_tiles(const TcTileArgs &a, int n_tiles, cudaStream_t st, const int *gate) {
    if (n_tiles <= 0) return cudaSuccess;
    k_tc_tiles<<<n_tiles, 256, 0, st>>>(a, gate);
    return cudaGetLastError();
}
