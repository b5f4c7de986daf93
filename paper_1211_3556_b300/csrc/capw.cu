// capw.cu -- polar-cap path with the operator's weights stored in HBM.
//
// The operator (Sec. 2, Eq. 1 with the tabulated kernel of Sec. 3) does not change
// between calls, so the weights dOmega K_lin(gamma) of the caps' base pairs (one per
// 16 symmetric pairs, see cap_common.cuh) are evaluated once per kernel table by
// k_capw_build -- with the same FP32 arithmetic, bit for bit, as the evaluating cap
// kernel uses -- and every call streams them instead of evaluating them.  The sum
// loop is then 32 paired FMAs per pixel and thread, fed by four 128-bit shared loads
// of the strip and one 128-bit load of the weight stream.
//
// A thread owns four adjacent base outputs jt .. jt + 3 (jt = j0 + 4 t) of a work
// item (256 base outputs, 64 threads) and walks the union of their windows on each
// input ring: NS = cnt + ceil(3 n_i / n_o) pixel steps (the four windows start at
// most that far apart), rounded up to groups of four.  Weights outside an output's
// own window are stored as 0 (as are those of outputs beyond the ring's base range),
// so each output sums exactly the terms of its window, in the same order as the
// evaluating kernel.  The weight stream of an item is [step s][thread t] float4
// (outputs jt .. jt + 3), rows of 64 threads (in the last item of a ring only the first
// ones have outputs; the others' entries are neither written nor read), steps running
// on across its rings; an item of ring r starts at capw_ring[r].x + (j0 / 256)
// capw_ring[r].y * 64 float4.
//
// The strips are staged as in the evaluating kernel, but with the symmetric copy and
// the strip rows split by residue modulo 4: lanes four pixels apart then read
// consecutive float4.  Each item stages a strip long enough for the union of its last
// active thread, so every position a thread reads was copied.
#include "skconv.h"
#include "cap_common.cuh"

namespace {

using namespace capc;

constexpr int NTW = 64;     // threads per work item: four adjacent base outputs each
constexpr int OPT = 4;      // outputs per thread
static_assert(CT == OPT * NTW, "an item is 256 base outputs");
// work items per block and strip buffers per item: two buffers (ring p + 1 staged while
// ring p is summed) for narrow windows where they fit in shared memory; one for the
// wide windows of blocked summation, whose rings take long enough to sum that staging
// each one in turn costs little, and which then fit 6 / 3 items per block instead of
// 4 / 2 (measured at 300', Nside 1024: 20.3 -> 16.5 ms per map)
template <int LS, bool BLK>
__host__ __device__ constexpr int capw_slots() { return LS <= 288 ? 6 : (LS <= 640 && BLK ? 3 : 2); }
template <int LS, bool BLK>
__host__ __device__ constexpr int capw_bufs() { return BLK ? 1 : (LS <= 640 ? 2 : 1); }
// dynamic shared memory: strips [slots][NB][4][LS] float4, then the full and empty
// mbarriers of every buffer and the abort flag (16-byte multiple), then with blocked
// summation the threads' running totals [64 values][threads] float
__host__ __device__ constexpr size_t capw_strip_bytes(int ls, int nb, int slots) { return (size_t)slots * nb * 4 * ls * 16; }
__host__ __device__ constexpr size_t capw_bar_bytes(int nb, int slots) { return ((size_t)2 * slots * nb * 8 + 4 + 15) / 16 * 16; }
__host__ __device__ constexpr size_t capw_tot_bytes(bool blk, int slots) { return blk ? (size_t)64 * slots * 64 * 4 : 0; }
// node tables of up to this many nodes are held as (value, slope) pairs, larger ones as
// values (as in the evaluating kernel, whose weights the builder reproduces)
constexpr int PAIR_TABLE_NODES = 8192;

// The item's two warps (named barrier 1 + slot).
__device__ __forceinline__ void slot_sync(int slot) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + slot), "r"(NTW) : "memory");
}

// The strip of input ring P for an item with outputs j0 .. jlast: the union windows of
// all its active threads, from pixel u0 = centre(j0) - before.
__device__ __forceinline__ Strip stripw_of(const PairInfo &P, int j0, int jlast, int n_o, int s_o, unsigned mg,
                                           int sh) {
    int before, cnt;
    win_shape(P, before, cnt);
    const int jl = j0 + OPT * ((jlast - j0) / OPT);      // first output of the last active thread
    const int c0 = centre_of(j0, n_o, s_o, P, mg, sh), c1 = centre_of(jl, n_o, s_o, P, mg, sh);
    return Strip{c1 - c0 + sk_capw_steps(cnt, P.n_i, n_o), c0 - before};
}

// 128-bit shared-memory load by 32-bit shared address.
__device__ __forceinline__ float4 lds4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

// Bulk prefetch of [p, p + bytes) into L2 (TMA; 16-byte aligned, a multiple of 16 bytes).
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// Steps of the weight stream the L2 prefetch keeps ahead of the sums (about a ring;
// measured at Nside 2048: 24 steps 0.754 ms, 48 0.773, 96 0.884, 160 0.927 -- a longer
// run-ahead displaces the symmetric copy from L2)
constexpr int PF_STEPS = 24;

// Streamed weights: read once per call, kept out of L1, first out of L2 (policy).
__device__ __forceinline__ float4 ld_stream(const float4 *p, uint64_t policy) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(policy));
    return v;
}

// The 16 images of one staged position for the four outputs: x values a, b (forward
// segments: the pixel and its quarter turn, each with its half turn and mirrors) and c,
// d (the reflected ones); acc[k][0..3] take the forward images and acc[k][4..7] the
// reflected ones, as in the evaluating kernel.
__device__ __forceinline__ void mac16x4(float2 (&acc)[OPT][8], const float4 w, const float4 a, const float4 b,
                                        const float4 c, const float4 d) {
    const float ws[OPT] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < OPT; ++k) {
        const float2 ww = f2(ws[k]);
        acc[k][0] = __ffma2_rn(ww, make_float2(a.x, a.y), acc[k][0]);
        acc[k][1] = __ffma2_rn(ww, make_float2(a.z, a.w), acc[k][1]);
        acc[k][2] = __ffma2_rn(ww, make_float2(b.x, b.y), acc[k][2]);
        acc[k][3] = __ffma2_rn(ww, make_float2(b.z, b.w), acc[k][3]);
        acc[k][4] = __ffma2_rn(ww, make_float2(c.x, c.y), acc[k][4]);
        acc[k][5] = __ffma2_rn(ww, make_float2(c.z, c.w), acc[k][5]);
        acc[k][6] = __ffma2_rn(ww, make_float2(d.x, d.y), acc[k][6]);
        acc[k][7] = __ffma2_rn(ww, make_float2(d.z, d.w), acc[k][7]);
    }
}

// Two strip buffers per item (NB == 2): ring g of a slot's sequence (rings of its items
// one after another) is staged into buffer g mod 2.  full[b] counts the bytes of a
// strip's bulk copies; empty[b] takes one arrival per warp when the warp is done with
// the ring in buffer b.  The warp that stages ring g + 1 (into buffer (g + 1) mod 2)
// waits for ring g - 1's release of that buffer: neither warp ever waits for the other
// otherwise.  With one buffer (NB == 1) the item's threads synchronise at every ring.
// Twelve warps per block at most: the SM's four sub-partitions hold 16K registers each
// and three warps of the block share one, so a thread gets at most 168 registers.
// BLK (operators whose outputs sum thousands of terms): the sums of each input ring are
// added to the thread's running totals, kept in its own slice of shared memory (the
// registers hold the 64 sums of one ring), so that the FP32 rounding grows with the
// terms of one ring and the number of rings, not with their product.
template <int LS, bool BLK>
__global__ void __launch_bounds__(NTW * capw_slots<LS, BLK>(), 1)
k_conv_capw(const __grid_constant__ JobsArg A) {
    constexpr int NB = capw_bufs<LS, BLK>(), SLOTS = capw_slots<LS, BLK>();
    constexpr int NTH = NTW * SLOTS;
    extern __shared__ __align__(16) float4 sx[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<char *>(sx) + capw_strip_bytes(LS, NB, SLOTS));
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 2 * SLOTS * NB);
    float *const tot = reinterpret_cast<float *>(reinterpret_cast<char *>(sx) + capw_strip_bytes(LS, NB, SLOTS) +
                                                 capw_bar_bytes(NB, SLOTS)) + threadIdx.x;   // value i at tot[i NTH]
    if (threadIdx.x == 0) {
        for (int b = 0; b < SLOTS * NB; ++b) {
            tc::mbar_init(tc::smem_u32(bars + b), 1);                  // full: the expect_tx arrival
            tc::mbar_init(tc::smem_u32(bars + SLOTS * NB + b), 2);     // empty: one arrival per warp
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int slot = threadIdx.x / NTW, t = threadIdx.x % NTW, warp = t >> 5, lane = t & 31;
    float4 *const sbuf = sx + slot * NB * 4 * LS;
    const uint32_t full0 = tc::smem_u32(bars + slot * NB), empty0 = tc::smem_u32(bars + SLOTS * NB + slot * NB);
    // the symmetric copy stays in L2 while its rings are re-read by neighbouring output
    // rings; the weight stream is read once and goes first
    const uint64_t pol_strip = tc::l2_policy_evict_last(), pol_w = tc::l2_policy_evict_first();
    uint32_t fphase = 0;    // bit b: parity of the next phase of full[b] (the same in every thread)
    uint32_t pend = 0;      // bit b set while a copy this thread's warp issued into buffer b is not waited for
    int gseq = 0;           // the slot's ring sequence number (the same in every thread of the slot)
    // Wait (bounded) until both warps released ring g - 1 from buffer (g + 1) mod 2 ... i.e.
    // until the buffer that ring g + 1 goes to is free; false after an abort.
    auto wait_free = [&](int g) -> bool {
        if (g < 1) return true;                // buffers start free
        const int gp = g - 1;
        return strip_wait(empty0 + 8 * (gp & 1), (uint32_t)(gp >> 1) & 1, abort_flag);
    };
    // work queue (items heaviest first); with two buffers the warp that stages after an
    // item's last ring takes the slot's next item and stages its first strip
    __shared__ int s_item[SLOTS];
    __shared__ int s_pref[SLOTS];
    if (t == 0) {
        s_item[slot] = atomicAdd(A.queue, 1);
        s_pref[slot] = 0;
    }
    for (;;) {
        slot_sync(slot);
        const int f = s_item[slot];
        const bool pref = NB == 2 && s_pref[slot] != 0;
        if (f >= A.total) break;
        const JobDesc &J = A.j[sk_find_job(A, f)];
        // the maps of a job's batch are the innermost index of its work: one item's maps
        // are taken one after another, so its weights come from HBM once and from L2 for
        // the other maps (queued map by map, a batch re-read the whole stream per map)
        const int local = f - J.flat_base;
        const int item = local / J.batch, map = local - item * J.batch;
        const int4 it = J.items[item];
        const int ro = it.x, j0 = it.y;
        const unsigned mg = (unsigned)it.z;            // division by 2 n_o (centre_of)
        const int sh = it.w;
        const RingDev R = J.rings[ro];
        const int Qo = R.n >> 2;
        const int T = base_count(Qo, R.s);
        const int jlast = min(j0 + CT - 1, T - 1);
        const int jt = j0 + OPT * t;
        const bool act = jt < T;
        const int ro_s = J.nr - 1 - ro;
        const float4 *hmap = J.hx + (long long)map * J.hstride;
        const int p0 = J.pair_off[ro], p1 = J.pair_off[ro + 1];
        const longlong2 wr = J.capw_ring[ro];
        // the item's stream: [step][thread] float4, rows of 64 threads of which the first
        // nthr have outputs
        const int nthr = (jlast - j0) / OPT + 1;
        const float4 *witem = J.capw + wr.x + (long long)(j0 / CT) * wr.y * NTW;
        const float4 *wp = witem + t;
        // thread 0 keeps the item's stream prefetched into L2 PF_STEPS steps ahead of the
        // sums, by bulk prefetches at ring boundaries (the steps up to pf are requested):
        // whole rows, or in an item with fewer threads the part of each row they read
        long long pf = 0;
        auto prefetch_to = [&](long long upto) {
            upto = min(upto, (long long)wr.y);
            if (t == 0 && upto > pf) {
                if (nthr == NTW) {
                    prefetch_l2(witem + pf * NTW, (uint32_t)((upto - pf) * NTW * 16));
                } else {
                    for (long long s = pf; s < upto; ++s) prefetch_l2(witem + s * NTW, (uint32_t)nthr * 16u);
                }
                pf = upto;
            }
        };
        prefetch_to(2 * PF_STEPS);

        float2 acc[OPT][8];
#pragma unroll
        for (int k = 0; k < OPT; ++k)
#pragma unroll
            for (int s = 0; s < 8; ++s) acc[k][s] = make_float2(0.0f, 0.0f);
        if constexpr (BLK) {
#pragma unroll
            for (int i = 0; i < 16 * OPT; ++i) tot[i * NTH] = 0.0f;
        }

        // ring p's strip into buffer b by bulk copies (by the calling warp), unless it
        // wraps the whole ring (then the item's threads copy it when they reach it)
        auto issue = [&](int p, int b) {
            const PairInfo Pn = J.pairs[p];
            const Strip S = stripw_of(Pn, j0, jlast, R.n, R.s, mg, sh);
            const int stop = __shfl_sync(0xffffffffu, *abort_flag, 0);
            if (S.L < Pn.n_i && !stop) {
                issue_strip<4, LS, true>(sbuf + b * 4 * LS, full0 + 8 * b, hmap + J.rings[Pn.ri].start, S, Pn, lane,
                                         pol_strip);
                pend |= 1u << b;
            }
        };
        // the first strip of item fn into buffer b by the calling warp; returns whether it was staged
        auto stage_first = [&](int fn, int b) -> int {
            const JobDesc &Jn = A.j[sk_find_job(A, fn)];
            const int ln = fn - Jn.flat_base;
            const int itm = ln / Jn.batch, mn = ln - itm * Jn.batch;
            const int4 itn = Jn.items[itm];
            const RingDev Rn = Jn.rings[itn.x];
            const int jln = min(itn.y + CT - 1, base_count(Rn.n >> 2, Rn.s) - 1);
            const PairInfo Pn = Jn.pairs[Jn.pair_off[itn.x]];
            const Strip Sn = stripw_of(Pn, itn.y, jln, Rn.n, Rn.s, (unsigned)itn.z, itn.w);
            const int stop = __shfl_sync(0xffffffffu, *abort_flag, 0);
            if (Sn.L < Pn.n_i && !stop) {
                const float4 *hn = Jn.hx + (long long)mn * Jn.hstride;
                issue_strip<4, LS, true>(sbuf + b * 4 * LS, full0 + 8 * b, hn + Jn.rings[Pn.ri].start, Sn, Pn, lane,
                                         pol_strip);
                pend |= 1u << b;
                return 1;
            }
            return 0;
        };
        if (NB == 2 && !pref && p0 < p1 && warp == 0) {
            if (!wait_free(gseq - 1)) { if (!*abort_flag) { *abort_flag = 1; sk_record_error(A.status, SK_ETIMEOUT); } }
            issue(p0, gseq & 1);
        }
        // weights of the first group of steps; later groups are loaded one group ahead
        float4 wc[4];
        if (act) {
#pragma unroll
            for (int q = 0; q < 4; ++q) wc[q] = ld_stream(wp + q * NTW, pol_w);
        }
        long long s0 = 0;       // stream step of the current group
        for (int p = p0; p < p1; ++p, ++gseq) {
            const int b = NB == 2 ? (gseq & 1) : 0;
            float4 *const xbuf = sbuf + b * 4 * LS;
            const PairInfo P = J.pairs[p];
            const Strip S = stripw_of(P, j0, jlast, R.n, R.s, mg, sh);
            const bool bulk = S.L < P.n_i;
            bool ok = true;
            if (NB == 2) {
                // release ring g - 1's buffer; the stager of ring g + 1 (the warps take turns)
                // waits until the other warp released it too, then stages ring g + 1 -- or,
                // after the item's last ring, the slot's next item's first ring
                __syncwarp();
                if (gseq >= 1 && lane == 0) tc::mbar_arrive1(empty0 + 8 * (b ^ 1));
                const bool stager = ((p + 1 - p0) & 1) == warp;
                if (stager) {
                    if (!wait_free(gseq)) ok = false;
                    if (p + 1 < p1) {
                        issue(p + 1, b ^ 1);
                    } else {
                        int fn = 0;
                        if (lane == 0) fn = *abort_flag ? A.total : atomicAdd(A.queue, 1);
                        fn = __shfl_sync(0xffffffffu, fn, 0);
                        const int staged = fn < A.total ? stage_first(fn, b ^ 1) : 0;
                        if (lane == 0) {
                            s_item[slot] = fn;          // read after the slot barrier that opens the next item
                            s_pref[slot] = staged;
                        }
                    }
                }
            } else {
                slot_sync(slot);
                if (bulk && warp == 0) issue(p, 0);
            }
            if (bulk) {
                if (strip_wait(full0 + 8 * b, (fphase >> b) & 1, abort_flag)) {
                    pend &= ~(1u << b);
                } else {
                    ok = false;
                }
                fphase ^= 1u << b;
            } else {
                // the buffer held ring g - 2: wait until both warps released it, copy, share
                if (NB == 2 && !wait_free(gseq - 1)) ok = false;
                copy_strip<4, LS>(xbuf, hmap + J.rings[P.ri].start, S, P, t, NTW);
                slot_sync(slot);
            }
            if (!ok && !*abort_flag) {
                *abort_flag = 1;
                sk_record_error(A.status, SK_ETIMEOUT);
            }
            int before, cnt;
            win_shape(P, before, cnt);
            const int ngroups = sk_capw_steps(cnt, P.n_i, R.n) >> 2;
            prefetch_to(s0 + PF_STEPS + 4 * ngroups);
            if (ok && act) {
                const int pA = centre_of(jt, R.n, R.s, P, mg, sh) - centre_of(j0, R.n, R.s, P, mg, sh);
                const int o0 = S.L - 1 - pA;          // natural position of the union's first pixel, reflected
                // shared addresses of union position q (segment 0) and of its reflection (segment 2);
                // segments 1 and 3 follow LS float4 later; a group of four positions is one float4 on
                const uint32_t xb = tc::smem_u32(xbuf);
                uint32_t af[4], ar[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    af[q] = xb + 16u * (uint32_t)split_index<4, LS>(pA + q);
                    ar[q] = xb + 16u * (uint32_t)(2 * LS + split_index<4, LS>(o0 - q));
                }
#pragma unroll 1
                for (int i = 0; i < ngroups; ++i) {
                    float4 wn[4];
                    const float4 *wq = wp + (s0 + 4) * NTW;     // the next group (the stream is padded)
#pragma unroll
                    for (int q = 0; q < 4; ++q) wn[q] = ld_stream(wq + q * NTW, pol_w);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 a = lds4(af[q]), b4 = lds4(af[q] + 16u * LS);
                        const float4 c = lds4(ar[q]), d = lds4(ar[q] + 16u * LS);
                        mac16x4(acc, wc[q], a, b4, c, d);
                        af[q] += 16u;
                        ar[q] -= 16u;
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) wc[q] = wn[q];
                    s0 += 4;
                }
                if constexpr (BLK) {
                    // the ring's sums into the running totals
#pragma unroll
                    for (int k = 0; k < OPT; ++k)
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int i = 2 * (8 * k + e);
                            tot[i * NTH] += acc[k][e].x;
                            tot[(i + 1) * NTH] += acc[k][e].y;
                            acc[k][e] = make_float2(0.0f, 0.0f);
                        }
                }
            } else {
                s0 += 4 * ngroups;
            }
        }
        if (NB == 1) {
            // the next item stages into this slot's one buffer: everyone must be done reading it
            slot_sync(slot);
            if (t == 0) s_item[slot] = *abort_flag ? A.total : atomicAdd(A.queue, 1);
        }
        if (*abort_flag) continue;
        float *yn = J.y + (long long)map * J.stride + R.start;
        float *ys = J.y + (long long)map * J.stride + J.rings[ro_s].start;
        if constexpr (BLK) {
#pragma unroll
            for (int k = 0; k < OPT; ++k)
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int i = 2 * (8 * k + e);
                    acc[k][e] = make_float2(tot[i * NTH], tot[(i + 1) * NTH]);
                }
        }
#pragma unroll
        for (int k = 0; k < OPT; ++k) {
            const int j = jt + k;
            if (j < T) {
                const int jr = Qo - j - R.s;            // reflection in the quarter
                store16(yn, ys, j, jr, jr < Qo && jr >= T, Qo, acc[k]);
            }
        }
    }
    // after an abort: wait (bounded) for the copies this warp issued that are still in flight
    if (pend) {
        for (int b = 0; b < NB; ++b)
            if ((pend >> b) & 1) tc::mbar_wait(full0 + 8 * b, (fphase >> b) & 1, WAIT_NS);
    }
}

// ---------------------------------------------------------------------------
// Weight builder: the stream of every item of a.j[0] (one kernel's cap items), the
// weights computed exactly as the evaluating kernel computes them -- fast_weight2 on
// narrow windows (MODE & 1), fast_weight otherwise, from the same shared node table,
// with the same exact-integer q -- and 0 outside each output's own window.
// ---------------------------------------------------------------------------
template <int MODE, typename TabT>
__global__ void __launch_bounds__(256)
k_capw_build(const __grid_constant__ JobsArg A, float4 *__restrict__ W, const int *gate) {
    constexpr bool SERIES = (MODE & 1) != 0, SMALLA = (MODE & 2) != 0, BIASED = (MODE & 4) != 0;
    if (gate && !*gate) return;                  // table unchanged: the weights stand
    extern __shared__ __align__(16) unsigned char smraw[];
    TabT *stab = reinterpret_cast<TabT *>(smraw);
    const JobDesc &J = A.j[0];
    const int ntab = J.kp.nt;
    for (int k = threadIdx.x; k < ntab + 2; k += blockDim.x) {
        if constexpr (sizeof(TabT) == sizeof(float2)) {
            float2 e = make_float2(0.0f, 0.0f);
            if (k < ntab - 1) {
                e = J.tab[k];
                e.x = fmaf(0.5f, e.y, e.x);
            }
            stab[k] = e;
        } else if (k < ntab) {
            stab[k] = J.tab[k].x;
        }
    }
    __syncthreads();
    const auto tabv = [&]() {
        if constexpr (sizeof(TabT) == sizeof(float2)) return SmemTab2{tc::smem_u32(stab)};
        else return static_cast<const float *>(stab);
    }();
    const int per_block = blockDim.x / NTW;
    const int t = threadIdx.x % NTW;
    for (int f = blockIdx.x * per_block + threadIdx.x / NTW; f < J.n_items; f += gridDim.x * per_block) {
        const int4 it = J.items[f];
        const int ro = it.x, j0 = it.y;
        const unsigned mg = (unsigned)it.z;
        const int sh = it.w;
        const RingDev R = J.rings[ro];
        const int T = base_count(R.n >> 2, R.s);
        const int jt = j0 + OPT * t;
        if (jt >= T) continue;                       // no outputs: the thread's rows stay unread
        const longlong2 wr = J.capw_ring[ro];
        float4 *wp = W + wr.x + (long long)(j0 / CT) * wr.y * NTW + t;
        long long s0 = 0;
        for (int p = J.pair_off[ro]; p < J.pair_off[ro + 1]; ++p) {
            const PairInfo P = J.pairs[p];
            int before, cnt;
            win_shape(P, before, cnt);
            const int NS = sk_capw_steps(cnt, P.n_i, R.n);
            const float Ae = fmaxf(P.A, 1e-30f);    // as the evaluating kernel: t >= 1e-30
            const int ct = centre_of(jt, R.n, R.s, P, mg, sh);
            int lo[OPT];                             // own window of output k in union positions
#pragma unroll
            for (int k = 0; k < OPT; ++k) lo[k] = centre_of(jt + k, R.n, R.s, P, mg, sh) - ct;
            for (int m = 0; m < NS; ++m) {
                float w[OPT];
                float xk[OPT];
#pragma unroll
                for (int k = 0; k < OPT; ++k)
                    xk[k] = (float)q_of(ct - before + m, jt + k, R.n, R.s, P) * P.c0;
                if (SERIES) {
                    const float2 w01 = fast_weight2<SMALLA, BIASED>(make_float2(xk[0], xk[1]), Ae, P.B, J.kp, tabv);
                    const float2 w23 = fast_weight2<SMALLA, BIASED>(make_float2(xk[2], xk[3]), Ae, P.B, J.kp, tabv);
                    w[0] = w01.x; w[1] = w01.y; w[2] = w23.x; w[3] = w23.y;
                } else {
#pragma unroll
                    for (int k = 0; k < OPT; ++k) w[k] = fast_weight<false, SMALLA, BIASED>(xk[k], Ae, P.B, J.kp, tabv);
                }
#pragma unroll
                for (int k = 0; k < OPT; ++k)
                    if (jt + k >= T || m < lo[k] || m >= lo[k] + cnt) w[k] = 0.0f;
                wp[(s0 + m) * NTW] = make_float4(w[0], w[1], w[2], w[3]);
            }
            s0 += NS;
        }
    }
}

// The same stream evaluated in FP64 (pair_weight64: FP64 chord from the pair's FP64
// (A, B), node coordinate and interpolation of the FP64 node values, one rounding to
// FP32), for operators with wide windows, whose outputs sum thousands of weights: there
// the FP32 evaluation's table-coordinate error (u up to the node count, one FP32 ulp)
// would otherwise reach 1e-6 of the result.  Same layout and window rules as k_capw_build.
__global__ void __launch_bounds__(256)
k_capw_build64(const __grid_constant__ JobsArg A, float4 *__restrict__ W, const int *gate) {
    if (gate && !*gate) return;                  // table unchanged: the weights stand
    const JobDesc &J = A.j[0];
    const int per_block = blockDim.x / NTW;
    const int t = threadIdx.x % NTW;
    for (int f = blockIdx.x * per_block + threadIdx.x / NTW; f < J.n_items; f += gridDim.x * per_block) {
        const int4 it = J.items[f];
        const int ro = it.x, j0 = it.y;
        const unsigned mg = (unsigned)it.z;
        const int sh = it.w;
        const RingDev R = J.rings[ro];
        const int T = base_count(R.n >> 2, R.s);
        const int jt = j0 + OPT * t;
        if (jt >= T) continue;                       // no outputs: the thread's rows stay unread
        const longlong2 wr = J.capw_ring[ro];
        float4 *wp = W + wr.x + (long long)(j0 / CT) * wr.y * NTW + t;
        long long s0 = 0;
        for (int p = J.pair_off[ro]; p < J.pair_off[ro + 1]; ++p) {
            const PairInfo P = J.pairs[p];
            const double2 ab = J.ab64[p];
            const double c0 = SK_PI / (2.0 * (double)R.n * (double)P.n_i);
            int before, cnt;
            win_shape(P, before, cnt);
            const int NS = sk_capw_steps(cnt, P.n_i, R.n);
            const int ct = centre_of(jt, R.n, R.s, P, mg, sh);
            int lo[OPT];                             // own window of output k in union positions
#pragma unroll
            for (int k = 0; k < OPT; ++k) lo[k] = centre_of(jt + k, R.n, R.s, P, mg, sh) - ct;
            for (int m = 0; m < NS; ++m) {
                float w[OPT];
#pragma unroll
                for (int k = 0; k < OPT; ++k) {
                    w[k] = 0.0f;
                    if (jt + k < T && m >= lo[k] && m < lo[k] + cnt) {
                        const double x = (double)q_of(ct - before + m, jt + k, R.n, R.s, P) * c0;
                        w[k] = pair_weight64(x, ab.x, ab.y, J.kp, J.kd, J.V64, J.dOmega);
                    }
                }
                wp[(s0 + m) * NTW] = make_float4(w[0], w[1], w[2], w[3]);
            }
            s0 += NS;
        }
    }
}

template <int LS, bool BLK>
cudaError_t launch_conv(const JobsArg &a, int grid, cudaStream_t st) {
    constexpr int NB = capw_bufs<LS, BLK>(), SLOTS = capw_slots<LS, BLK>();
    const size_t smem = capw_strip_bytes(LS, NB, SLOTS) + capw_bar_bytes(NB, SLOTS) + capw_tot_bytes(BLK, SLOTS);
    cudaError_t e = cudaFuncSetAttribute(k_conv_capw<LS, BLK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_conv_capw<LS, BLK><<<grid, NTW * SLOTS, smem, st>>>(a);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_build_m(const JobsArg &a, float4 *w, int grid, cudaStream_t st, const int *gate) {
    const int nt = a.j[0].kp.nt;
    if (nt <= PAIR_TABLE_NODES) {
        const size_t smem = (size_t)(nt + 2) * sizeof(float2);
        cudaError_t e = cudaFuncSetAttribute(k_capw_build<MODE, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        k_capw_build<MODE, float2><<<grid, 256, smem, st>>>(a, w, gate);
    } else {
        const size_t smem = (size_t)(nt + 2) * sizeof(float);
        cudaError_t e = cudaFuncSetAttribute(k_capw_build<MODE, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        k_capw_build<MODE, float><<<grid, 256, smem, st>>>(a, w, gate);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t sk_launch_conv_capw(const JobsArg &a, int ls, bool blocked, int grid, cudaStream_t st) {
    if (a.total <= 0) return cudaSuccess;
    switch (ls) {
        case SK_CAP_LS[0]:
            return blocked ? launch_conv<SK_CAP_LS[0], true>(a, grid, st) : launch_conv<SK_CAP_LS[0], false>(a, grid, st);
        case SK_CAP_LS[1]:
            return blocked ? launch_conv<SK_CAP_LS[1], true>(a, grid, st) : launch_conv<SK_CAP_LS[1], false>(a, grid, st);
        case SK_CAP_LS[2]:
            return blocked ? launch_conv<SK_CAP_LS[2], true>(a, grid, st) : launch_conv<SK_CAP_LS[2], false>(a, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

int sk_capw_items_per_block(int ls, bool blocked) { return ls <= 288 ? 6 : (ls <= 640 && blocked ? 3 : 2); }

cudaError_t sk_launch_capw_build64(const JobsArg &a, float4 *w, int grid, cudaStream_t st, const int *gate) {
    if (a.j[0].n_items <= 0) return cudaSuccess;
    k_capw_build64<<<grid, 256, 0, st>>>(a, w, gate);
    return cudaGetLastError();
}

cudaError_t sk_launch_capw_build(const JobsArg &a, int mode, float4 *w, int grid, cudaStream_t st,
                                 const int *gate) {
    if (a.j[0].n_items <= 0) return cudaSuccess;
    switch (mode) {
        case 0: return launch_build_m<0>(a, w, grid, st, gate);
        case 1: return launch_build_m<1>(a, w, grid, st, gate);
        case 2: return launch_build_m<2>(a, w, grid, st, gate);
        case 3: return launch_build_m<3>(a, w, grid, st, gate);
        case 4: return launch_build_m<4>(a, w, grid, st, gate);
        case 5: return launch_build_m<5>(a, w, grid, st, gate);
        case 6: return launch_build_m<6>(a, w, grid, st, gate);
        case 7: return launch_build_m<7>(a, w, grid, st, gate);
        default: return cudaErrorInvalidValue;
    }
}
