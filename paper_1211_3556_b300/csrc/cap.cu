// cap.cu -- polar-cap path: one weight evaluation shared by up to 16 symmetric pairs.
//
// The HEALPix pixelisation is invariant under
//   * a quarter turn in phi (pixel j -> j + n/4 on every ring),
//   * the reflection phi -> pi/2 - phi (pixel j -> n/4 - j - s on a ring whose
//     pixels sit at phi = pi (2j + s) / n),
//   * the mirror about the equator (ring r <-> ring 4N - r, same phis),
// and the angle between two pixel centres is invariant under all three.  So a
// pair (o, i) and its images have the same weight dOmega K_lin(gamma).  A
// thread owns one "base" output of the first half quarter of a northern ring,
// evaluates the weight of each window pair once (the per-pair formula:
// chord from A + B sin^2(dphi/2), asin series, table lerp), and applies it to
// the 16 images: 4 quarter turns x 2 hemispheres x {pair, reflected pair}.
// Outputs on a symmetry axis (phi = 0 or pi/4) are their own reflections (or
// a quarter turn of it): they keep the 8 images without reflection, so no
// output is written twice.  Same operator as the per-pair path (Sec. 2, Eq. 1
// with the tabulated kernel of Sec. 3); only the order of work differs.
//
// Symmetric copy of the input (k_cap_sym, once per call): for every ring r the
// caps read, H_r[a] = (x_r[a], x_r[a + n/2], x_m[a], x_m[a + n/2]) with m the
// mirror ring, stored even pixels first, then odd ones.  One float4 of H holds a
// pixel, its half turn and both mirrors, so the 16 images of a window pixel a
// (base frame) are four float4: H[a], H[a + n/4] (the other two quarter turns),
// H[b], H[b + n/4] with b = n/4 - s - a its reflection.
//
// Work item: (northern output ring, first base pixel) for CT base outputs,
// CT / 2 threads, each owning two adjacent base outputs jA, jB = jA + 1; a
// block runs four work items side by side (two for the largest strip class),
// each in its own slot with its own named barrier, so that they share one copy
// of the node table.  For every input
// ring of the window a work item stages four segments of H covering the union of its
// CT windows -- the window pixels from a0 and from a0 + n/4, their reflections
// from b0 and b0 + n/4 (read backwards) -- with 1-D bulk copies (TMA) issued by
// eight lanes of one of its warps (the four take turns): each segment splits
// into an even and an odd
// part, contiguous in H up to one wrap past phi = 2 pi.  Two buffers per item:
// ring p + 1 is copied while ring p is summed (an mbarrier per buffer counts its
// bytes; one named barrier per ring frees the buffer of ring p - 1).  Rings whose
// strip wraps the whole ring (a few near the poles) are copied by all threads.
// A thread walks the union of its two windows (they start at most a pixel or two
// apart): four 128-bit loads feed the 16 images of both outputs, and both
// weights come from one paired evaluation (fma.rn.f32x2: two IEEE
// operations).  Because lanes two pixels apart read consecutive float4 of one
// parity, a warp's loads hit distinct banks.  The node values V_k dOmega sit in
// shared memory (FP32, the slope formed on the fly): the lanes of a warp look up
// nodes spread over a few hundred entries, a gather that costs a few bank
// wavefronts from shared memory but one L1 wavefront per distinct line from
// global memory.
#include "skconv.h"
#include "cap_common.cuh"

namespace {

using capc::CT;
using capc::WAIT_NS;
using capc::base_count;
using capc::centre_of;
using capc::q_of;
using capc::seg_start;
using capc::store16;
using capc::strip_wait;
using capc::win_shape;
using capc::Strip;
constexpr int NTH = CT / 2;         // threads per work item: two adjacent base outputs each
static_assert(NTH == 128, "an item's strips are issued by its four warps in turn");
// work items in flight per block (they share one node table): four where their strips fit
template <int LS>
__host__ __device__ constexpr int cap_slots() { return LS <= 640 ? 4 : 2; }
__host__ __device__ constexpr int cap_max_slots() { return 4; }
// node tables of up to this many nodes are held as (value, slope) pairs, larger ones as values
constexpr int PAIR_TABLE_NODES = 8192;
// strip buffers per work item: two (stage ring p + 1 while ring p is summed) where they fit
template <int LS>
__host__ __device__ constexpr int cap_bufs() { return LS <= 320 ? 2 : 1; }
// dynamic shared memory: strips [slots][NB][4][LS] float4, then one mbarrier per
// strip buffer and the abort flag (16-byte multiple), then the node table
__host__ __device__ constexpr size_t cap_strip_bytes(int ls, int nb, int slots) { return (size_t)slots * nb * 4 * ls * 16; }
__host__ __device__ constexpr size_t cap_bar_bytes(int nb, int slots) { return ((size_t)slots * nb * 8 + 4 + 15) / 16 * 16; }

__device__ __forceinline__ void slot_sync(int slot) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + slot), "r"(NTH) : "memory");
}
// Buffer hand-over of a two-buffer item: at the top of ring p every warp is done with
// ring p - 1; the warp that stages ring p + 1 (into ring p - 1's buffer) waits for the
// other three (bar.sync), which only signal (bar.arrive) and go on.  Two barriers per
// slot, by the parity of p: a warp can run at most one ring ahead of the slowest (it
// needs ring p + 1's strip, staged only after everyone finished ring p - 1), so it
// never arrives twice in one phase.
__device__ __forceinline__ void ring_handover(int slot, int parity, bool stager) {
    const int id = 1 + cap_max_slots() + 2 * slot + parity;
    if (stager) asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(NTH) : "memory");
    else asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(NTH) : "memory");
}

// Strip layout of one segment: even positions first, then odd ones.  A lane owns
// two adjacent outputs, so at one step the lanes of a warp read positions about
// two apart; with this layout they read consecutive float4 (one parity) instead
// of every other one.
template <int LS>
__device__ __forceinline__ int split_index(int m) { return capc::split_index<2, LS>(m); }

// The strip of input ring P for the item's outputs j0 .. jlast: L window
// positions from pixel u0 (base frame); the segments start at the natural pixels
// seg_start(0..3).
__device__ __forceinline__ Strip strip_of(const PairInfo &P, int j0, int jlast, int n_o, int s_o, unsigned mg, int sh) {
    int before, cnt;
    win_shape(P, before, cnt);
    const int c0 = centre_of(j0, n_o, s_o, P, mg, sh), c1 = centre_of(jlast, n_o, s_o, P, mg, sh);
    return Strip{c1 - c0 + cnt, c0 - before};
}
// Bulk copies (strips shorter than the ring) and plain copies (strips that wrap it)
// of ring P's strip in the parity layout.
template <int LS>
__device__ __forceinline__ void issue_strip(float4 *buf, uint32_t bar, const float4 *hrow, const Strip &S,
                                            const PairInfo &P, int lane) {
    capc::issue_strip<2, LS>(buf, bar, hrow, S, P, lane);
}
template <int LS>
__device__ __forceinline__ void copy_strip(float4 *buf, const float4 *hrow, const Strip &S, const PairInfo &P, int t) {
    capc::copy_strip<2, LS>(buf, hrow, S, P, t, NTH);
}

// The 16 images of staged position m (forward segments at xf[i], xf[LS + i],
// reflected ones at xr[-i], xr[LS - i]): acc[0..3] = (north, its half turn),
// (south, its half turn) for quarter turns 0 and 1; acc[4..7] the same for the
// reflected pair.
template <int LS>
__device__ __forceinline__ void mac16(float2 *acc, float w, const float4 *xf, const float4 *xr, int i) {
    const float2 ww = f2(w);
    const float4 a = xf[i], b = xf[LS + i], c = xr[-i], d = xr[LS - i];
    acc[0] = __ffma2_rn(ww, make_float2(a.x, a.y), acc[0]);
    acc[1] = __ffma2_rn(ww, make_float2(a.z, a.w), acc[1]);
    acc[2] = __ffma2_rn(ww, make_float2(b.x, b.y), acc[2]);
    acc[3] = __ffma2_rn(ww, make_float2(b.z, b.w), acc[3]);
    acc[4] = __ffma2_rn(ww, make_float2(c.x, c.y), acc[4]);
    acc[5] = __ffma2_rn(ww, make_float2(c.z, c.w), acc[5]);
    acc[6] = __ffma2_rn(ww, make_float2(d.x, d.y), acc[6]);
    acc[7] = __ffma2_rn(ww, make_float2(d.z, d.w), acc[7]);
}

// H rows of rings [r0, r0 + gridDim.x) of every map of job J (grid: rings x map slices),
// pixels split by residue modulo SPLIT: row position i holds pixel
// a = SPLIT (i mod n/SPLIT) + floor(i / (n/SPLIT)).
template <int SPLIT>
__global__ void k_cap_sym(const JobDesc J, int r0) {
    const int r = r0 + blockIdx.x;
    const RingDev R = J.rings[r];
    const int n = R.n, h = n >> 1, w = n / SPLIT;
    const long long mstart = J.rings[J.nr - 1 - r].start;
    for (int map = blockIdx.y; map < J.batch; map += gridDim.y) {
        const float *xr = J.x + (long long)map * J.stride + R.start;
        const float *xm = J.x + (long long)map * J.stride + mstart;
        float4 *out = J.hx + (long long)map * J.hstride + R.start;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int e = i / w;
            const int a = SPLIT * (i - e * w) + e;
            const int a2 = a + h < n ? a + h : a + h - n;
            out[i] = make_float4(xr[a], xr[a2], xm[a], xm[a2]);
        }
    }
}

template <int LS, int MODE, typename TabT>
__global__ void __launch_bounds__(NTH * cap_slots<LS>())
k_conv_cap(const __grid_constant__ JobsArg A) {
    constexpr bool SERIES = (MODE & 1) != 0, SMALLA = (MODE & 2) != 0, BIASED = (MODE & 4) != 0;
    constexpr int NB = cap_bufs<LS>(), SLOTS = cap_slots<LS>();
    extern __shared__ __align__(16) float4 sx[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<char *>(sx) + cap_strip_bytes(LS, NB, SLOTS));
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + SLOTS * NB);
    // one node table per launch (every job of a launch uses the same kernel table):
    // (value, slope) pairs, or the values alone
    TabT *stab = reinterpret_cast<TabT *>(reinterpret_cast<char *>(bars) + cap_bar_bytes(NB, SLOTS));
    if (threadIdx.x == 0) {
        for (int b = 0; b < SLOTS * NB; ++b) tc::mbar_init(tc::smem_u32(bars + b), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // a (value, slope) table becomes (midpoint, slope), M_k = V_k + S_k / 2, and is
    // padded: entries nt - 1 .. nt + 1 hold (0, 0), so that pairs beyond the cut read
    // weight 0 (fast_weight with SmemTab2)
    const int ntab = A.j[0].kp.nt;
    for (int k = threadIdx.x; k < ntab + 2; k += NTH * SLOTS) {
        if constexpr (sizeof(TabT) == sizeof(float2)) {
            float2 e = make_float2(0.0f, 0.0f);
            if (k < ntab - 1) {
                e = A.j[0].tab[k];
                e.x = fmaf(0.5f, e.y, e.x);
            }
            stab[k] = e;
        } else if (k < ntab) {
            stab[k] = A.j[0].tab[k].x;
        }
    }
    __syncthreads();
    // the weight lookups read the table by its shared address (SmemTab2) where it holds pairs
    const auto tabv = [&]() {
        if constexpr (sizeof(TabT) == sizeof(float2)) return SmemTab2{tc::smem_u32(stab)};
        else return static_cast<const float *>(stab);
    }();
    const int slot = threadIdx.x / NTH, t = threadIdx.x % NTH;
    float4 *const sbuf = sx + slot * NB * 4 * LS;
    const uint32_t bar0 = tc::smem_u32(bars + slot * NB);
    uint32_t phase = 0;     // bit b: parity of the next phase of buffer b (the same in every thread)
    uint32_t pend = 0;      // bit b set while a copy this thread's warp issued into buffer b is not waited for
    // work queue: each slot takes the next item (items are ordered heaviest first), so the
    // slots that drew light items take more of them and all finish together
    // With two buffers the warp that stages after an item's last ring also takes the
    // slot's next item from the queue (one ring before it is needed, so the queue's
    // balance is kept) and stages that item's first strip into the free buffer: the item
    // boundary then waits neither for the queue atomic nor for a first copy.  The buffer
    // of an item's first ring (bbase) follows on from the previous item's last ring.
    __shared__ int s_item[SLOTS];
    __shared__ int s_pref[SLOTS];       // 1: the item's first strip is staged already
    if (t == 0) {
        s_item[slot] = atomicAdd(A.queue, 1);
        s_pref[slot] = 0;
    }
    int bbase = 0;
    for (;;) {
        slot_sync(slot);
        const int f = s_item[slot];
        const bool pref = NB == 2 && s_pref[slot] != 0;
        if (f >= A.total) break;
        const JobDesc &J = A.j[sk_find_job(A, f)];
        const int local = f - J.flat_base;
        const int map = local / J.n_items;
        const int4 it = J.items[local - map * J.n_items];
        const int ro = it.x, j0 = it.y;
        const unsigned mg = (unsigned)it.z;            // division by 2 n_o (centre_of)
        const int sh = it.w;
        const RingDev R = J.rings[ro];
        const int Qo = R.n >> 2;
        const int T = base_count(Qo, R.s);
        const int jlast = min(j0 + CT - 1, T - 1);
        const int jA = j0 + 2 * t, jB = jA + 1;
        const bool actA = jA < T, actB = jB < T;
        const int jrA = Qo - jA - R.s, jrB = Qo - jB - R.s;   // reflections in the quarter
        const bool reflA = actA && jrA < Qo && jrA >= T;
        const bool reflB = actB && jrB < Qo && jrB >= T;
        const int ro_s = J.nr - 1 - ro;
        const float4 *hmap = J.hx + (long long)map * J.hstride;
        const int p0 = J.pair_off[ro], p1 = J.pair_off[ro + 1];

        float2 accA[8], accB[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) { accA[s] = make_float2(0.0f, 0.0f); accB[s] = make_float2(0.0f, 0.0f); }
        // wide windows (A.ctot): each ring's sums go into the thread's running totals in a
        // private slice of global scratch (L2-resident; the registers and shared memory are
        // full), so that the FP32 rounding grows with the terms of one ring and the number of
        // rings, not with their product
        const long long ntot = (long long)gridDim.x * blockDim.x;
        float *const tt = A.ctot ? A.ctot + (long long)blockIdx.x * blockDim.x + threadIdx.x : nullptr;
        if (tt) {
#pragma unroll
            for (int i = 0; i < 32; ++i) tt[i * ntot] = 0.0f;
        }

        // ring p's strip into buffer b by bulk copies, unless it wraps; the item's warps
        // take turns (ring p by warp (p - p0) mod 4), and the issuing warp takes lane 0's
        // view of the abort flag
        auto issue = [&](int p, int b) {
            if (((p - p0) & 3) != (t >> 5)) return;
            const PairInfo Pn = J.pairs[p];
            const Strip S = strip_of(Pn, j0, jlast, R.n, R.s, mg, sh);
            const int stop = __shfl_sync(0xffffffffu, *abort_flag, 0);
            if (S.L < Pn.n_i && !stop) {
                issue_strip<LS>(sbuf + b * 4 * LS, bar0 + 8 * b, hmap + J.rings[Pn.ri].start, S, Pn, t & 31);
                pend |= 1u << b;
            }
        };
        // the first strip of item fn into buffer b, by the calling warp (bulk copies; a strip
        // that wraps its ring is copied by the item itself); returns whether it was staged
        auto stage_first = [&](int fn, int b) -> int {
            const JobDesc &Jn = A.j[sk_find_job(A, fn)];
            const int ln = fn - Jn.flat_base;
            const int mn = ln / Jn.n_items;
            const int4 itn = Jn.items[ln - mn * Jn.n_items];
            const RingDev Rn = Jn.rings[itn.x];
            const int jln = min(itn.y + CT - 1, base_count(Rn.n >> 2, Rn.s) - 1);
            const PairInfo Pn = Jn.pairs[Jn.pair_off[itn.x]];
            const Strip Sn = strip_of(Pn, itn.y, jln, Rn.n, Rn.s, (unsigned)itn.z, itn.w);
            const int stop = __shfl_sync(0xffffffffu, *abort_flag, 0);
            if (Sn.L < Pn.n_i && !stop) {
                const float4 *hn = Jn.hx + (long long)mn * Jn.hstride;
                issue_strip<LS>(sbuf + b * 4 * LS, bar0 + 8 * b, hn + Jn.rings[Pn.ri].start, Sn, Pn, t & 31);
                pend |= 1u << b;
                return 1;
            }
            return 0;
        };
        if (NB == 2 && !pref && p0 < p1) issue(p0, bbase);
        for (int p = p0; p < p1; ++p) {
            const int b = NB == 2 ? (((p - p0) + bbase) & 1) : 0;
            float4 *const xbuf = sbuf + b * 4 * LS;
            const PairInfo P = J.pairs[p];
            const Strip S = strip_of(P, j0, jlast, R.n, R.s, mg, sh);
            const bool bulk = S.L < P.n_i;
            // every thread is done with ring p - 1: its buffer takes ring p + 1 (two
            // buffers) or ring p (one)
            if (NB == 2) {
                const bool stager = ((p + 1 - p0) & 3) == (t >> 5);
                ring_handover(slot, (p - p0) & 1, stager);
                if (p + 1 < p1) {
                    issue(p + 1, b ^ 1);
                } else if (stager) {
                    int fn = 0;
                    if ((t & 31) == 0) fn = *abort_flag ? A.total : atomicAdd(A.queue, 1);
                    fn = __shfl_sync(0xffffffffu, fn, 0);
                    const int staged = fn < A.total ? stage_first(fn, b ^ 1) : 0;
                    if ((t & 31) == 0) {
                        s_item[slot] = fn;          // read after the slot barrier that opens the next item
                        s_pref[slot] = staged;
                    }
                }
            } else {
                slot_sync(slot);
                if (bulk) issue(p, 0);
            }
            bool ok = true;
            if (bulk) {
                if (strip_wait(bar0 + 8 * b, (phase >> b) & 1, abort_flag)) {
                    pend &= ~(1u << b);
                } else {
                    ok = false;
                    if (!*abort_flag) {
                        *abort_flag = 1;
                        sk_record_error(A.status, SK_ETIMEOUT);
                    }
                }
                phase ^= 1u << b;
            } else {
                // buffer b held ring p - 2, which a slow warp may still read (two buffers)
                if (NB == 2) slot_sync(slot);
                copy_strip<LS>(xbuf, hmap + J.rings[P.ri].start, S, P, t);
                slot_sync(slot);
            }
            if (ok && actA) {
                int before, cnt;
                win_shape(P, before, cnt);
                const int cb = centre_of(j0, R.n, R.s, P, mg, sh);
                const int cA = centre_of(jA, R.n, R.s, P, mg, sh);
                const int dl = actB ? centre_of(jB, R.n, R.s, P, mg, sh) - cA : 0;   // 0, 1 or 2
                const int cnt_u = cnt + dl;             // union of the two windows, from A's start
                // |q| < 2^24 on these windows (checked when the plan was built): exact in FP32
                const float qA0 = (float)q_of(cA - before, jA, R.n, R.s, P);
                const float dqo = (float)(2 * R.n);     // q step per input pixel
                const float dqi = (float)(2 * P.n_i);   // q of output jA minus q of output jB
                const int pA = cA - cb;                 // strip position of the union's first pixel
                const int o0 = S.L - 1 - pA;            // its natural position in the reflected segments
                const float Ae = fmaxf(P.A, 1e-30f);    // t >= 1e-30: a normal number for rsqrt
                const float4 *xr0 = xbuf + 2 * LS;
                if (SERIES) {
                    // narrow windows only: a pixel of the union outside one output's window is
                    // outside its cut, and the cut test gives it weight 0.  Pixels go in pairs
                    // (pA + m, pA + m + 1): one of each parity, i = m / 2.
                    const float4 *x0 = xbuf + split_index<LS>(pA), *x1 = xbuf + split_index<LS>(pA + 1);
                    const float4 *r0 = xr0 + split_index<LS>(o0), *r1 = xr0 + split_index<LS>(o0 - 1);
                    float2 q = make_float2(qA0, qA0 - dqi);   // q of pixel m for outputs (A, B)
                    int m = 0;
                    if (cnt_u >= 2) {
                        // weights one pixel pair ahead of the sums that use them
                        float2 w0 = fast_weight2<SMALLA, BIASED>(__fmul2_rn(q, f2(P.c0)), Ae, P.B, J.kp, tabv);
                        float2 w1 = fast_weight2<SMALLA, BIASED>(__fmul2_rn(__fadd2_rn(q, f2(dqo)), f2(P.c0)), Ae, P.B, J.kp, tabv);
                        q = __fadd2_rn(q, f2(2.0f * dqo));
#pragma unroll 1
                        for (; m + 3 < cnt_u; m += 2) {
                            const int i = m >> 1;
                            const float2 q1 = __fadd2_rn(q, f2(dqo));
                            const float2 v0 = fast_weight2<SMALLA, BIASED>(__fmul2_rn(q, f2(P.c0)), Ae, P.B, J.kp, tabv);
                            const float2 v1 = fast_weight2<SMALLA, BIASED>(__fmul2_rn(q1, f2(P.c0)), Ae, P.B, J.kp, tabv);
                            q = __fadd2_rn(q1, f2(dqo));
                            mac16<LS>(accA, w0.x, x0, r0, i);
                            mac16<LS>(accB, w0.y, x0, r0, i);
                            mac16<LS>(accA, w1.x, x1, r1, i);
                            mac16<LS>(accB, w1.y, x1, r1, i);
                            w0 = v0;
                            w1 = v1;
                        }
                        const int i = m >> 1;
                        mac16<LS>(accA, w0.x, x0, r0, i);
                        mac16<LS>(accB, w0.y, x0, r0, i);
                        mac16<LS>(accA, w1.x, x1, r1, i);
                        mac16<LS>(accB, w1.y, x1, r1, i);
                        m += 2;
                    }
                    if (m < cnt_u) {                           // an odd count: the last pixel alone
                        const int i = m >> 1;
                        const float2 w0 = fast_weight2<SMALLA, BIASED>(__fmul2_rn(q, f2(P.c0)), Ae, P.B, J.kp, tabv);
                        mac16<LS>(accA, w0.x, x0, r0, i);
                        mac16<LS>(accB, w0.y, x0, r0, i);
                    }
                } else {
                    // windows may be whole rings: restrict each output to its own window
                    for (int m = 0; m < cnt_u; ++m) {
                        const float qa = fmaf((float)m, dqo, qA0);
                        float wa = fast_weight<SERIES, SMALLA, BIASED>(qa * P.c0, Ae, P.B, J.kp, tabv);
                        float wb = fast_weight<SERIES, SMALLA, BIASED>((qa - dqi) * P.c0, Ae, P.B, J.kp, tabv);
                        wa = m < cnt ? wa : 0.0f;
                        wb = m >= dl ? wb : 0.0f;
                        const float4 *xm = xbuf + split_index<LS>(pA + m);
                        const float4 *rm = xr0 + split_index<LS>(o0 - m);
                        mac16<LS>(accA, wa, xm, rm, 0);
                        mac16<LS>(accB, wb, xm, rm, 0);
                    }
                }
                if (tt) {
#pragma unroll
                    for (int s = 0; s < 8; ++s) {
                        tt[(4 * s) * ntot] += accA[s].x;
                        tt[(4 * s + 1) * ntot] += accA[s].y;
                        tt[(4 * s + 2) * ntot] += accB[s].x;
                        tt[(4 * s + 3) * ntot] += accB[s].y;
                        accA[s] = make_float2(0.0f, 0.0f);
                        accB[s] = make_float2(0.0f, 0.0f);
                    }
                }
            }
        }
        if (NB == 2) {
            bbase = ((p1 - p0) + bbase) & 1;        // the buffer the next item's first strip went to
        } else {
            // the next item stages into this slot's one buffer: everyone must be done reading it
            slot_sync(slot);
            if (t == 0) s_item[slot] = *abort_flag ? A.total : atomicAdd(A.queue, 1);
        }
        if (*abort_flag) continue;
        float *yn = J.y + (long long)map * J.stride + R.start;
        float *ys = J.y + (long long)map * J.stride + J.rings[ro_s].start;
        if (tt) {
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                accA[s] = make_float2(tt[(4 * s) * ntot], tt[(4 * s + 1) * ntot]);
                accB[s] = make_float2(tt[(4 * s + 2) * ntot], tt[(4 * s + 3) * ntot]);
            }
        }
        if (actA) store16(yn, ys, jA, jrA, reflA, Qo, accA);
        if (actB) store16(yn, ys, jB, jrB, reflB, Qo, accB);
    }
    // after an abort: wait (bounded) for the copies this warp issued that are still in flight
    if (pend) {
        for (int b = 0; b < NB; ++b)
            if ((pend >> b) & 1) tc::mbar_wait(bar0 + 8 * b, (phase >> b) & 1, WAIT_NS);
    }
}

size_t cap_smem(int LS, int nt, bool pairs) {
    const int nb = LS <= 320 ? 2 : 1, slots = LS <= 640 ? 4 : 2;     // cap_bufs, cap_slots
    return cap_strip_bytes(LS, nb, slots) + cap_bar_bytes(nb, slots) + (pairs ? (size_t)(nt + 2) * 8 : (size_t)nt * 4);
}

int max_nt(const JobsArg &a) {
    int m = 2;
    for (int j = 0; j < a.n_jobs; ++j) m = a.j[j].kp.nt > m ? a.j[j].kp.nt : m;
    return m;
}

template <int LS, int MODE, typename TabT>
cudaError_t launch_t(const JobsArg &a, int nt, int grid, cudaStream_t st) {
    const size_t smem = cap_smem(LS, nt, sizeof(TabT) == sizeof(float2));
    cudaError_t e = cudaFuncSetAttribute(k_conv_cap<LS, MODE, TabT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_conv_cap<LS, MODE, TabT><<<grid, NTH * cap_slots<LS>(), smem, st>>>(a);
    return cudaGetLastError();
}

template <int LS, int MODE>
cudaError_t launch_lm(const JobsArg &a, int grid, cudaStream_t st) {
    const int nt = max_nt(a);
    return nt <= PAIR_TABLE_NODES ? launch_t<LS, MODE, float2>(a, nt, grid, st)
                                  : launch_t<LS, MODE, float>(a, nt, grid, st);
}

template <int LS, int MODE, typename TabT>
int occupancy_t(int nt) {
    const size_t smem = cap_smem(LS, nt, sizeof(TabT) == sizeof(float2));
    cudaFuncSetAttribute(k_conv_cap<LS, MODE, TabT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_conv_cap<LS, MODE, TabT>, NTH * cap_slots<LS>(), smem);
    return nb;
}

template <int LS, int MODE>
int occupancy_lm(int nt) {
    return nt <= PAIR_TABLE_NODES ? occupancy_t<LS, MODE, float2>(nt) : occupancy_t<LS, MODE, float>(nt);
}

template <int LS>
cudaError_t launch_ls(const JobsArg &a, int mode, int grid, cudaStream_t st) {
    switch (mode) {
        case 0: return launch_lm<LS, 0>(a, grid, st);
        case 1: return launch_lm<LS, 1>(a, grid, st);
        case 2: return launch_lm<LS, 2>(a, grid, st);
        case 3: return launch_lm<LS, 3>(a, grid, st);
        case 4: return launch_lm<LS, 4>(a, grid, st);
        case 5: return launch_lm<LS, 5>(a, grid, st);
        case 6: return launch_lm<LS, 6>(a, grid, st);
        case 7: return launch_lm<LS, 7>(a, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int LS>
int occupancy_ls(int mode, int nt) {
    switch (mode) {
        case 0: return occupancy_lm<LS, 0>(nt);
        case 1: return occupancy_lm<LS, 1>(nt);
        case 2: return occupancy_lm<LS, 2>(nt);
        case 3: return occupancy_lm<LS, 3>(nt);
        case 4: return occupancy_lm<LS, 4>(nt);
        case 5: return occupancy_lm<LS, 5>(nt);
        case 6: return occupancy_lm<LS, 6>(nt);
        case 7: return occupancy_lm<LS, 7>(nt);
        default: return 0;
    }
}

}  // namespace

cudaError_t sk_launch_cap_sym(const JobDesc &j, int r0, int r1, int split, cudaStream_t st) {
    if (r1 <= r0 || j.batch <= 0) return cudaSuccess;
    const dim3 grid(r1 - r0, j.batch < 65535 ? j.batch : 65535);
    if (split == 4) k_cap_sym<4><<<grid, 256, 0, st>>>(j, r0);
    else if (split == 2) k_cap_sym<2><<<grid, 256, 0, st>>>(j, r0);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t sk_launch_conv_cap(const JobsArg &a, int ls, int mode, int grid, cudaStream_t st) {
    if (a.total <= 0) return cudaSuccess;
    switch (ls) {
        case SK_CAP_LS[0]: return launch_ls<SK_CAP_LS[0]>(a, mode, grid, st);
        case SK_CAP_LS[1]: return launch_ls<SK_CAP_LS[1]>(a, mode, grid, st);
        case SK_CAP_LS[2]: return launch_ls<SK_CAP_LS[2]>(a, mode, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

int sk_cap_items_per_block(int ls) { return ls <= 640 ? 4 : 2; }

int sk_cap_blocks_per_sm(int ls, int mode, int nt) {
    switch (ls) {
        case SK_CAP_LS[0]: return occupancy_ls<SK_CAP_LS[0]>(mode, nt);
        case SK_CAP_LS[1]: return occupancy_ls<SK_CAP_LS[1]>(mode, nt);
        case SK_CAP_LS[2]: return occupancy_ls<SK_CAP_LS[2]>(mode, nt);
        default: return 0;
    }
}
