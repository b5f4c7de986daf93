// cap_common.cuh -- geometry of the polar-cap work items, shared by the cap kernel
// that evaluates its weights (cap.cu) and the one that streams stored weights
// (capw.cu), and by the weight builder.
//
// Symmetry (Sec. 2's pixelisation): a quarter turn in phi, the reflection
// phi -> pi/2 - phi and the mirror about the equator map pixel centres onto pixel
// centres and keep angles, so a "base" pair (output of the first half quarter of a
// northern ring, input pixel) carries the weight of 16 pairs.  The input is read
// from a symmetric copy H of the maps: H_r[.] = (x_r[a], x_r[a + n/2], x_m[a],
// x_m[a + n/2]) for pixel a of ring r (m the mirror ring), stored with the pixels
// split by residue modulo SPLIT (2 or 4): pixel a at (a mod SPLIT) n/SPLIT +
// floor(a / SPLIT).  A work item's strip of input ring i is four segments of H
// (window pixels, their quarter turn, the reflections and their quarter turn),
// each staged with the same residue split, so that lanes SPLIT pixels apart read
// consecutive float4.
#pragma once
#include "skconv_internal.cuh"
#include "skconv_launch.h"
#include "tc.cuh"

namespace capc {

constexpr int CT = SK_CAP_CT;                          // base outputs per work item
constexpr unsigned long long WAIT_NS = 2000000000ull;  // bound of every wait on a copy

// Bounded wait for a strip: false after WAIT_NS, or at once when another thread of the
// block has given up (the abort flag).
__device__ __forceinline__ bool strip_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    if (tc::mbar_try(bar, parity)) return true;
    const unsigned long long t0 = tc::gtimer();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (tc::mbar_try(bar, parity)) return true;
        if (*abort_flag || tc::gtimer() - t0 > WAIT_NS) return false;
    }
}

// Nearest input pixel of output jo: floor(num / (2 n_o)) with num below 2^31
// (in the caps jo < n_o / 4 <= 2 Nside and n_i <= 4 Nside <= 32768), by the
// item's multiply-high constants for the divisor 2 n_o: mg = ceil(2^(31+l) / d),
// l = ceil(log2 d), quotient = umulhi(num, mg) >> (l - 1), exact for every
// num < 2^31 (Granlund and Montgomery 1994, Thm 4.2).
__device__ __forceinline__ int centre_of(int jo, int n_o, int s_o, const PairInfo &P, unsigned mg, int sh) {
    const unsigned num = (unsigned)(2 * jo + s_o) * (unsigned)P.n_i + (unsigned)(1 - P.s_i) * (unsigned)n_o;
    return (int)(__umulhi(num, mg) >> sh);
}

// q of window pixel jlo (may be negative) for output jo: both products are below 2^31.
__device__ __forceinline__ int q_of(int jlo, int jo, int n_o, int s_o, const PairInfo &P) {
    return (2 * jlo + P.s_i) * n_o - (2 * jo + s_o) * P.n_i;
}

// Window start relative to the centre, and length, of input ring P.
__device__ __forceinline__ void win_shape(const PairInfo &P, int &before, int &cnt) {
    if (P.W < 0) { before = (P.n_i - 1) / 2; cnt = P.n_i; }
    else         { before = P.W; cnt = 2 * P.W + 1; }
}

// Base outputs of a quarter ring of Q pixels with shift s: [0, T).
__device__ __forceinline__ int base_count(int Q, int s) { return s ? (Q + 1) / 2 : Q / 2 + 1; }

// Position of staged position m in a strip row of LS float4 (residues of m modulo SPLIT
// in blocks of LS / SPLIT).
template <int SPLIT, int LS>
__device__ __forceinline__ int split_index(int m) {
    return (m & (SPLIT - 1)) * (LS / SPLIT) + (m / SPLIT);
}

// Position of pixel a (any integer) of a ring of n pixels in its H row.
template <int SPLIT>
__device__ __forceinline__ int h_index(int a, int n) {
    a %= n;
    if (a < 0) a += n;
    return (a & (SPLIT - 1)) * (n / SPLIT) + a / SPLIT;
}
// The same for -2n < a < 2n (the segment starts of a strip shorter than the ring).
template <int SPLIT>
__device__ __forceinline__ int h_index_near(int a, int n) {
    a = a < 0 ? a + n : a;
    a = a < 0 ? a + n : a;
    a = a >= n ? a - n : a;
    a = a >= n ? a - n : a;
    return (a & (SPLIT - 1)) * (n / SPLIT) + a / SPLIT;
}

// The strip of input ring P for an item: L window positions from pixel u0 (base
// frame); the segments start at the natural pixels seg_start(0..3).
struct Strip {
    int L, u0;
};
// Segment g: window pixels from u0 (g = 0) and from u0 + n/4 (g = 1); their
// reflections n/4 - s - (u0 + m) (g = 2) and that + n/4 (g = 3) in natural order,
// i.e. starting at the reflection of the last position.
__device__ __forceinline__ int seg_start(int g, const Strip &S, const PairInfo &P) {
    const int Q = P.n_i >> 2;
    const int rf = Q - P.s_i - S.u0 - (S.L - 1);
    return g == 0 ? S.u0 : g == 1 ? S.u0 + Q : g == 2 ? rf : rf + Q;
}

// Bulk copies of ring P's strip (L < n_i: each residue part of a segment is at most
// a ring's residue row, so it is one or two contiguous pieces of H) into buf,
// completing on mbarrier bar.  Called by the 32 lanes of one warp; lanes
// 0 .. 4 SPLIT - 1 each copy one (segment, residue) part.  HINT: the copies carry the
// L2 policy `policy` for the lines of H.
template <int SPLIT, int LS, bool HINT = false>
__device__ __forceinline__ void issue_strip(float4 *buf, uint32_t bar, const float4 *hrow, const Strip &S,
                                            const PairInfo &P, int lane, uint64_t policy = 0) {
    if (lane == 0) tc::mbar_expect_tx(bar, (uint32_t)(4 * S.L) * 16u);
    __syncwarp();
    if (lane < 4 * SPLIT) {
        const int g = lane / SPLIT, e = lane % SPLIT;
        const int n = P.n_i, w = n / SPLIT;
        const int cnt = (S.L - e + SPLIT - 1) / SPLIT;       // positions e, e + SPLIT, ... below L
        if (cnt > 0) {
            const int i0 = h_index_near<SPLIT>(seg_start(g, S, P) + e, n);
            const int row = i0 / w, k0 = i0 - row * w;         // residue row of the part and its start
            const float4 *src = hrow + row * w;
            const uint32_t dst = tc::smem_u32(buf + g * LS + e * (LS / SPLIT));
            const int len = min(cnt, w - k0);
            if constexpr (HINT) {
                tc::bulk_g2s_hint(dst, src + k0, (uint32_t)len * 16u, bar, policy);
                if (cnt > len) tc::bulk_g2s_hint(dst + (uint32_t)len * 16u, src, (uint32_t)(cnt - len) * 16u, bar, policy);
            } else {
                tc::bulk_g2s(dst, src + k0, (uint32_t)len * 16u, bar);
                if (cnt > len) tc::bulk_g2s(dst + (uint32_t)len * 16u, src, (uint32_t)(cnt - len) * 16u, bar);
            }
        }
    }
}

// The same strip copied by the nth threads of an item with plain loads (strips that
// wrap the whole ring); the caller synchronises the item's threads afterwards.
template <int SPLIT, int LS>
__device__ __forceinline__ void copy_strip(float4 *buf, const float4 *hrow, const Strip &S, const PairInfo &P,
                                           int t, int nth) {
    for (int g = 0; g < 4; ++g) {
        const int a0 = seg_start(g, S, P);
        for (int m = t; m < S.L; m += nth) buf[g * LS + split_index<SPLIT, LS>(m)] = hrow[h_index<SPLIT>(a0 + m, P.n_i)];
    }
}

// Outputs of base pixel j (and of its reflection jr when it has one) from the 8
// accumulators of its 16 images: (north, its half turn), (south, its half turn) for
// quarter turns 0 and 1, then the same for the reflected pair.
__device__ __forceinline__ void store16(float *yn, float *ys, int j, int jr, bool refl, int Q, const float2 *acc) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if (r == 1 && !refl) break;
        const int jj = r ? jr : j;
        const float2 *a = acc + 4 * r;
        yn[jj] = a[0].x;
        yn[jj + 2 * Q] = a[0].y;
        ys[jj] = a[1].x;
        ys[jj + 2 * Q] = a[1].y;
        yn[jj + Q] = a[2].x;
        yn[jj + 3 * Q] = a[2].y;
        ys[jj + Q] = a[3].x;
        ys[jj + 3 * Q] = a[3].y;
    }
}

}  // namespace capc
