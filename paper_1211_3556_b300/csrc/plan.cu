// plan.cu -- which path covers which output ring, the work items of each path,
// and the launch sequences of the forward operator and of the table gradient.
//
// Rings are split three ways when a kernel handle is built:
//  * belt: a symmetric range of equatorial rings whose whole window lies in the
//    belt (all rings of 4 Nside pixels), computed as ring-wise Toeplitz sums;
//  * caps: the remaining northern rings (not the equator ring) with their
//    southern mirrors, evaluated per pair and shared by the 8 symmetric images;
//  * general: whatever neither covers (e.g. the equator ring when no belt
//    exists at a small Nside and a wide cut), evaluated per pair.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "skconv_host.h"

namespace {

template <typename T>
int upload(const std::vector<T> &h, T **d) {
    *d = nullptr;
    if (h.empty()) return SK_OK;
    SK_CU(cudaMalloc(d, sizeof(T) * h.size()));
    SK_CU(cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
    return SK_OK;
}

int centre(int jo, int n_o, int s_o, const PairInfo &P) {
    long long num = (long long)(2 * jo + s_o) * P.n_i + (long long)(1 - P.s_i) * n_o;
    return (int)(num / (2LL * n_o));
}

// Strip length a cap item needs for input ring P, and the largest |q| of its windows.
// The cap kernel evaluates narrow windows in pixel pairs, one pixel past the
// window when its count is odd (that pixel is outside the cut).
// The stored-weight kernel's strip holds the union windows of its last active thread
// (outputs j0 + 4 k .. + 3): the larger of the two lengths sizes the item's strip class.
void cap_needs(int j0, int jlast, int n_o, int s_o, const PairInfo &P, int &L, long long &qmax) {
    int cnt = P.W < 0 ? P.n_i : 2 * P.W + 1;
    L = centre(jlast, n_o, s_o, P) - centre(j0, n_o, s_o, P) + cnt + 1;
    const int jl = j0 + 4 * ((jlast - j0) / 4);
    L = std::max(L, centre(jl, n_o, s_o, P) - centre(j0, n_o, s_o, P) + sk_capw_steps(cnt, P.n_i, n_o));
    // q at the window centre is below n_o + n_i in magnitude; each step adds 2 n_o
    qmax = (long long)n_o + P.n_i + (long long)(cnt + 1) * 2 * n_o;
}

// Multiply-high division by d (2 <= d < 2^31) for numerators below 2^31:
// mg = ceil(2^(31+l) / d) with l = ceil(log2 d) (below 2^32), and
// floor(n / d) = umulhi(n, mg) >> sh, sh = l - 1 (Granlund and Montgomery 1994).
void div_magic(unsigned d, unsigned &mg, int &sh) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    const unsigned long long m = ((1ull << (31 + l)) + d - 1) / d;
    mg = (unsigned)m;
    sh = l - 1;
}

int belt_cost_p(int n4) {
    // choose the outputs-per-thread P: tail waste of the last segment against the
    // per-chunk overhead of reloading P + 3 strip values for 4P FFMAs
    const int Ps[] = {5, 7, 9, 11, 13, 15, 17};
    int best = 13;
    double bc = 1e300;
    for (int P : Ps) {
        int ts = 32 * P;
        int nseg = (n4 + ts - 1) / ts;
        double c = (double)nseg * ts * (1.0 + 3.0 / P);
        if (c < bc - 1e-9) { bc = c; best = P; }
    }
    return best;
}

}  // namespace

void sk_capw_free(sk_kern *k) {
    cudaFree(k->d_capw);
    k->d_capw = nullptr;
}

void sk_plan_free(sk_kern *k) {
    sk_capw_free(k);
    cudaFree(k->d_beltw); k->d_beltw = nullptr;
    cudaFree(k->d_capw_ring); k->d_capw_ring = nullptr;
    k->h_capw_ring.clear();
    k->capw_len = 0;
    cudaFree(k->d_items_gen); k->d_items_gen = nullptr;
    cudaFree(k->d_ring_path); k->d_ring_path = nullptr;
    cudaFree(k->d_bgrp); k->d_bgrp = nullptr;
    cudaFree(k->d_bpr); k->d_bpr = nullptr;
    cudaFree(k->d_items_belt); k->d_items_belt = nullptr;
    for (TcPlan &T : k->tcp) {
        cudaFree(T.d_tiles); T.d_tiles = nullptr;
        cudaFree(T.d_group); T.d_group = nullptr;
        cudaFree(T.d_rng); T.d_rng = nullptr;
        cudaFree(T.d_A); T.d_A = nullptr;
        T.h_tiles.clear();
        T.ok = false;
    }
    for (int c = 0; c < SK_CAP_LS_CLASSES; ++c)
        for (int v = 0; v < 2; ++v) {
            cudaFree(k->d_items_cap[c][v]); k->d_items_cap[c][v] = nullptr;
            k->h_items_cap[c][v].clear();
        }
    cudaFree(k->d_items_gcap); k->d_items_gcap = nullptr;
    k->n_items_gcap = 0;
    k->gcap_walk = 0;
    k->h_items_belt.clear();
    k->h_items_gen.clear();
    cudaFree(k->d_band_items); k->d_band_items = nullptr;
    k->bands.clear();
    k->bands_P = 0;
    {
        std::lock_guard<std::mutex> lock(k->subsets_mu);
        for (auto &r : k->subsets) cudaFree(r.d_items);
        k->subsets.clear();
    }
    k->plan_ok = false;
}

int sk_plan_ring_subset(sk_kern *k, int lo, int hi, bool sym, const SkItems **out) {
    std::lock_guard<std::mutex> lock(k->subsets_mu);
    for (auto &r : k->subsets)
        if (r.lo == lo && r.hi == hi && r.sym == sym && r.P == k->belt_P) { *out = &r.items; return SK_OK; }
    // a bounded cache: past SK_MAX_RING_SUBSETS ranges the lists are dropped (after every
    // launch that may read them has finished) and rebuilt as ranges are asked for again
    if (k->subsets.size() >= (size_t)SK_MAX_RING_SUBSETS) {
        SK_CU(cudaDeviceSynchronize());
        for (auto &r : k->subsets) cudaFree(r.d_items);
        k->subsets.clear();
    }
    const sk_geom *g = k->g;
    const int nr = g->nr;
    auto in = [&](int r) { return (r >= lo && r < hi) || (sym && nr - 1 - r >= lo && nr - 1 - r < hi); };
    std::vector<int4> all;
    size_t off_belt = 0, n_belt = 0, off_cap[SK_CAP_LS_CLASSES][2] = {}, n_cap[SK_CAP_LS_CLASSES][2] = {};
    size_t off_gen = 0, n_gen = 0;
    bool caps = false;
    int bg[2][2] = {{0, -1}, {0, 0}};     // belt groups (all without a plan)
    int smin = 1 << 30, smax = 0;          // rings of the symmetric copy the cap items read
    if (k->plan_ok) {
        // a belt item (ring group, tile) writes rings b_lo + 16 group .. + 15; a cap item its
        // northern ring and the mirror; a per-pair item its ring.  The groups of the range
        // and those of its mirror are kept as two group ranges (the belt weight rows of the
        // groups between them are not needed)
        int gmin[2] = {1 << 30, 1 << 30}, gmax[2] = {-1, -1};
        for (const int4 &it : k->h_items_belt) {
            const int r0 = k->b_lo + it.x * SK_BELT_G, r1 = std::min(r0 + SK_BELT_G, k->b_lo + k->nb);
            const bool north = r0 < hi && r1 > lo, mirror = sym && r0 < nr - lo && r1 > nr - hi;
            if (north || mirror) all.push_back(it);
            for (int q = 0; q < 2; ++q)
                if (q == 0 ? north : mirror) {
                    gmin[q] = std::min(gmin[q], it.x);
                    gmax[q] = std::max(gmax[q], it.x);
                }
        }
        for (int q = 0; q < 2; ++q) {
            bg[q][0] = gmax[q] >= 0 ? gmin[q] : 0;
            bg[q][1] = gmax[q] >= 0 ? gmax[q] + 1 : 0;
        }
        // overlapping (or adjacent) ranges: one range
        if (bg[1][1] > bg[1][0] && bg[0][1] > bg[0][0] && bg[1][0] <= bg[0][1] && bg[0][0] <= bg[1][1]) {
            bg[0][0] = std::min(bg[0][0], bg[1][0]);
            bg[0][1] = std::max(bg[0][1], bg[1][1]);
            bg[1][0] = bg[1][1] = 0;
        }
        n_belt = all.size();
        for (int c = 0; c < SK_CAP_LS_CLASSES; ++c)
            for (int v = 0; v < 2; ++v) {
                off_cap[c][v] = all.size();
                for (const int4 &it : k->h_items_cap[c][v])
                    if (in(it.x) || in(nr - 1 - it.x)) {
                        all.push_back(it);
                        // the symmetric copy rows its windows read
                        const int a = k->h_pair_off[it.x], z = k->h_pair_off[it.x + 1] - 1;
                        smin = std::min(smin, k->h_pairs[a].ri);
                        smax = std::max(smax, k->h_pairs[z].ri + 1);
                    }
                n_cap[c][v] = all.size() - off_cap[c][v];
                caps = caps || n_cap[c][v] > 0;
            }
        off_gen = all.size();
        for (const int4 &it : k->h_items_gen)
            if (in(it.x)) all.push_back(it);
    } else {
        off_gen = 0;
        for (int r = 0; r < nr; ++r)
            if (in(r))
                for (int j = 0; j < g->h_rings[r].n; j += 128) all.push_back(make_int4(r, j, 0, 0));
    }
    n_gen = all.size() - off_gen;
    sk_kern::RingSubset rs{lo, hi, k->belt_P, sym, nullptr, SkItems{}};
    if (!all.empty()) {
        cudaError_t e = cudaMalloc(&rs.d_items, sizeof(int4) * all.size());
        if (e == cudaSuccess) e = cudaMemcpy(rs.d_items, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(rs.d_items);
            return sk_fail(SK_ENOMEM, "ring subset: %s", cudaGetErrorString(e));
        }
    }
    rs.items.belt = n_belt ? rs.d_items + off_belt : nullptr;
    rs.items.n_belt = (int)n_belt;
    for (int c = 0; c < SK_CAP_LS_CLASSES; ++c)
        for (int v = 0; v < 2; ++v) {
            rs.items.cap[c][v] = n_cap[c][v] ? rs.d_items + off_cap[c][v] : nullptr;
            rs.items.n_cap[c][v] = (int)n_cap[c][v];
        }
    rs.items.gen = n_gen ? rs.d_items + off_gen : nullptr;
    rs.items.n_gen = (int)n_gen;
    if (caps) {
        rs.items.sym[0][0] = std::max(0, smin);
        rs.items.sym[0][1] = std::min(k->sym_hi, smax);
    }
    for (int q = 0; q < 2; ++q) {
        rs.items.bg[q][0] = bg[q][0];
        rs.items.bg[q][1] = bg[q][1];
    }
    k->subsets.push_back(rs);                       // entries of other tile widths stay (in use elsewhere)
    *out = &k->subsets.back().items;
    return SK_OK;
}

int sk_plan_rebuild_belt_items(sk_kern *k) {
    cudaFree(k->d_items_belt);
    k->d_items_belt = nullptr;
    k->n_items_belt = 0;
    if (k->nb == 0) return SK_OK;
    const int n4 = (int)(4 * k->g->nside);
    const int ts = 32 * k->belt_P;
    const int nseg = (n4 + ts - 1) / ts;
    std::vector<int4> it;
    for (int g = 0; g < k->ngroups; ++g)
        for (int s = 0; s < nseg; ++s) it.push_back(make_int4(g, s, 0, 0));
    k->n_items_belt = (int)it.size();
    k->h_items_belt = it;
    if (int rc = upload(it, &k->d_items_belt)) return rc;
    // the band partition of the host-buffer path holds belt items: rebuild it (a no-op
    // before the first plan is complete)
    return k->plan_ok ? sk_plan_bands(k) : SK_OK;
}

// Tiles of a tensor-core belt form: one per (group, input ring) with any window.  3xTF32
// (bf false): E0 = the union's first offset rounded down to a multiple of 4, K covers the
// union plus the 7 extra columns of a segment's 8 output pixels, rounded up to 8 (one
// TF32 k-step); BF16x3: E0 a multiple of 8 (the operand rows hold 8 pixels), K rounded up to
// 16.  Chunks of consecutive tiles with at least SK_TC_CHUNK_KSTEPS k-steps of 8 columns
// are accumulated together in tensor memory.
static int plan_tc(sk_kern *k, const std::vector<int2> &grp, const std::vector<int2> &ew, int HM, int R2, int n4,
                   int b_lo, bool bf, TcPlan &T) {
    const int ealign = bf ? 8 : 4, kalign = bf ? 16 : 8;
    std::vector<int4> tl;
    std::vector<int> tg;
    std::vector<int4> tr(k->ngroups);
    long long kb = 0;
    int kmax = 0;
    for (int gi = 0; gi < k->ngroups; ++gi) {
        const int first = (int)tl.size();
        for (int i = grp[gi].x; i <= grp[gi].y; ++i) {
            int lo = 1 << 30, hi = -(1 << 30);
            for (int w = 0; w < SK_BELT_G; ++w) {
                const int rb = gi * SK_BELT_G + w, d = i - (b_lo + rb);
                if (rb >= k->nb || d < -HM || d > HM) continue;
                const int2 e = ew[(size_t)rb * R2 + d + HM];
                if (e.x > e.y) continue;
                lo = std::min(lo, e.x);
                hi = std::max(hi, e.y);
            }
            if (lo > hi) continue;
            const int E0 = lo >= 0 ? (lo / ealign) * ealign : -(((-lo) + ealign - 1) / ealign) * ealign;
            const int K = (hi - E0 + 8 + kalign - 1) / kalign * kalign;
            // A bytes: K columns of 128 rows, hi and lo parts (4 or 2 bytes an element) -> KB
            const int akb = bf ? K / 2 : K;
            tl.push_back(make_int4(i, E0, K, (int)std::min<long long>(kb, 1 << 30)));
            tg.push_back(gi);
            kb += akb;
            kmax = std::max(kmax, K);
        }
        int ks = 0, nchunk = 0;
        for (int u = first; u < (int)tl.size(); ++u) {
            if (ks == 0) tl[u].z |= SK_TC_FIRST;
            ks += (tl[u].z & SK_TC_K_MASK) / 8;
            if (ks >= SK_TC_CHUNK_KSTEPS || u + 1 == (int)tl.size()) {
                tl[u].z |= SK_TC_LAST;
                ks = 0;
                ++nchunk;
            }
        }
        tr[gi] = make_int4(first, (int)tl.size() - first, nchunk, 0);
    }
    const int nn = std::min(256, (n4 / 8) & ~15);
    T.ok = false;
    if (nn < 16 || kmax > 64 || kb >= (1 << 30) || tl.empty()) return SK_OK;
    T.nn = nn;
    T.nblk = (n4 + 8 * nn - 1) / (8 * nn);
    T.kmax = kmax;
    T.stages = sk_tc_stages(kmax, nn, bf, nullptr);
    T.kb = kb;
    if (T.stages < 2) return SK_OK;
    T.h_tiles = tl;
    int rc;
    if ((rc = upload(tl, &T.d_tiles))) return rc;
    if ((rc = upload(tg, &T.d_group))) return rc;
    if ((rc = upload(tr, &T.d_rng))) return rc;
    T.ok = true;
    return SK_OK;
}

int sk_plan_build(sk_kern *k) {
    const sk_geom *g = k->g;
    const int nr = g->nr;
    const long long N = g->nside;
    const int n4 = (int)(4 * N);
    const int eq = (int)(2 * N - 1);           // equator ring (0-based)
    const auto &R = g->h_rings;
    const auto &off = k->h_pair_off;
    const auto &pairs = k->h_pairs;

    // ---- belt: rings whose whole window has 4N pixels per ring and narrow windows
    auto belt_ok = [&](int r) {
        if (R[r].n != n4) return false;
        for (int p = off[r]; p < off[r + 1]; ++p) {
            const PairInfo &P = pairs[p];
            if (P.n_i != n4 || P.W < 0) return false;
            int nch = (2 * P.W + 1 + 3) / 4;
            if (4 * nch > n4) return false;
            // the streamed strips and weight rows of the widest tile must fit in shared memory
            if (sk_belt_smem_bytes(17, 2 * P.W + 8) > (size_t)200 * 1024) return false;
        }
        return true;
    };
    int b_lo = eq, b_hi = eq;
    if (belt_ok(eq)) {
        while (b_lo - 1 >= 0 && belt_ok(b_lo - 1) && belt_ok(nr - 1 - (b_lo - 1))) --b_lo;
        b_hi = nr - 1 - b_lo;
        k->b_lo = b_lo;
        k->nb = b_hi - b_lo + 1;
    } else {
        k->b_lo = eq;
        k->nb = 0;
    }

    std::vector<char> covered(nr, 0);
    if (k->nb > 0) {
        int HM = 0;
        for (int r = b_lo; r <= b_hi; ++r) HM = std::max(HM, std::max(r - k->h_lo[r], k->h_hi[r] - r));
        k->HM = HM;
        const int R2 = 2 * HM + 1;
        k->ngroups = (k->nb + SK_BELT_G - 1) / SK_BELT_G;
        const int nb_pad = k->ngroups * SK_BELT_G;
        int EMIN = 1 << 30, EMAX = -(1 << 30);
        for (int rb = 0; rb < k->nb; ++rb) {
            const int r = b_lo + rb;
            for (int p = off[r]; p < off[r + 1]; ++p) {
                const PairInfo &P = pairs[p];
                const int ec = (R[r].s + 1 - P.s_i) >> 1;     // offset of the nearest input pixel
                EMIN = std::min(EMIN, ec - P.W);
                EMAX = std::max(EMAX, ec + P.W);
            }
        }
        std::vector<int2> ew((size_t)nb_pad * R2, make_int2(1, 0));     // exact offset range per row
        for (int rb = 0; rb < k->nb; ++rb) {
            const int r = b_lo + rb;
            covered[r] = 1;
            for (int p = off[r]; p < off[r + 1]; ++p) {
                const PairInfo &P = pairs[p];
                const int d = P.ri - r;
                const int ec = (R[r].s + 1 - P.s_i) >> 1;
                ew[(size_t)rb * R2 + d + HM] = make_int2(ec - P.W, ec + P.W);
            }
        }
        const int WPM = ((EMAX - EMIN + 1) + 3) & ~3;
        k->EMIN = EMIN; k->EMAX = EMIN + WPM - 1; k->WPM = WPM;
        std::vector<int2> grp(k->ngroups);
        for (int gi = 0; gi < k->ngroups; ++gi) {
            int lo = 1 << 30, hi = -1;
            for (int w = 0; w < SK_BELT_G; ++w) {
                int rb = gi * SK_BELT_G + w;
                if (rb >= k->nb) break;
                lo = std::min(lo, k->h_lo[b_lo + rb]);
                hi = std::max(hi, k->h_hi[b_lo + rb]);
            }
            grp[gi] = make_int2(lo, hi);
        }
        // pair rows as the FP32 kernel streams them: strip si of group gi is input
        // ring grp[gi].x + si; warp w applies rows (2w, i) and (2w + 1, i) to it
        int smax = 0;
        for (int gi = 0; gi < k->ngroups; ++gi) smax = std::max(smax, grp[gi].y - grp[gi].x + 1);
        k->smax = smax;
        // (first offset - EMIN, 4-offset chunks) of the union of both rows' windows; (0, 0) = empty
        std::vector<int2> pr((size_t)k->ngroups * smax * SK_BELT_WARPS, make_int2(0, 0));
        for (int gi = 0; gi < k->ngroups; ++gi)
            for (int si = 0; si <= grp[gi].y - grp[gi].x; ++si)
                for (int w = 0; w < SK_BELT_WARPS; ++w) {
                    int lo = 1 << 30, hi = -(1 << 30);
                    for (int q = 0; q < 2; ++q) {
                        const int rb = gi * SK_BELT_G + 2 * w + q;
                        const int d = grp[gi].x + si - (b_lo + rb);
                        if (rb >= k->nb || d < -HM || d > HM) continue;
                        const int2 e = ew[(size_t)rb * R2 + d + HM];
                        if (e.x > e.y) continue;
                        lo = std::min(lo, e.x);
                        hi = std::max(hi, e.y);
                    }
                    if (lo <= hi)
                        pr[((size_t)gi * smax + si) * SK_BELT_WARPS + w] = make_int2(lo - EMIN, (hi - lo + 4) / 4);
                }
        int rc;
        if ((rc = upload(grp, &k->d_bgrp))) return rc;
        k->h_bgrp = grp;
        if ((rc = upload(pr, &k->d_bpr))) return rc;
        k->belt_P = belt_cost_p(n4);
        if ((rc = sk_plan_rebuild_belt_items(k))) return rc;
        // tensor-core belt forms: 3xTF32 and BF16x3
        for (int f = 0; f < 2; ++f)
            if ((rc = plan_tc(k, grp, ew, HM, R2, n4, b_lo, f == 1, k->tcp[f]))) return rc;
    }

    // ---- caps: northern rings below the belt (never the equator ring) and mirrors
    std::vector<int4> cap_items[SK_CAP_LS_CLASSES][2];
    const int cap_end = k->nb > 0 ? b_lo : eq;
    k->n_cap_rings = 0;
    std::vector<char> cap_wide(nr, 0);      // cap rings whose windows are too wide for the sine series
    for (int r = 0; r < cap_end; ++r) {
        const int Q = R[r].n / 4;
        const int T = R[r].s ? (Q + 1) / 2 : Q / 2 + 1;     // base outputs (the rest are reflections)
        int need = 0;
        bool ok = (nr - 1 - r) != r;
        bool series = true;        // |dphi / 2| <= 1/8 on every window of the ring
        for (int p = off[r]; p < off[r + 1]; ++p) {
            const PairInfo &P = pairs[p];
            if (P.W < 0 || (P.W + 2.5) * SK_PI / P.n_i > 0.125) series = false;
        }
        for (int j0 = 0; j0 < T && ok; j0 += SK_CAP_CT) {
            const int jl = std::min(j0 + SK_CAP_CT - 1, T - 1);
            for (int p = off[r]; p < off[r + 1]; ++p) {
                int L; long long qm;
                cap_needs(j0, jl, R[r].n, R[r].s, pairs[p], L, qm);
                need = std::max(need, L);
                if (qm >= (1LL << 24)) ok = false;
            }
        }
        int cls = -1;
        for (int c = 0; c < SK_CAP_LS_CLASSES && ok; ++c)
            if (need <= SK_CAP_LS[c]) { cls = c; break; }
        if (!ok || cls < 0) continue;
        covered[r] = covered[nr - 1 - r] = 1;
        if (!series) cap_wide[r] = cap_wide[nr - 1 - r] = 1;
        ++k->n_cap_rings;
        unsigned mg; int sh;
        div_magic(2u * (unsigned)R[r].n, mg, sh);
        for (int j0 = 0; j0 < T; j0 += SK_CAP_CT)
            cap_items[cls][series ? 1 : 0].push_back(make_int4(r, j0, (int)mg, sh));
    }
    // input rings of the cap items: their symmetric copy is built per call
    k->sym_hi = 0;
    for (int c = 0; c < SK_CAP_LS_CLASSES; ++c)
        for (int v = 0; v < 2; ++v)
            for (const int4 &it : cap_items[c][v])
                for (int p = off[it.x]; p < off[it.x + 1]; ++p) k->sym_hi = std::max(k->sym_hi, pairs[p].ri + 1);
    k->sym_stride = k->sym_hi >= nr ? g->npix : R[k->sym_hi].start;
    for (int c = 0; c < SK_CAP_LS_CLASSES; ++c)
        for (int v = 0; v < 2; ++v) {
            // heavier rings first: per-item cost grows with the number of window pixels
            std::stable_sort(cap_items[c][v].begin(), cap_items[c][v].end(), [&](const int4 &a, const int4 &b) {
                return (off[a.x + 1] - off[a.x]) > (off[b.x + 1] - off[b.x]);
            });
            k->n_items_cap[c][v] = (int)cap_items[c][v].size();
            k->h_items_cap[c][v] = cap_items[c][v];
            int rc = upload(cap_items[c][v], &k->d_items_cap[c][v]);
            if (rc) return rc;
        }
    // the table gradient's cap items: one list, longest window walks first (a walk's steps,
    // the window pixels of all the ring's window rings, set a gradient task's length)
    {
        std::vector<long long> walk(nr, 0);
        std::vector<int4> all;
        for (int c = 0; c < SK_CAP_LS_CLASSES; ++c)
            for (int v = 0; v < 2; ++v)
                for (const int4 &it : cap_items[c][v]) {
                    if (walk[it.x] == 0)
                        for (int p = off[it.x]; p < off[it.x + 1]; ++p)
                            walk[it.x] += pairs[p].W < 0 ? pairs[p].n_i : 2 * pairs[p].W + 1;
                    k->gcap_walk = std::max(k->gcap_walk, walk[it.x]);
                    all.push_back(it);
                }
        std::stable_sort(all.begin(), all.end(),
                         [&](const int4 &a, const int4 &b) { return walk[a.x] > walk[b.x]; });
        k->n_items_gcap = (int)all.size();
        if (int rc = upload(all, &k->d_items_gcap)) return rc;
    }
    // layout of the stored cap weights: the items of a ring share its step count (the sum
    // over its window rings of the union steps), rings one after another
    {
        std::vector<char> is_cap(nr, 0);
        for (int c = 0; c < SK_CAP_LS_CLASSES; ++c)
            for (int v = 0; v < 2; ++v)
                for (const int4 &it : cap_items[c][v]) is_cap[it.x] = 1;
        k->h_capw_ring.assign(nr, make_longlong2(-1, 0));
        long long len = 0;
        for (int r = 0; r < nr; ++r) {
            if (!is_cap[r]) continue;
            long long steps = 0;
            for (int p = off[r]; p < off[r + 1]; ++p) {
                const PairInfo &P = pairs[p];
                steps += sk_capw_steps(P.W < 0 ? P.n_i : 2 * P.W + 1, P.n_i, R[r].n);
            }
            const int Q = R[r].n / 4;
            const int T = R[r].s ? (Q + 1) / 2 : Q / 2 + 1;
            const long long items = (T + SK_CAP_CT - 1) / SK_CAP_CT;
            k->h_capw_ring[r] = make_longlong2(len, steps);
            len += items * steps * (SK_CAP_CT / 4);
        }
        // the kernel loads one group of four steps ahead of the one it sums
        k->capw_len = len > 0 ? len + 8 * (SK_CAP_CT / 4) : 0;
        if (int rc = upload(k->h_capw_ring, &k->d_capw_ring)) return rc;
    }

    // ---- general: the rest
    std::vector<int4> gen;
    std::vector<unsigned char> path(nr, 1);
    for (int r = 0; r < nr; ++r)
        if (cap_wide[r]) path[r] = 3;
    for (int r = b_lo; r < b_lo + k->nb; ++r) path[r] = 0;
    for (int r = 0; r < nr; ++r)
        if (!covered[r]) {
            path[r] = 2;
            for (int j = 0; j < R[r].n; j += 128) gen.push_back(make_int4(r, j, 0, 0));
        }
    if (int rc0 = upload(path, &k->d_ring_path)) return rc0;
    k->h_ring_path = path;
    k->n_items_gen = (int)gen.size();
    k->h_items_gen = gen;
    int rc = upload(gen, &k->d_items_gen);
    if (rc) return rc;
    // window pixels of the widest output: the summation mode of the belt and caps
    k->max_terms = 0;
    for (int r = 0; r < nr; ++r) {
        long long t = 0;
        for (int p = off[r]; p < off[r + 1]; ++p) t += pairs[p].W < 0 ? pairs[p].n_i : 2 * pairs[p].W + 1;
        k->max_terms = std::max(k->max_terms, t);
    }
    k->blocked = k->max_terms > SK_BLOCKED_TERMS;
    k->plan_ok = true;
    return sk_plan_bands(k);
}

int sk_plan_bands(sk_kern *k) {
    if (!k->plan_ok) return SK_OK;
    if (!k->bands.empty() && k->bands_P == k->belt_P) return SK_OK;
    cudaFree(k->d_band_items);
    k->d_band_items = nullptr;
    k->bands.clear();
    const sk_geom *g = k->g;
    const int nr = g->nr, eq = nr / 2;                   // equator ring (0-based): distance eq from both poles
    auto dist = [&](int r) { return std::min(r, nr - 1 - r); };
    // band edges in pole distance: equal pixel counts (both hemispheres)
    const int K = SK_HOST_BANDS;
    std::vector<int> edge(K + 1, eq + 1);
    edge[0] = 0;
    {
        long long tot = g->npix, acc = 0;
        int b = 1;
        for (int d = 0; d <= eq && b < K; ++d) {
            acc += (d == eq) ? g->h_rings[d].n : 2LL * g->h_rings[d].n;
            while (b < K && acc * K >= tot * b) edge[b++] = d + 1;
        }
        for (int i = 1; i <= K; ++i) edge[i] = std::max(edge[i], edge[i - 1]);
    }
    auto band_of = [&](int d) {
        int b = 0;
        while (b + 1 < K && d >= edge[b + 1]) ++b;
        return b;
    };
    // largest pole distance of any input ring of output ring r
    auto reach = [&](int r) {
        const int lo = k->h_lo[r], hi = k->h_hi[r];
        return (lo <= eq && eq <= hi) ? eq : std::max(dist(lo), dist(hi));
    };
    std::vector<std::vector<int4>> belt(K), gen(K), cap[SK_CAP_LS_CLASSES][2];
    for (int c = 0; c < SK_CAP_LS_CLASSES; ++c)
        for (int v = 0; v < 2; ++v) cap[c][v].resize(K);
    std::vector<int> reach_b(K, 0), ready(K);
    for (int b = 0; b < K; ++b) ready[b] = b;
    for (const int4 &it : k->h_items_belt) {
        // a group of belt rings runs in the band of its ring nearest the equator; the
        // outputs of its other rings are ready only then
        int dmax = 0, rmax = 0;
        for (int w = 0; w < SK_BELT_G; ++w) {
            const int r = k->b_lo + it.x * SK_BELT_G + w;
            if (r >= k->b_lo + k->nb) break;
            dmax = std::max(dmax, dist(r));
            rmax = std::max(rmax, reach(r));
        }
        const int b = band_of(dmax);
        belt[b].push_back(it);
        reach_b[b] = std::max(reach_b[b], rmax);
        for (int w = 0; w < SK_BELT_G; ++w) {
            const int r = k->b_lo + it.x * SK_BELT_G + w;
            if (r >= k->b_lo + k->nb) break;
            ready[band_of(dist(r))] = std::max(ready[band_of(dist(r))], b);
        }
    }
    for (int c = 0; c < SK_CAP_LS_CLASSES; ++c)
        for (int v = 0; v < 2; ++v)
            for (const int4 &it : k->h_items_cap[c][v]) {
                const int b = band_of(dist(it.x));
                cap[c][v][b].push_back(it);
                reach_b[b] = std::max(reach_b[b], reach(it.x));
            }
    for (const int4 &it : k->h_items_gen) {
        const int b = band_of(dist(it.x));
        gen[b].push_back(it);
        reach_b[b] = std::max(reach_b[b], reach(it.x));
    }
    // one device array, band by band and path by path
    std::vector<int4> all;
    struct Off { size_t belt, cap[SK_CAP_LS_CLASSES][2], gen; };
    std::vector<Off> off(K);
    for (int b = 0; b < K; ++b) {
        off[b].belt = all.size();
        all.insert(all.end(), belt[b].begin(), belt[b].end());
        for (int c = 0; c < SK_CAP_LS_CLASSES; ++c)
            for (int v = 0; v < 2; ++v) {
                off[b].cap[c][v] = all.size();
                all.insert(all.end(), cap[c][v][b].begin(), cap[c][v][b].end());
            }
        off[b].gen = all.size();
        all.insert(all.end(), gen[b].begin(), gen[b].end());
    }
    int4 *d = nullptr;
    if (int rc = upload(all, &d)) return rc;
    k->d_band_items = d;
    k->bands.resize(K);
    for (int b = 0; b < K; ++b) {
        sk_kern::Band &B = k->bands[b];
        B.n_lo = edge[b];
        B.n_hi = std::min(edge[b + 1], eq + 1);
        B.s_lo = std::max(nr - edge[b + 1], eq + 1);
        B.s_hi = nr - edge[b];
        B.need = band_of(reach_b[b]);
        B.need = std::max(B.need, b);
        B.ready = ready[b];
        B.items.belt = belt[b].empty() ? nullptr : d + off[b].belt;
        B.items.n_belt = (int)belt[b].size();
        for (int c = 0; c < SK_CAP_LS_CLASSES; ++c)
            for (int v = 0; v < 2; ++v) {
                B.items.cap[c][v] = cap[c][v][b].empty() ? nullptr : d + off[b].cap[c][v];
                B.items.n_cap[c][v] = (int)cap[c][v][b].size();
            }
        B.items.gen = gen[b].empty() ? nullptr : d + off[b].gen;
        B.items.n_gen = (int)gen[b].size();
    }
    // symmetric copies for the caps: the run of band b builds those of the bands up to
    // its `need` that no earlier band built (their maps have arrived by then)
    for (int b = 0, built = -1; b < K; ++b) {
        sk_kern::Band &B = k->bands[b];
        const int upto = std::max(built, B.need);
        if (upto > built) {
            const sk_kern::Band &F = k->bands[built + 1], &U = k->bands[upto];
            B.items.sym[0][0] = std::min(F.n_lo, k->sym_hi);
            B.items.sym[0][1] = std::min(U.n_hi, k->sym_hi);
            B.items.sym[1][0] = std::min(U.s_lo, k->sym_hi);
            B.items.sym[1][1] = std::min(F.s_hi, k->sym_hi);
            built = upto;
        }
    }
    k->bands_P = k->belt_P;
    return SK_OK;
}

size_t sk_plan_workspace_bytes(const sk_kern *k) {
    if (!k->plan_ok || k->nb == 0) return 0;
    // the FP32 belt's ring-pair rows (when the operator does not store them)
    const size_t pairs = (size_t)k->ngroups * k->smax * SK_BELT_WARPS * k->WPM * sizeof(float2);
    return (pairs + 255) & ~(size_t)255;
}

size_t sk_sym_bytes(const sk_kern *k, long long batch) {
    if (!k->plan_ok || k->sym_hi == 0 || batch <= 0) return 0;
    return ((size_t)batch * (size_t)k->sym_stride * sizeof(float4) + 255) & ~(size_t)255;
}

int sk_job_wants_tc(const SkJob &j, int path) {
    const sk_kern *k = j.k;
    int f = -1;
    if (path == SK_PATH_TENSOR) f = 0;
    else if (path == SK_PATH_BF16X3) f = 1;
    else if (path == SK_PATH_AUTO && k->belt_form == SK_BELT_TENSOR) f = 0;
    else if (path == SK_PATH_AUTO && k->belt_form == SK_BELT_BF16X3) f = 1;
    if (f < 0 || !k->plan_ok || k->nb == 0 || !k->tcp[f].ok || j.batch <= 0) return -1;
    return f;
}

// The belt ring groups a job runs: [g[0], g[1]) and [g[2], g[3]) (a ring subset's
// northern groups and their mirror; the whole belt otherwise).
static void job_groups(const SkJob &j, int g[4]) {
    const SkItems *sub = j.sub;
    if (!sub || sub->bg[0][1] < 0) {
        g[0] = 0; g[1] = j.k->ngroups; g[2] = g[3] = 0;
        return;
    }
    g[0] = sub->bg[0][0]; g[1] = sub->bg[0][1]; g[2] = sub->bg[1][0]; g[3] = sub->bg[1][1];
    if (sub->n_belt == 0) g[0] = g[1] = g[2] = g[3] = 0;
}

// Running totals of the evaluating cap launches of wide-window jobs: one slice per
// stream (narrow and polar launches run concurrently), each for up to 2048 threads per SM.
static size_t ctot_bytes(const SkJob *jobs, int n, int path) {
    if (path == SK_PATH_GENERAL) return 0;
    for (int i = 0; i < n; ++i) {
        const sk_kern *k = jobs[i].k;
        if (k->plan_ok && k->blocked && !k->d_capw && jobs[i].batch > 0)
            return (size_t)2 * k->ctx->num_sms * 2048 * 32 * sizeof(float);
    }
    return 0;
}

size_t sk_jobs_workspace_bytes(const SkJob *jobs, int n, int path) {
    size_t b = 0;
    for (int i = 0; i < n; ++i) {
        b += sk_plan_workspace_bytes(jobs[i].k) + sk_sym_bytes(jobs[i].k, jobs[i].batch);
    }
    return b + ctot_bytes(jobs, n, path);
}

// ---------------------------------------------------------------------------
// launch sequences
// ---------------------------------------------------------------------------

namespace {

JobDesc base_desc(const SkJob &jb) {
    const sk_kern *k = jb.k;
    JobDesc d;
    memset(&d, 0, sizeof d);
    d.rings = k->g->d_rings;
    d.pair_off = k->d_pair_off;
    d.pairs = k->d_pairs;
    d.tab = k->d_tab;
    d.kp = k->kp;
    d.kd = k->kd;
    d.ab64 = k->d_ab64;
    d.V64 = k->d_V;
    d.dOmega = 4.0 * SK_PI / (double)k->g->npix;
    d.nr = k->g->nr;
    d.x = jb.x;
    d.y = jb.y;
    d.stride = jb.stride;
    d.batch = (int)jb.batch;
    d.n4 = (int)(4 * k->g->nside);
    return d;
}

// The job's belt fields; w is the per-call weight workspace (rows or ring pairs).
JobDesc belt_desc(const SkJob &jb, float *w) {
    const sk_kern *k = jb.k;
    JobDesc d = base_desc(jb);
    d.b_lo = k->b_lo; d.nb = k->nb; d.HM = k->HM; d.WPM = k->WPM;
    d.EMIN = k->EMIN; d.EMAX = k->EMAX;
    d.bgrp = k->d_bgrp;
    d.smax = k->smax; d.bpr = k->d_bpr; d.bwp = reinterpret_cast<const float2 *>(w);
    return d;
}

// Collects jobs for one kernel family and launches them SK_MAXJ at a time.
struct Batcher {
    JobsArg a;
    Batcher() { reset(); }
    void reset() { memset(&a, 0, sizeof a); }
    bool full() const { return a.n_jobs == SK_MAXJ; }
    void add(JobDesc d, const int4 *items, int n_items) {
        d.items = items;
        d.n_items = n_items;
        d.flat_base = a.total;
        a.j[a.n_jobs++] = d;
        a.total += n_items * d.batch;
    }
};

int grid_for(int total, int per_sm, int sms) {
    int g = std::max(1, per_sm) * sms;
    return std::min(total, g);
}

}  // namespace

int sk_capw_build(sk_kern *k, bool force, cudaStream_t st, const int *gate) {
    if (!k->plan_ok || k->capw_len == 0 || !k->capw_wanted) {
        sk_capw_free(k);
        return SK_OK;
    }
    const size_t bytes = (size_t)k->capw_len * sizeof(float4);
    if (!k->d_capw) {
        // the weights are a cache of the operator: unless asked for, build them only where
        // they leave half of the free device memory to the maps and workspaces
        size_t free_b = 0, total_b = 0;
        SK_CU(cudaMemGetInfo(&free_b, &total_b));
        if (!force && bytes > free_b / 2) return SK_OK;
        if (cudaMalloc(&k->d_capw, bytes) != cudaSuccess) {
            cudaGetLastError();
            k->d_capw = nullptr;
            return SK_OK;
        }
    }
    SkJob jb{k, nullptr, nullptr, 1, 0};
    for (int c = 0; c < SK_CAP_LS_CLASSES; ++c)
        for (int v = 0; v < 2; ++v) {
            const int n = k->n_items_cap[c][v];
            if (n == 0) continue;
            JobsArg a;
            memset(&a, 0, sizeof a);
            a.j[0] = base_desc(jb);
            a.j[0].items = k->d_items_cap[c][v];
            a.j[0].n_items = n;
            a.j[0].capw_ring = k->d_capw_ring;
            a.n_jobs = 1;
            a.total = n;
            const int mode = v | (k->kp.small_angle ? 2 : 0) | (k->layout == SK_NODES_BIASED ? 4 : 0);
            const int grid = std::min((n + 3) / 4, 8 * k->ctx->num_sms);
            if (k->blocked)
                SK_CU(sk_launch_capw_build64(a, k->d_capw, grid, st, gate));
            else
                SK_CU(sk_launch_capw_build(a, mode, k->d_capw, grid, st, gate));
        }
    return SK_OK;
}

int sk_beltw_build(sk_kern *k, cudaStream_t st, const int *gate) {
    if (!k->plan_ok || k->nb == 0) return SK_OK;
    if (!k->d_beltw) {
        const size_t bytes = (size_t)k->ngroups * k->smax * SK_BELT_WARPS * k->WPM * sizeof(float2);
        if (cudaMalloc(&k->d_beltw, bytes) != cudaSuccess) {
            cudaGetLastError();
            k->d_beltw = nullptr;                   // the pre-pass stays per call
            return SK_OK;
        }
    }
    SkJob jb{k, nullptr, nullptr, 1, 0};
    SK_CU(sk_launch_belt_pairs(belt_desc(jb, nullptr), 0, k->ngroups, k->d_beltw, st, gate, k->blocked));
    return SK_OK;
}

int sk_tca_build(sk_kern *k, int form, cudaStream_t st, const int *gate) {
    TcPlan &T = k->tcp[form];
    if (!T.ok) return SK_OK;
    if (!T.d_A) {
        if (gate) return SK_OK;                     // built on first use, from the table then
        if (cudaMalloc(&T.d_A, (size_t)T.kb * 1024) != cudaSuccess) {
            cudaGetLastError();
            T.d_A = nullptr;                        // that form runs the FP32 belt
            return SK_OK;
        }
    }
    TcTileArgs a;
    memset(&a, 0, sizeof a);
    a.tiles = T.d_tiles;
    a.tile_group = T.d_group;
    a.A = T.d_A;
    a.rings = k->g->d_rings;
    a.pair_off = k->d_pair_off;
    a.pairs = k->d_pairs;
    a.kp = k->kp;
    a.tab = k->d_tab;
    a.b_lo = k->b_lo;
    a.nb = k->nb;
    a.n4 = (int)(4 * k->g->nside);
    a.bf16 = form;
    SK_CU(sk_launch_tc_tiles(a, (int)T.h_tiles.size(), st, gate));
    return SK_OK;
}

int sk_run_jobs(sk_ctx *ctx, const SkJob *jobs, int n, int path, void *ws, cudaStream_t st) {
    // jobs whose belt runs on the tensor cores (their A tiles are built on first use; a
    // ring subset runs the tile groups of its belt rings)
    std::vector<int> use_tc(n, -1);            // the form, or -1
    for (int i = 0; i < n; ++i) {
        sk_kern *k = const_cast<sk_kern *>(jobs[i].k);
        const int f = sk_job_wants_tc(jobs[i], path);
        if (f < 0) continue;
        if (!k->tcp[f].d_A) {
            int rc = sk_tca_build(k, f, st);
            if (rc) return rc;
        }
        if (k->tcp[f].d_A) use_tc[i] = f;
    }

    // belt weight rows of the FP32 belt: stored with the operator, else one pre-pass
    // per job into the workspace, shared by all its maps
    std::vector<float *> wrows(n, nullptr);
    char *wp = (char *)ws;
    if (path != SK_PATH_GENERAL) {
        for (int i = 0; i < n; ++i) {
            const sk_kern *k = jobs[i].k;
            if (!k->plan_ok || k->nb == 0 || jobs[i].batch == 0) continue;
            wrows[i] = (float *)wp;
            wp += sk_plan_workspace_bytes(k);
            if (use_tc[i] >= 0) continue;
            if (k->d_beltw) {
                wrows[i] = (float *)k->d_beltw;
                continue;
            }
            if (!jobs[i].weights) continue;             // rows already in the workspace
            JobDesc d = belt_desc(jobs[i], nullptr);
            cudaEvent_t ev = sk_prof_begin(ctx, st);
            // ring pairs: the groups a ring subset runs (one or two ranges), or all
            const SkItems *sub = jobs[i].sub;
            if (!sub || sub->bg[0][1] < 0) {
                SK_CU(sk_launch_belt_pairs(d, 0, k->ngroups, (float2 *)wrows[i], st, nullptr, k->blocked));
            } else {
                for (int q = 0; q < 2; ++q)
                    if (sub->bg[q][1] > sub->bg[q][0])
                        SK_CU(sk_launch_belt_pairs(d, sub->bg[q][0], sub->bg[q][1], (float2 *)wrows[i], st, nullptr,
                                                   k->blocked));
            }
            sk_prof_end(ctx, "belt_weights", ev, st);
        }
    }

    // The polar cap rings of the evaluating kernels and any per-pair rings are small
    // launches: run them on the context's side stream, forked from `st` here (after the
    // belt weight rows, so that the belt is launched before the polar caps take SMs) and
    // joined back at the end.  The symmetric copies of the maps' cap input rings (in the
    // workspace after the belt rows of all jobs) go first: on the side stream, beside the
    // FP32 belt (whose blocks take work from a grid-stride loop), or on `st` before the
    // tensor-core belt, whose one CTA per SM runs a fixed share of the items and would
    // wait for SMs the copies hold (a band run of the host-buffer path builds its band's
    // rings).
    cudaStream_t side = ctx->aux;
    bool any_tc = false;
    for (int i = 0; i < n; ++i) any_tc = any_tc || use_tc[i] >= 0;
    cudaStream_t sym_st = any_tc ? st : side;
    std::vector<float4 *> hx(n, nullptr);
    auto sym = [&](int i, int r0, int r1, cudaStream_t s) -> int {
        if (r1 <= r0) return SK_OK;
        JobDesc d = base_desc(jobs[i]);
        d.hx = hx[i];
        d.hstride = jobs[i].k->sym_stride;
        cudaEvent_t ev = sk_prof_begin(ctx, s);
        SK_CU(sk_launch_cap_sym(d, r0, r1, jobs[i].k->d_capw ? 4 : 2, s));
        sk_prof_end(ctx, "cap_sym", ev, s);
        return SK_OK;
    };
    if (path != SK_PATH_GENERAL) {
        SK_CU(cudaEventRecord(ctx->ev_fork, st));
        SK_CU(cudaStreamWaitEvent(side, ctx->ev_fork, 0));
        char *hp = (char *)ws;
        for (int i = 0; i < n; ++i) hp += sk_plan_workspace_bytes(jobs[i].k);
        for (int i = 0; i < n; ++i) {
            const size_t bytes = sk_sym_bytes(jobs[i].k, jobs[i].batch);
            if (!bytes) continue;
            hx[i] = (float4 *)hp;
            hp += bytes;
            const SkItems *sub = jobs[i].sub;
            int rc = sub ? sym(i, sub->sym[0][0], sub->sym[0][1], sym_st) : sym(i, 0, jobs[i].k->sym_hi, sym_st);
            if (!rc && sub) rc = sym(i, sub->sym[1][0], sub->sym[1][1], sym_st);
            if (rc) return rc;
        }
    }

    if (path == SK_PATH_GENERAL) {
        Batcher b;
        auto flush = [&]() -> int {
            if (b.a.total > 0) {
                b.a.status = ctx->d_status;
                cudaEvent_t ev = sk_prof_begin(ctx, st);
                SK_CU(sk_launch_conv_general(b.a, grid_for(b.a.total, 16, ctx->num_sms), st));
                sk_prof_end(ctx, "conv_general", ev, st);
            }
            b.reset();
            return SK_OK;
        };
        for (int i = 0; i < n; ++i) {
            if (jobs[i].batch == 0) continue;
            b.add(base_desc(jobs[i]), jobs[i].k->d_items_all, jobs[i].k->n_items_all);
            if (b.full()) { int rc = flush(); if (rc) return rc; }
        }
        return flush();
    }

    // tensor-core belt: one launch per job over all its maps, reading the maps directly
    {
        for (int i = 0; i < n; ++i) {
            const int f = use_tc[i];
            if (f < 0) continue;
            const sk_kern *k = jobs[i].k;
            const TcPlan &T = k->tcp[f];
            int gr[4];
            job_groups(jobs[i], gr);
            if (gr[1] <= gr[0] && gr[3] <= gr[2]) continue;       // a subset without belt rings
            TcArgs a;
            memset(&a, 0, sizeof a);
            a.rings = k->g->d_rings;
            a.y = jobs[i].y;
            a.stride = jobs[i].stride;
            a.batch = (int)jobs[i].batch;
            a.b_lo = k->b_lo;
            a.nb = k->nb;
            a.n4 = (int)(4 * k->g->nside);
            a.tiles = T.d_tiles;
            a.trng = T.d_rng;
            a.A = T.d_A;
            a.x = jobs[i].x;
            a.nn = T.nn;
            a.nblk = T.nblk;
            a.kmax = T.kmax;
            a.nstages = T.stages;
            a.bf16 = f;
            a.ga0 = gr[0]; a.ga1 = gr[1]; a.gb0 = gr[2]; a.gb1 = gr[3];
            a.total = ((gr[1] - gr[0]) + (gr[3] - gr[2])) * (int)jobs[i].batch * T.nblk;
            a.status = ctx->d_status;
            a.queue = ctx->d_queue + ctx->next_queue;
            ctx->next_queue = (ctx->next_queue + 1) % sk_ctx::NQUEUE;
            SK_CU(cudaMemsetAsync(a.queue, 0, sizeof(int), st));
            cudaEvent_t ev = sk_prof_begin(ctx, st);
            SK_CU(sk_launch_belt_tc(a, std::min(a.total, ctx->num_sms), st));
            sk_prof_end(ctx, f ? "conv_belt_bf16" : "conv_belt_tc", ev, st);
        }
    }

    // belt: one launch family per (tile width P, blocked summation)
    const int Ps[] = {5, 7, 9, 11, 13, 15, 17};
    for (int blk = 0; blk < 2; ++blk)
    for (int P : Ps) {
        Batcher b;
        auto flush = [&]() -> int {
            if (b.a.total > 0) {
                b.a.status = ctx->d_status;
                int per = sk_belt_blocks_per_sm(b.a, P, blk != 0);
                cudaEvent_t ev = sk_prof_begin(ctx, st);
                SK_CU(sk_launch_conv_belt(b.a, P, blk != 0, grid_for(b.a.total, per, ctx->num_sms), st));
                sk_prof_end(ctx, "conv_belt", ev, st);
            }
            b.reset();
            return SK_OK;
        };
        for (int i = 0; i < n; ++i) {
            const sk_kern *k = jobs[i].k;
            if (!k->plan_ok || k->nb == 0 || k->belt_P != P || (int)k->blocked != blk || jobs[i].batch == 0)
                continue;
            if (use_tc[i] >= 0) continue;                         // done on the tensor cores
            const SkItems *sub = jobs[i].sub;
            const int4 *items = sub ? sub->belt : k->d_items_belt;
            const int n_items = sub ? sub->n_belt : k->n_items_belt;
            if (n_items == 0) continue;
            JobDesc d = belt_desc(jobs[i], wrows[i]);
            b.add(d, items, n_items);
            if (b.full()) { int rc = flush(); if (rc) return rc; }
        }
        int rc = flush();
        if (rc) return rc;
    }

    // caps; the launches wait for the copies.  Jobs with stored weights: one launch per
    // strip class, any tables together, the items of rings with wide windows (the polar
    // rings: few items, each a long run of whole-ring strips) first, so that the work queue
    // hands them out before the many narrow-window items.  The launch with the most items
    // runs on `st`; the others (a wide cut's short strip classes: a few blocks, some of them
    // one long item) go first, on the side stream, so that their blocks run beside it
    // rather than before it with most of the GPU idle -- the big launch's blocks take items
    // from its queue, so those that start late take fewer.  With one launch, no launch
    // beside the tensor-core belt holds SMs its static schedule is waiting for.
    SK_CU(cudaEventRecord(ctx->ev_sym, side));
    SK_CU(cudaStreamWaitEvent(st, ctx->ev_sym, 0));
    {
        struct CapwLaunch { JobsArg a; int c, blk; };
        std::vector<CapwLaunch> cl;
        for (int c = 0; c < SK_CAP_LS_CLASSES; ++c)
            for (int blk = 0; blk < 2; ++blk) {
                Batcher b;
                auto flush = [&]() {
                    if (b.a.total > 0) cl.push_back(CapwLaunch{b.a, c, blk});
                    b.reset();
                };
                for (int v = 0; v < 2; ++v)
                for (int i = 0; i < n; ++i) {
                    const sk_kern *k = jobs[i].k;
                    const SkItems *sub = jobs[i].sub;
                    const int4 *citems = sub ? sub->cap[c][v] : k->d_items_cap[c][v];
                    const int cn = sub ? sub->n_cap[c][v] : k->n_items_cap[c][v];
                    if (!k->plan_ok || !k->d_capw || (int)k->blocked != blk || cn == 0 || jobs[i].batch == 0)
                        continue;
                    JobDesc d = base_desc(jobs[i]);
                    d.cap_ls = SK_CAP_LS[c];
                    d.hx = hx[i];
                    d.hstride = k->sym_stride;
                    d.capw = k->d_capw;
                    d.capw_ring = k->d_capw_ring;
                    b.add(d, citems, cn);
                    if (b.full()) flush();
                }
                flush();
            }
        size_t main_l = 0;
        for (size_t l = 1; l < cl.size(); ++l)
            if (cl[l].a.total > cl[main_l].a.total) main_l = l;
        if (cl.size() > 1 && sym_st == st) {          // the side stream waits for the copies too
            SK_CU(cudaEventRecord(ctx->ev_sym, st));
            SK_CU(cudaStreamWaitEvent(side, ctx->ev_sym, 0));
        }
        auto launch = [&](CapwLaunch &L, cudaStream_t cs) -> int {
            L.a.status = ctx->d_status;
            cudaEvent_t ev = sk_prof_begin(ctx, cs);
            const int ipb = sk_capw_items_per_block(SK_CAP_LS[L.c], L.blk != 0);
            const int blocks = (L.a.total + ipb - 1) / ipb;
            int *q = ctx->d_queue + ctx->next_queue;
            ctx->next_queue = (ctx->next_queue + 1) % sk_ctx::NQUEUE;
            SK_CU(cudaMemsetAsync(q, 0, sizeof(int), cs));
            L.a.queue = q;
            SK_CU(sk_launch_conv_capw(L.a, SK_CAP_LS[L.c], L.blk != 0, std::min(blocks, ctx->num_sms), cs));
            sk_prof_end(ctx, "conv_capw", ev, cs);
            return SK_OK;
        };
        for (size_t l = 0; l < cl.size(); ++l)
            if (l != main_l) { int rc = launch(cl[l], side); if (rc) return rc; }
        if (!cl.empty()) { int rc = launch(cl[main_l], st); if (rc) return rc; }
    }
    // jobs whose caps evaluate their weights: one launch family per (strip class, mode,
    // summation); wide-window jobs sum ring by ring into the running totals at the end of
    // the workspace (after the symmetric copies), one half per stream
    float *ctot = nullptr;
    if (ctot_bytes(jobs, n, path)) {
        char *p = (char *)ws;
        for (int i = 0; i < n; ++i) p += sk_plan_workspace_bytes(jobs[i].k) + sk_sym_bytes(jobs[i].k, jobs[i].batch);
        ctot = (float *)p;
    }
    const long long ctot_half = (long long)ctx->num_sms * 2048 * 32;
    for (int c = 0; c < SK_CAP_LS_CLASSES; ++c)
        for (int mode = 0; mode < 8; ++mode)
        for (int blk = 0; blk < 2; ++blk) {
            const int v = mode & 1;
            Batcher b;
            auto flush = [&]() -> int {
                if (b.a.total > 0) {
                    b.a.status = ctx->d_status;
                    int mnt = 2;
                    for (int j = 0; j < b.a.n_jobs; ++j) mnt = std::max(mnt, b.a.j[j].kp.nt);
                    int per = sk_cap_blocks_per_sm(SK_CAP_LS[c], mode, mnt);
                    cudaStream_t cs = v ? st : side;
                    cudaEvent_t ev = sk_prof_begin(ctx, cs);
                    // a block works on several items at a time
                    const int ipb = sk_cap_items_per_block(SK_CAP_LS[c]);
                    const int blocks = (b.a.total + ipb - 1) / ipb;
                    int *q = ctx->d_queue + ctx->next_queue;
                    ctx->next_queue = (ctx->next_queue + 1) % sk_ctx::NQUEUE;
                    SK_CU(cudaMemsetAsync(q, 0, sizeof(int), cs));
                    b.a.queue = q;
                    b.a.ctot = blk ? ctot + (v ? 0 : ctot_half) : nullptr;
                    // at most 2048 threads per SM: the totals' slice holds every thread of the grid
                    SK_CU(sk_launch_conv_cap(b.a, SK_CAP_LS[c], mode, grid_for(blocks, per, ctx->num_sms), cs));
                    sk_prof_end(ctx, v ? "conv_cap" : "conv_cap_polar", ev, cs);
                }
                b.reset();
                return SK_OK;
            };
            for (int i = 0; i < n; ++i) {
                const sk_kern *k = jobs[i].k;
                const SkItems *sub = jobs[i].sub;
                const int4 *citems = sub ? sub->cap[c][v] : k->d_items_cap[c][v];
                const int cn = sub ? sub->n_cap[c][v] : k->n_items_cap[c][v];
                if (!k->plan_ok || k->d_capw || cn == 0 || jobs[i].batch == 0) continue;
                if ((int)(k->blocked && ctot) != blk) continue;
                const int kmode = v | (k->kp.small_angle ? 2 : 0) | (k->layout == SK_NODES_BIASED ? 4 : 0);
                if (kmode != mode) continue;
                // one node table per launch (the blocks load it once)
                if (b.a.n_jobs > 0 && b.a.j[0].tab != k->d_tab) { int rc = flush(); if (rc) return rc; }
                JobDesc d = base_desc(jobs[i]);
                d.cap_ls = SK_CAP_LS[c];
                d.hx = hx[i];
                d.hstride = k->sym_stride;
                b.add(d, citems, cn);
                if (b.full()) { int rc = flush(); if (rc) return rc; }
            }
            int rc = flush();
            if (rc) return rc;
        }

    // general fallback rings
    {
        Batcher b;
        auto flush = [&]() -> int {
            if (b.a.total > 0) {
                b.a.status = ctx->d_status;
                cudaEvent_t ev = sk_prof_begin(ctx, side);
                SK_CU(sk_launch_conv_general(b.a, grid_for(b.a.total, 16, ctx->num_sms), side));
                sk_prof_end(ctx, "conv_general", ev, side);
            }
            b.reset();
            return SK_OK;
        };
        for (int i = 0; i < n; ++i) {
            const sk_kern *k = jobs[i].k;
            if (jobs[i].batch == 0) continue;
            const SkItems *sub = jobs[i].sub;
            const int4 *items = sub ? sub->gen : (k->plan_ok ? k->d_items_gen : k->d_items_all);
            const int ni = sub ? sub->n_gen : (k->plan_ok ? k->n_items_gen : k->n_items_all);
            if (ni == 0) continue;
            b.add(base_desc(jobs[i]), items, ni);
            if (b.full()) { int rc = flush(); if (rc) return rc; }
        }
        int rc = flush();
        if (rc) return rc;
    }
    SK_CU(cudaEventRecord(ctx->ev_join, side));
    SK_CU(cudaStreamWaitEvent(st, ctx->ev_join, 0));
    return SK_OK;
}

// Table-gradient workspace: FP64 bins, the caps' symmetric copy of x, the belt's
// ring-pair sums.
static size_t grad_bins_bytes(const sk_kern *k) { return (sizeof(double) * k->nt + 255) & ~(size_t)255; }
static size_t grad_belt_bytes(const sk_kern *k) {
    if (!k->plan_ok || k->nb == 0) return 0;
    return (sizeof(float) * (size_t)k->nb * (2 * k->HM + 1) * k->WPM + 255) & ~(size_t)255;
}
// The caps' (k, f) cache: with more maps than one pass of the cap gradient takes, each of
// its warps (two blocks per SM) keeps the (k, f) of its walk's steps over an output's windows,
// at most the longest walk of a cap ring and KF_MAX_STEPS.
constexpr int KF_MAX_STEPS = 2048;
static int grad_kf_steps(const sk_kern *k, long long batch) {
    if (!k->plan_ok || k->n_items_gcap == 0 || batch <= SK_GRAD_CAP_MAPS) return 0;
    return (int)std::min<long long>(k->gcap_walk, KF_MAX_STEPS);
}
static int grad_cap_grid(int num_sms) { return 2 * num_sms; }     // persistent: two blocks per SM
static size_t grad_kf_bytes(const sk_kern *k, long long batch, int num_sms) {
    return sizeof(int2) * 32 * (size_t)grad_kf_steps(k, batch) * grad_cap_grid(num_sms) *
           (SK_GRAD_CAP_THREADS / 32);
}
size_t sk_grad_workspace_bytes(const sk_kern *k, long long batch, int num_sms) {
    return grad_bins_bytes(k) + sk_sym_bytes(k, batch) + grad_belt_bytes(k) + grad_kf_bytes(k, batch, num_sms);
}

int sk_run_grad(sk_ctx *ctx, const sk_kern *k, const float *x, const float *gy, long long batch,
                long long stride, float *out, double *acc, cudaStream_t st) {
    SK_CU(cudaMemsetAsync(acc, 0, sizeof(double) * k->nt, st));
    if (batch > 0) {
        SkJob jb{k, x, nullptr, batch, stride};
        auto general = [&](const int4 *items, int n_items) -> int {
            if (n_items <= 0) return SK_OK;
            Batcher b;
            b.add(base_desc(jb), items, n_items);
            b.a.status = ctx->d_status;
            cudaEvent_t ev = sk_prof_begin(ctx, st);
            SK_CU(sk_launch_grad_general(b.a, gy, acc, grid_for(b.a.total, 8, ctx->num_sms), st));
            sk_prof_end(ctx, "grad_general", ev, st);
            return SK_OK;
        };
        if (!k->plan_ok) {
            if (int rc = general(k->d_items_all, k->n_items_all)) return rc;
        } else {
            // belt rings: ring-pair cross-correlations
            if (k->nb > 0) {
                JobDesc d = belt_desc(jb, nullptr);
                float *C = reinterpret_cast<float *>(reinterpret_cast<char *>(acc) + grad_bins_bytes(k) +
                                                     sk_sym_bytes(k, batch));
                std::vector<int> lo(k->nb), np(k->nb);
                for (int rb = 0; rb < k->nb; ++rb) {
                    const int o = k->b_lo + rb;
                    lo[rb] = k->h_pairs[k->h_pair_off[o]].ri;
                    np[rb] = k->h_pair_off[o + 1] - k->h_pair_off[o];
                }
                cudaEvent_t ev = sk_prof_begin(ctx, st);
                SK_CU(sk_launch_grad_belt(d, gy, C, acc, lo.data(), np.data(), st));
                sk_prof_end(ctx, "grad_belt", ev, st);
            }
            // cap rings: symmetric base pairs over x's symmetric copy (after the FP64 bins)
            if (k->sym_hi > 0) {
                JobDesc d = base_desc(jb);
                d.hx = reinterpret_cast<float4 *>(reinterpret_cast<char *>(acc) + grad_bins_bytes(k));
                const int kf_steps = grad_kf_steps(k, batch);
                int2 *kfc = kf_steps > 0 ? reinterpret_cast<int2 *>(reinterpret_cast<char *>(acc) + grad_bins_bytes(k) +
                                                                     sk_sym_bytes(k, batch) + grad_belt_bytes(k))
                                         : nullptr;
                d.hstride = k->sym_stride;
                cudaEvent_t ev = sk_prof_begin(ctx, st);
                SK_CU(sk_launch_cap_sym(d, 0, k->sym_hi, 2, st));
                sk_prof_end(ctx, "cap_sym", ev, st);
                // every strip class's items in one launch, the longest walks first, so that the
                // polar rings' long tasks run beside the others rather than in a launch of their own
                if (k->n_items_gcap > 0) {
                    JobsArg a;
                    memset(&a, 0, sizeof a);
                    a.j[0] = d;
                    a.j[0].items = k->d_items_gcap;
                    a.j[0].n_items = k->n_items_gcap;
                    a.n_jobs = 1;
                    a.total = k->n_items_gcap;
                    a.status = ctx->d_status;
                    a.queue = ctx->d_queue + ctx->next_queue;
                    ctx->next_queue = (ctx->next_queue + 1) % sk_ctx::NQUEUE;
                    SK_CU(cudaMemsetAsync(a.queue, 0, sizeof(int), st));
                    ev = sk_prof_begin(ctx, st);
                    // persistent blocks (two per SM: 256 threads of 128 registers)
                    SK_CU(sk_launch_grad_cap(a, gy, acc, std::min(8 * a.total, grad_cap_grid(ctx->num_sms)), kfc,
                                             kf_steps, st));
                    sk_prof_end(ctx, "grad_cap", ev, st);
                }
            }
            // the other rings: per pixel
            if (int rc = general(k->d_items_gen, k->n_items_gen)) return rc;
        }
    }
    SK_CU(sk_launch_grad_finish(acc, k->nt, 4.0 * SK_PI / (double)k->g->npix, out, st));
    return SK_OK;
}
