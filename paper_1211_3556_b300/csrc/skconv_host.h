// skconv_host.h -- host-side handle structures and planner interface.
#pragma once
#include <cuda_runtime.h>
#include <stdarg.h>

#include <deque>
#include <mutex>
#include <string>
#include <vector>

#include "skconv.h"
#include "skconv_internal.cuh"
#include "skconv_launch.h"

constexpr int SK_HOST_BANDS = 24;  // ring bands of the host-buffer pipeline (sk_convolve_host; 16 / 24 / 32 measured 6.14 / 6.06 / 6.08 ms at Nside 2048)
constexpr int SK_MAX_RING_SUBSETS = 256;   // ring ranges whose work items an operator keeps

struct sk_ctx {
    int device = 0;
    int num_sms = 0;
    int *d_status = nullptr;       // device status word
    // work-queue counters of the cap launches (one per launch in flight, reused in turn;
    // each is zeroed on the launch's stream right before it)
    static constexpr int NQUEUE = 64;
    int *d_queue = nullptr;
    int next_queue = 0;
    void *ws = nullptr;            // reusable workspace (maps of sk_convolve_host, belt weights, grad bins)
    size_t ws_bytes = 0;
    size_t ws_limit = 0;           // cap on ws_bytes (sk_set_workspace_limit); 0: none
    // side stream for the small launches that overlap the large ones (polar caps,
    // per-pair fallback rings), forked from and joined into the caller's stream
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_sym = nullptr;  // the side stream's symmetric copies for the caps are built
    // optional per-launch timing (sk_profile_enable): events around each kernel
    bool prof = false;
    struct ProfRec { const char *name; cudaEvent_t a, b; };
    std::vector<ProfRec> prof_recs;
    // host-buffer pipeline: copy streams and per-band events (created on first use)
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t ev_in[SK_HOST_BANDS] = {}, ev_out[SK_HOST_BANDS] = {}, ev_done = nullptr;
};

// A subset of a kernel's work items (the output rings of one band); null lists mean
// "none of this path".
struct SkItems {
    const int4 *belt = nullptr;
    int n_belt = 0;
    const int4 *cap[SK_CAP_LS_CLASSES][2] = {};
    int n_cap[SK_CAP_LS_CLASSES][2] = {};
    const int4 *gen = nullptr;
    int n_gen = 0;
    // rings whose symmetric copy (the cap kernel's input) this subset's run builds:
    // [sym[0][0], sym[0][1]) and [sym[1][0], sym[1][1])
    int sym[2][2] = {};
    // belt ring groups whose weight rows the run needs: [bg[0][0], bg[0][1]) and
    // [bg[1][0], bg[1][1]) (a range and its mirror), or all when bg[0][1] < 0
    int bg[2][2] = {{0, -1}, {0, 0}};
};

struct sk_geom {
    sk_ctx *ctx = nullptr;
    int device = 0;                        // the context's device (the handle may outlive the context)
    long long nside = 0, npix = 0;
    int nr = 0;
    RingDev *d_rings = nullptr;
    double *d_z = nullptr, *d_rho = nullptr, *d_theta = nullptr;
    std::vector<RingDev> h_rings;
};

// One tensor-core form of the belt: one tile per (ring group, input ring) with
// (input ring, E0, K | chunk flags, A offset in KB), its group, and per group (first
// tile, tiles); the A store (hi/lo tiles, built when the form is first used and rebuilt
// with the table); the operand-row block (nn segments of 8 pixels) and its stages.
struct TcPlan {
    bool ok = false;
    std::vector<int4> h_tiles;
    int4 *d_tiles = nullptr;
    int *d_group = nullptr;
    int4 *d_rng = nullptr;                 // per group: first tile, tiles, chunks, 0
    long long kb = 0;
    unsigned char *d_A = nullptr;
    int kmax = 0, nn = 0, nblk = 0, stages = 0;
};

struct sk_kern {
    sk_ctx *ctx = nullptr;
    int device = 0;                        // the context's device (the handle may outlive the context)
    const sk_geom *g = nullptr;
    int nt = 0, layout = 0;
    double tc = 0.0;
    KernParams kp{};
    double *d_V = nullptr;                 // FP64 node values
    float2 *d_tab = nullptr;               // FP32 (value, slope) * dOmega
    int *d_pair_off = nullptr;
    PairInfo *d_pairs = nullptr;
    double *d_dphimax = nullptr;
    double2 *d_ab64 = nullptr;             // FP64 chord coefficients per pair (table gradient)
    KernParams64 kd{};
    int n_pairs = 0;
    std::vector<int> h_pair_off, h_lo, h_hi;
    std::vector<PairInfo> h_pairs;

    // every ring, 128 outputs per item: the per-pair path and the table gradient
    int4 *d_items_all = nullptr;
    int n_items_all = 0;

    // plan of the specialised paths
    bool plan_ok = false;
    int4 *d_items_gen = nullptr;           // rings neither belt nor cap covers
    int n_items_gen = 0;
    // belt
    int b_lo = 0, nb = 0, HM = 0, WPM = 0, EMIN = 0, EMAX = 0, ngroups = 0;
    int belt_P = 13;
    int2 *d_bgrp = nullptr;
    int smax = 0;                          // strips per group of the pair layout
    int2 *d_bpr = nullptr;                 // [groups][smax][warps] pair-row chunk ranges
    int4 *d_items_belt = nullptr;
    int n_items_belt = 0;
    // caps (one item list per strip class)
    // [strip class][sin series valid]
    int4 *d_items_cap[SK_CAP_LS_CLASSES][2] = {};
    int n_items_cap[SK_CAP_LS_CLASSES][2] = {};
    // the table gradient's cap items: every class in one list, the longest window walks
    // (window pixels summed over the ring's window rings) first; the longest walk
    int4 *d_items_gcap = nullptr;
    int n_items_gcap = 0;
    long long gcap_walk = 0;
    int n_cap_rings = 0;
    // the cap kernel reads the symmetric copy of input rings [0, sym_hi): sym_stride float4 per map
    int sym_hi = 0;
    long long sym_stride = 0;
    std::vector<unsigned char> h_ring_path;
    unsigned char *d_ring_path = nullptr;  // per output ring: 0 belt, 1 cap (either hemisphere) with
                                           // narrow windows, 3 cap with wide or whole-ring windows,
                                           // 2 general
    // stored cap weights (capw.cu): per output ring (float4 offset of its first item's
    // weights, pixel steps per item), the stream length in float4 (with the tail the
    // kernel's one-group-ahead loads read), and the stream itself -- null when the caps
    // evaluate their weights per call (sk_kernel_set_cap_weights)
    std::vector<longlong2> h_capw_ring;
    longlong2 *d_capw_ring = nullptr;
    long long capw_len = 0;
    float4 *d_capw = nullptr;
    bool capw_wanted = true;
    int *d_changed = nullptr;              // sk_kernel_update_values_async: whether the values changed
    // stored belt weights of the FP32 belt kernel (ring-pair rows of all groups, as the
    // pair-row pre-pass writes them), rebuilt with the table; null: the pre-pass runs
    // per call into the workspace
    float2 *d_beltw = nullptr;
    int belt_form = SK_BELT_FP32;          // the belt of SK_PATH_AUTO
    // outputs sum more than SK_BLOCKED_TERMS terms: the FP32 belt and the stored-weight
    // caps sum each input ring apart and add it to the output's total
    bool blocked = false;
    long long max_terms = 0;               // largest number of window pixels of one output
    // tensor-core belt forms (belt_tc.cu): [0] 3xTF32, [1] BF16x3
    TcPlan tcp[2];
    // host copies of the item lists, and their partition into ring bands by distance
    // from the nearest pole (sk_convolve_host overlaps the copies of one band with the
    // sums of another); rebuilt when the belt tile width changes
    std::vector<int4> h_items_belt, h_items_cap[SK_CAP_LS_CLASSES][2], h_items_gen;
    std::vector<int2> h_bgrp;              // per belt ring group: first and last input ring
    struct Band {
        int n_lo, n_hi, s_lo, s_hi;   // output rings [n_lo, n_hi) and [s_lo, s_hi)
        int need;                     // last band whose input rings the sums read
        int ready;                    // last band whose sums write output rings of this band
        SkItems items;
    };
    std::vector<Band> bands;
    int bands_P = 0;
    int4 *d_band_items = nullptr;
    // sk_convolve_rings: the work items writing output rings [lo, hi), per range asked for
    // (an entry per tile width; a deque keeps the entries in place as it grows, the mutex
    // guards it against concurrent first calls)
    struct RingSubset {
        int lo, hi, P;
        bool sym;                          // the range and its mirror about the equator
        int4 *d_items;
        SkItems items;
    };
    std::deque<RingSubset> subsets;
    std::mutex subsets_mu;
};

// api.cu
int sk_fail(int code, const char *fmt, ...);
cudaEvent_t sk_prof_begin(sk_ctx *ctx, cudaStream_t st);
void sk_prof_end(sk_ctx *ctx, const char *name, cudaEvent_t a, cudaStream_t st);
int sk_ctx_workspace(sk_ctx *ctx, size_t bytes, void **out);
// Argument checks of the map-taking entry points (null, batch, stride, alignment, overlap).
int sk_check_maps(const char *who, const sk_kern *k, const void *in, const void *out, int64_t batch,
                  int64_t stride, bool disjoint = true);

// plan.cu
int sk_plan_build(sk_kern *k);
// Stored cap weights: allocate (if absent) and evaluate the weight stream from the current
// node table on the legacy stream.  Without `force` the stream is only allocated if it
// takes at most half of the free device memory; a failed allocation leaves the caps
// evaluating their weights per call.
// With `gate`, the rebuild kernels run on `st` and return at once unless *gate is set.
int sk_capw_build(sk_kern *k, bool force = false, cudaStream_t st = 0, const int *gate = nullptr);
void sk_capw_free(sk_kern *k);
// Stored belt ring-pair rows: allocate (if absent) and evaluate from the current table
// (same gate and stream rules as sk_capw_build; an allocation that fails leaves the
// pre-pass per call).
int sk_beltw_build(sk_kern *k, cudaStream_t st = 0, const int *gate = nullptr);
// A tiles of a tensor-core belt form (0 3xTF32, 1 BF16x3): allocate (if absent; a failed
// allocation leaves that form to the FP32 belt) and evaluate them from the current table,
// gated as above.
int sk_tca_build(sk_kern *k, int form, cudaStream_t st = 0, const int *gate = nullptr);
void sk_plan_free(sk_kern *k);
int sk_plan_rebuild_belt_items(sk_kern *k);
size_t sk_plan_workspace_bytes(const sk_kern *k);
size_t sk_sym_bytes(const sk_kern *k, long long batch);   // symmetric copy of `batch` maps

// One job of a launch sequence.
struct SkJob {
    const sk_kern *k;
    const float *x;
    float *y;
    long long batch, stride;
    const SkItems *sub = nullptr;   // only these items (null: all of the kernel's)
    bool weights = true;            // run the belt weight pre-pass (else the workspace holds it)
};
// Partition of k's items into ring bands (kept in k; rebuilt when stale).
int sk_plan_bands(sk_kern *k);
// The items that write output rings [lo, hi) (kept in k; *out points into it).
// Work items that write rings [lo, hi), and with sym also the mirror rings
// [nr - hi, nr - lo) (a cap item, which writes a ring and its mirror, taken once).
int sk_plan_ring_subset(sk_kern *k, int lo, int hi, bool sym, const SkItems **out);
// Launch sequence of the forward operator for a set of jobs.  `ws` must hold
// sk_jobs_workspace_bytes(jobs, n, path) bytes: the belt weight rows of every job,
// then the symmetric copies of every job's maps for the caps, then (wide-window jobs
// whose caps evaluate their weights) the running totals of those launches.
size_t sk_jobs_workspace_bytes(const SkJob *jobs, int n, int path = SK_PATH_AUTO);
// The tensor-core form job j's belt runs under `path` (0 3xTF32, 1 BF16x3; given its
// tiles exist), or -1.
int sk_job_wants_tc(const SkJob &j, int path);
int sk_run_jobs(sk_ctx *ctx, const SkJob *jobs, int n, int path, void *ws, cudaStream_t st);
// Table gradient: `acc` is the start of sk_grad_workspace_bytes(k, batch, num_sms) bytes of
// workspace (the FP64 bins, the caps' symmetric copy of x, the belt's ring-pair sums, the
// caps' (k, f) cache).
size_t sk_grad_workspace_bytes(const sk_kern *k, long long batch, int num_sms);
int sk_run_grad(sk_ctx *ctx, const sk_kern *k, const float *x, const float *gy, long long batch,
                long long stride, float *out, double *acc, cudaStream_t st);

#define SK_CU(call)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return sk_fail(e_ == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA,           \
                           "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)
