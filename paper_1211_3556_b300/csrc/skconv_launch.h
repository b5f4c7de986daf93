// skconv_launch.h -- declarations shared by the library's .cu files: the job
// table every convolution kernel receives by value, and the launchers.
//
// A launch processes a flat list of work items.  Items of job j occupy flat
// indices [flat_base_j, flat_base_j + n_items_j * batch_j): map b of job j uses
// the job's per-map item list again.  Blocks stride over the flat list, so a
// launch is persistent (a grid sized to the GPU) and may mix jobs of different
// Nside, kernels and batch sizes.
#pragma once
#include <cuda_runtime.h>
#include "skconv_internal.cuh"

// Outputs with more window terms than this sum each input ring apart (blocked summation):
// plain FP32 accumulation of n terms drifts by about 1e-8 sqrt(n) relative, 5e-7 at the
// few hundred terms of the usual cuts and 1-3e-6 at the 2e4 of a 300' cut.
constexpr long long SK_BLOCKED_TERMS = 2000;
constexpr int SK_MAXJ = 16;            // jobs per launch (more: several launches)
constexpr int SK_MAX_NODES = 16384;    // largest kernel table
constexpr int SK_BELT_G = 16;          // output rings per belt block (two per consumer warp)
constexpr int SK_BELT_WARPS = SK_BELT_G / 2;   // consumer warps per belt block
constexpr int SK_BELT_STAGES = 20;     // input-ring strips in flight per belt block

struct JobDesc {
    // operator
    const RingDev *rings;
    const int *pair_off;
    const PairInfo *pairs;
    const float2 *tab;
    KernParams kp;
    KernParams64 kd;          // table gradient only
    const double2 *ab64;      // FP64 (A, B) per pair (table gradient, FP64-evaluated stored weights)
    const double *V64;        // FP64 node values and dOmega (FP64-evaluated stored weights)
    double dOmega;
    int nr;
    // maps
    const float *x;
    float *y;
    long long stride;
    int batch;
    // this launch's items of the job (one map's worth) and their flat range
    const int4 *items;
    int n_items;
    int flat_base;
    // belt (Toeplitz) path
    int b_lo;             // first belt output ring
    int nb;               // belt output rings
    int HM;               // max |input ring - output ring| over the belt
    int WPM;              // weights per (output ring, input ring) row: offsets EMIN .. EMIN+WPM-1, multiple of 4
    int EMIN, EMAX;       // pixel offset range of all belt windows
    int n4;               // pixels per belt ring (4 Nside)
    const int2 *bgrp;     // [groups] first and last input ring of each group
    // belt weights as ring pairs, streamed with the strips (FP32 CUDA-core path)
    int smax;             // strips per group in the pair layout (max over groups)
    const int2 *bpr;      // [groups][smax][SK_BELT_WARPS] (o, nch): the pair row covers offsets
                          // EMIN + o .. EMIN + o + 4 nch - 1 (union of both rows' windows)
    const float2 *bwp;    // [groups][smax][SK_BELT_WARPS][WPM]: element c = (weight of ring 2w, of
                          // ring 2w+1) at offset EMIN + o + c, zero past 4 nch
    // cap path
    int cap_ls;           // strip stride class
    float4 *hx;           // symmetric copy of the input rings the caps read (workspace, per call):
                          // ring r of map b at hx + b hstride + rings[r].start, n_r float4
    long long hstride;    // float4 per map of hx
    // stored cap weights (capw.cu): the weight stream, and per output ring (x) the float4
    // offset of the ring's first work item, (y) the pixel steps of one item
    const float4 *capw;
    const longlong2 *capw_ring;
};

struct JobsArg {
    int n_jobs;
    int total;            // flat items over all jobs
    int *status;          // device status word
    int *queue;           // work-queue counter (zero at launch) of kernels that take items dynamically
    float *ctot;          // evaluating caps of wide-window operators: per-thread running totals,
                          // [32][gridDim.x blockDim.x] floats (null: plain accumulation)
    JobDesc j[SK_MAXJ];
};

__device__ __forceinline__ int sk_find_job(const JobsArg &a, int f) {
    int j = 0;
    while (j + 1 < a.n_jobs && f >= a.j[j + 1].flat_base) ++j;
    return j;
}

// tensor-core belt (belt_tc.cu): items of SK_BELT_G rings x 8 nn pixels of one map
constexpr int SK_TC_MAX_STAGES = 6;
// tile field z: K in the low bits, and whether the tile starts / ends a chunk of tiles
// accumulated together (at least SK_TC_CHUNK_KSTEPS k-steps, or the group's last)
constexpr int SK_TC_K_MASK = 0xFFFF;
constexpr int SK_TC_FIRST = 1 << 16;
constexpr int SK_TC_LAST = 1 << 17;
constexpr int SK_TC_CHUNK_KSTEPS = 6;
struct TcArgs {
    const RingDev *rings;
    float *y;
    long long stride;
    int batch;
    int b_lo, nb, n4;
    const int4 *tiles;          // per tile: (input ring, E0, K | chunk flags, offset of its A pair in KB)
    const int4 *trng;           // per ring group: first tile, tiles, chunks, 0
    const unsigned char *A;     // stored A tiles (TF32 hi, then lo, no-swizzle K-major)
    const float *x;             // the maps (map b at x + b stride, rings as `rings` gives)
    int nn, nblk, kmax, nstages;
    int bf16;                   // 0: 3xTF32 (TF32 parts, 4-pixel operand rows), 1: BF16x3 (8-pixel rows)
    int ga0, ga1, gb0, gb1;     // the ring groups run: [ga0, ga1) then [gb0, gb1)
    int total;                  // items: groups x maps x pixel blocks
    int *queue;                 // the launch's item counter (zero at launch)
    int *status;
};
struct TcTileArgs {
    const int4 *tiles;
    const int *tile_group;
    unsigned char *A;
    const RingDev *rings;
    const int *pair_off;
    const PairInfo *pairs;
    KernParams kp;
    const float2 *tab;
    int b_lo, nb, n4;
    int bf16;
};
// pipeline stages for (kmax, nn, form) and the launch's shared memory; 0 = does not fit
int sk_tc_stages(int kmax, int nn, bool bf16, size_t *smem);
cudaError_t sk_launch_belt_tc(const TcArgs &a, int grid, cudaStream_t st);
// A tiles of all n_tiles tiles; with `gate`, only if *gate is non-zero
cudaError_t sk_launch_tc_tiles(const TcTileArgs &a, int n_tiles, cudaStream_t st, const int *gate = nullptr);

// set-up kernels (geometry.cu)
cudaError_t sk_launch_ring_geom(long long nside, RingDev *rings, double *z, double *rho,
                                double *theta, cudaStream_t st);
cudaError_t sk_launch_pair_ranges(int nr, const double *theta, double tc, int *lo, int *hi,
                                  cudaStream_t st);
cudaError_t sk_launch_pair_info(int nr, const RingDev *rings, const double *z, const double *rho,
                                const double *theta, const int *off, const int *lo, double tc,
                                PairInfo *pairs, double *dphimax, double2 *ab64, cudaStream_t st);
cudaError_t sk_launch_tabulate(const double *kl, int lmin, int lmax, int nt, double tc, int layout,
                               double taper_start, double *V, cudaStream_t st);
// (value, slope) dOmega table from FP64 nodes; with `gate`, only if *gate is non-zero
cudaError_t sk_launch_make_table(const double *V, int nt, double dOmega, float2 *tab, cudaStream_t st,
                                 const int *gate = nullptr);
// V = nv where they differ (one block, nt <= 16384); *changed = 1 if they did, else 0
cudaError_t sk_launch_update_values(const double *nv, double *V, int nt, int *changed, cudaStream_t st);
// in-cut pairs summed per class cls[ring] (total[0] if cls is null), or per output ring
cudaError_t sk_launch_count_pairs(int nr, int max_n, const RingDev *rings, const int *off,
                                  const PairInfo *pairs, const double *dphimax, const unsigned char *cls,
                                  unsigned long long *total, cudaStream_t st, bool per_ring = false);

// convolution kernels; grid = number of blocks (persistent)
cudaError_t sk_launch_conv_general(const JobsArg &a, int grid, cudaStream_t st);
// weight rows of belt ring groups [g0, g1) (the rows of other groups are not written);
// with `gate`, only if *gate is non-zero
// (w64: weights evaluated in FP64 -- pair_weight64 -- for operators with wide windows)
cudaError_t sk_launch_belt_pairs(const JobDesc &j, int g0, int g1, float2 *w, cudaStream_t st,
                                 const int *gate = nullptr, bool w64 = false);
size_t sk_belt_smem_bytes(int P, int wpm);   // dynamic shared memory of a belt block
// blocked: per-strip partial sums added to each output's total (operators with wide windows)
cudaError_t sk_launch_conv_belt(const JobsArg &a, int P, bool blocked, int grid, cudaStream_t st);
// mode bits: 1 sin series valid on every window of the items, 2 theta_cut <= 0.25
// (asin series), 4 biased node layout
cudaError_t sk_launch_conv_cap(const JobsArg &a, int ls, int mode, int grid, cudaStream_t st);
// symmetric copy (hx) of rings [r0, r1) of every map of job j, for the cap kernels, pixels
// split by residue modulo `split` (2: the evaluating kernel, 4: the stored-weight kernel)
cudaError_t sk_launch_cap_sym(const JobDesc &j, int r0, int r1, int split, cudaStream_t st);
int sk_belt_blocks_per_sm(const JobsArg &a, int P, bool blocked);
int sk_cap_blocks_per_sm(int ls, int mode, int nt);
constexpr int SK_CAP_LS_CLASSES = 3;
constexpr int SK_CAP_LS[SK_CAP_LS_CLASSES] = {288, 640, 1280};  // strip positions per row of the cap path (float4)
constexpr int SK_CAP_CT = 256;         // base output pixels per cap work item
// Pixel steps of a stored-weight cap thread on an input ring whose windows hold cnt
// pixels: the union of its four outputs' windows (they start at most ceil(3 n_i / n_o)
// pixels apart), rounded up to whole groups of four.
__host__ __device__ inline int sk_capw_steps(int cnt, int n_i, int n_o) {
    return (cnt + (3 * n_i + n_o - 1) / n_o + 3) & ~3;
}
// stored-weight cap kernel (capw.cu): items of one strip class; the jobs' hx hold the
// symmetric copies split by residue modulo 4
// blocked: each input ring's sums added to running totals (operators with wide windows)
cudaError_t sk_launch_conv_capw(const JobsArg &a, int ls, bool blocked, int grid, cudaStream_t st);
int sk_capw_items_per_block(int ls, bool blocked);
// weight streams of the items of a.j[0] (a kernel's cap items of one list) into w; mode as
// sk_launch_conv_cap
// the same stream with every weight evaluated in FP64 (operators with wide windows)
cudaError_t sk_launch_capw_build64(const JobsArg &a, float4 *w, int grid, cudaStream_t st,
                                   const int *gate = nullptr);
cudaError_t sk_launch_capw_build(const JobsArg &a, int mode, float4 *w, int grid, cudaStream_t st,
                                 const int *gate = nullptr);
int sk_cap_items_per_block(int ls);   // cap work items a block holds at a time (one node table)

// table gradient (grad.cu)
cudaError_t sk_launch_grad_general(const JobsArg &a, const float *gy, double *acc, int grid,
                                   cudaStream_t st);
cudaError_t sk_launch_grad_finish(const double *acc, int nt, double scale, float *out, cudaStream_t st);
// belt rings by ring-pair cross-correlations (j: the belt fields, x, batch, stride) into the
// FP32 sums C (sk_grad_belt_floats(j) floats), then the bins
size_t sk_grad_belt_floats(const JobDesc &j);
// h_lo, h_np: per belt output ring (rb = 0 .. nb - 1), the first ring of its window and
// the window's ring count (host arrays; the launch shapes depend on them)
cudaError_t sk_launch_grad_belt(const JobDesc &j, const float *gy, float *C, double *acc, const int *h_lo,
                                const int *h_np, cudaStream_t st);
// cap rings by symmetric base pairs (a.j[0]: the cap items, x's symmetric copy in hx)
// The caps' table gradient: GC = SK_GRAD_CAP_MAPS maps per pass over a warp's windows, blocks of
// SK_GRAD_CAP_THREADS; with more maps than one pass takes, each warp caches the (k, f) of the
// first kf_steps steps of its walk in kfc ([grid x warps per block][kf_steps][32] int2; null
// with kf_steps 0: no cache).
constexpr int SK_GRAD_CAP_MAPS = 4;
constexpr int SK_GRAD_CAP_THREADS = 256;
cudaError_t sk_launch_grad_cap(const JobsArg &a, const float *gy, double *acc, int grid, int2 *kfc, int kf_steps,
                               cudaStream_t st);
