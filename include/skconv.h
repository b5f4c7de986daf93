/*
 * skconv.h -- C ABI of the B300 real-space spherical convolution library.
 *
 * The operation (Sutter, Wandelt & Elsner, "Accelerating convolutions on the
 * sphere with hybrid GPU/CPU kernel splitting", Sec. 2, Eq. 1): a radially
 * symmetric kernel is split into a harmonic part K^_l (l <= l_cut) and a
 * compact real-space part K^_theta supported on [0, theta_cut].  This library
 * applies the real-space part to pixelised maps:
 *
 *   y_o = dOmega * sum_{i : gamma(o,i) <= theta_cut} K_lin(gamma(o,i)) * x_i,
 *   dOmega = 4 pi / Npix,  gamma(o,i) = angle between pixel centres,
 *
 * where K_lin interpolates the tabulated kernel linearly in theta between
 * nodes (Sec. 3: the tabulated real-space kernel, optionally with half of the
 * nodes in the first 1/16 of the support).  Maps are HEALPix RING-ordered
 * (the paper's pixelisation, Sec. 2), FP32, with the HEALPix library's pixel
 * numbering (the first pixel of an unshifted ring at phi = 0).
 *
 * Conventions for every entry point:
 *  - Return value: SK_OK (0) or a negative SK_E* code.  No exception crosses
 *    the ABI.  sk_last_error() gives a message for the calling thread.
 *  - Device pointers (d_*) are CUDA device addresses on the context's device,
 *    owned by the caller.  Map buffers are contiguous FP32 [batch][map_stride]
 *    with map_stride >= Npix; the first Npix entries of each row are the map in
 *    RING order.  Map pointers must be 16-byte aligned and map_stride a
 *    multiple of 4 (SK_EINVAL otherwise).  Input and output must not overlap
 *    (SK_EINVAL).
 *  - Host pointers (h_*) are ordinary host memory; page-locked memory gives the
 *    fastest copies.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Launches
 *    are asynchronous on it; device-side failures are recorded in the
 *    context's status word and reported by sk_get_status().
 *  - Handles (sk_ctx, sk_geom, sk_kern) are owned by the library and are
 *    immutable after creation apart from sk_kernel_set_tiles.  Calls that use
 *    the context's internal workspace (noted below) must not overlap on the
 *    GPU: issue them on one stream, or synchronise between streams.
 */
#ifndef SKCONV_H
#define SKCONV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SK_OK            0
#define SK_EINVAL       -1   /* bad argument: size, alignment, aliasing, NULL   */
#define SK_ENOMEM       -2   /* a device or host allocation failed              */
#define SK_ECUDA        -3   /* a CUDA runtime call failed                       */
#define SK_ETIMEOUT     -4   /* a bounded device-side wait gave up               */
#define SK_EUNSUPPORTED -5   /* valid but outside what this build supports       */

/* Node layouts of the tabulated kernel (Sec. 3). */
#define SK_NODES_UNIFORM   0  /* n nodes theta_k = k theta_cut / (n-1)                      */
#define SK_NODES_BIASED    1  /* nodes 0..n/2 uniform on [0, theta_cut/16], the rest uniform */
                              /* on [theta_cut/16, theta_cut]: half the nodes in 1/16 of the  */
                              /* support, the bias the paper uses for the oscillating kernel  */

/* Path selection for sk_convolve_path / sk_convolve_jobs / sk_graph_capture. */
#define SK_PATH_AUTO       0   /* belt Toeplitz + symmetric caps where they apply; the belt in */
                               /* the operator's form (sk_kernel_set_belt_form, the autotuner) */
#define SK_PATH_GENERAL    1   /* per-pair evaluation for every output ring        */
#define SK_PATH_TENSOR     2   /* as AUTO, with the belt as 3xTF32 tcgen05 contractions (ring  */
                               /* group x input ring weight tiles against 8-pixel segments of  */
                               /* the maps; caps stay FP32) where the operator has that form   */
#define SK_PATH_FP32       3   /* as AUTO, with the belt on the FP32 CUDA-core kernel          */
#define SK_PATH_BF16X3     4   /* as SK_PATH_TENSOR with BF16x3 products (BF16 hi/lo parts,    */
                               /* three kind::f16 MMAs): ~1e-5 relative, NOT within 1e-6      */

/* Belt forms of an operator (sk_kernel_set_belt_form). */
#define SK_BELT_FP32       0   /* FP32 FMAs, ring-pair weight rows streamed with the strips   */
#define SK_BELT_TENSOR     1   /* 3xTF32 tcgen05 MMAs (stored weight tiles x the maps read in sliding rows) */
#define SK_BELT_BF16X3     2   /* the same with BF16x3 products: about twice the MMA rate, ~1e-5 */
                               /* relative error (outside the 1e-6 bound; never chosen by the    */
                               /* autotuner)                                                     */

typedef struct sk_ctx  sk_ctx;
typedef struct sk_geom sk_geom;
typedef struct sk_kern sk_kern;

/* ---- context ------------------------------------------------------------ */

/* Bind a context to CUDA device `device` (makes it current on this thread).
 * The context owns a device status word and a reusable workspace.
 * Errors: SK_EINVAL (bad device), SK_ENOMEM, SK_ECUDA. */
int sk_create(sk_ctx **out, int device);
/* Release a context.  The handles made with it (geometries, operators, Fourier belts,
 * harmonic handles, resampling plans, graphs) may be destroyed before or after it --
 * each records its device -- but every other call on such a handle needs its context. */
int sk_destroy(sk_ctx *ctx);

/* Cap the context's workspace (the scratch memory that sk_convolve, sk_convolve_jobs,
 * sk_convolve_host, sk_grad_table and the ring-band calls grow on demand) at `bytes`;
 * 0 removes the cap (the default).  A call whose workspace would have to grow past the
 * cap fails with SK_ENOMEM before launching any kernel, and the context stays usable (a
 * later call under a higher cap, or no cap, succeeds).  The cap does not shrink a
 * workspace already allocated, and it does not cover the operator's own stored tables
 * (cap weights, tensor tiles), which fall back to their evaluated forms when they do
 * not fit.  Errors: SK_EINVAL (NULL context, bytes < 0). */
int sk_set_workspace_limit(sk_ctx *ctx, int64_t bytes);

/* Message of the last failed call on the calling thread ("" if none). */
const char *sk_last_error(void);

/* Synchronise `stream` and return the device status word (SK_OK, or e.g.
 * SK_ETIMEOUT recorded by a kernel), then clear it. */
int sk_get_status(sk_ctx *ctx, void *stream);

/* ---- geometry: HEALPix RING pixelisation (Sec. 2) ------------------------- */

/* 12 * nside^2; -1 if nside is not a power of two in [1, 8192]. */
int64_t sk_npix(int64_t nside);

/* Per-ring tables for `nside` (power of two, 1..8192), computed on the device
 * in FP64: pixel count, first pixel, phi shift, z = cos(theta), sin(theta).
 * Errors: SK_EINVAL (bad nside), SK_ENOMEM, SK_ECUDA. */
int sk_geometry_create(sk_ctx *ctx, int64_t nside, sk_geom **out);
int sk_geometry_destroy(sk_geom *g);

/* Copy the per-ring tables to the host (each array has 4*nside-1 entries;
 * any pointer may be NULL).  For tests and tooling. */
int sk_geometry_rings(const sk_geom *g, int32_t *h_n, int64_t *h_start, int32_t *h_shift,
                      double *h_z, double *h_sinth);

/* ---- tabulated real-space kernel K^_theta (Sec. 2 Eq. 1, Sec. 3) --------- */

/* Build the operator for geometry `g` from a kernel table: n_nodes FP64 node
 * values `h_values` (host; copied) on [0, theta_cut] in the given node layout.
 * theta_cut in radians, 0 < theta_cut <= pi.  Computes on the device the
 * per-ring-pair window bounds (which input rings and phi ranges can hold
 * pixels within theta_cut of each output ring) and the work plan.  The
 * geometry must outlive the operator.
 * Errors: SK_EINVAL (n_nodes < 2, or < 4 for the biased layout, bad
 * theta_cut or layout), SK_EUNSUPPORTED (n_nodes > 16384), SK_ENOMEM, SK_ECUDA. */
int sk_kernel_create(sk_ctx *ctx, const sk_geom *g, const double *h_values, int64_t n_nodes,
                     double theta_cut, int layout, sk_kern **out);

/* Tabulate the real-space part of the split of a kernel given by its Legendre
 * coefficients (Sec. 2, Eq. 1: K^_theta = the part of sum_l (2l+1)/(4pi) K_l
 * P_l(cos theta) above l_cut, truncated at theta_cut), on the device in FP64:
 *   V_k = taper(theta_k) * sum_{l=lmin}^{lmax} (2l+1)/(4 pi) h_kl[l] P_l(cos theta_k)
 * with taper = 1 for theta <= taper_start*theta_cut and a raised cosine down to
 * 0 at theta_cut (taper_start >= 1: no taper).  h_kl has lmax+1 entries (host).
 * Writes the n_nodes FP64 values to h_values_out (host) if it is not NULL and,
 * if `out` is not NULL, builds the operator as sk_kernel_create would.
 * Errors as sk_kernel_create, plus SK_EINVAL for lmin > lmax or lmax < 0. */
int sk_kernel_from_legendre(sk_ctx *ctx, const sk_geom *g, const double *h_kl, int64_t lmin,
                            int64_t lmax, int64_t n_nodes, double theta_cut, int layout,
                            double taper_start, double *h_values_out, sk_kern **out);
int sk_kernel_destroy(sk_kern *k);

/* Replace the node values of an operator (same count, cut and layout), e.g.
 * between training steps; the window tables are kept.  h_values: n_nodes FP64
 * (host; copied).  Synchronises the device.  Errors: SK_EINVAL, SK_ECUDA. */
int sk_kernel_update_values(sk_kern *k, const double *h_values);

/* Stored weights of the polar caps.  The operator does not change between calls, so
 * sk_kernel_create (and sk_kernel_update_values) evaluate the weights
 * dOmega K_lin(gamma) of the caps' symmetric base pairs once -- the same FP32 values,
 * bit for bit, that the sums would otherwise compute per call -- and keep them on the
 * device as a stream that the cap sums read (16 bytes per four base pairs, plus the
 * union windows' zeros: about 2.3 GB at Nside 2048 and theta_cut 20', 1/16 of the
 * cap pairs).  Results are bit-identical either way; stored weights make the caps'
 * sums bound by memory and shared-memory bandwidth instead of the weight evaluation.
 * At creation the stream is built only if it takes at most half of the free device
 * memory.  stored = 0 frees it (the caps then evaluate per call); stored = 1 builds it
 * (SK_ENOMEM if it does not fit).  Synchronises the device; not safe while k is in
 * use.  Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA. */
int sk_kernel_set_cap_weights(sk_kern *k, int stored);
/* Device bytes of k's stored cap weights (0: the caps evaluate per call). */
int sk_kernel_cap_weight_bytes(const sk_kern *k, int64_t *bytes);

/* Replace the node values from device memory, asynchronously on `stream`: d_values
 * holds n_nodes FP64 values (device; read on `stream`).  One kernel compares them with
 * the current values and takes them only if any differs; the (value, slope) table and
 * the stored cap weights are rebuilt on `stream` only then (their kernels return at
 * once otherwise).  No host synchronisation, so a training step that updates the table
 * can be captured in a CUDA graph.  Calls on `stream` after this one see the new
 * values; calls on other streams must be ordered after it by the caller, and calls
 * still running with k on other streams must finish before it.  The first call
 * allocates a 4-byte flag (make it before any stream capture).  When the values change
 * at every call, sk_kernel_set_cap_weights(k, 0) saves the weights' rebuild (one
 * evaluation of the cap weights per update).  Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA. */
int sk_kernel_update_values_async(sk_kern *k, const double *d_values, void *stream);

/* Number of ordered pixel pairs (o, i) with gamma(o,i) <= theta_cut, counted on
 * the device in FP64 from the per-ring-pair phi windows.  Blocks until done. */
int sk_count_pairs(sk_ctx *ctx, const sk_kern *k, int64_t *out);

/* Pair counts split by the path that evaluates each output ring:
 * out3[0] belt (ring-wise Toeplitz sums), out3[1] polar caps (one weight
 * evaluation for up to 16 symmetric pairs), out3[2] per-pair general path.  Their sum is
 * sk_count_pairs.  Blocks until done.  Errors: SK_EINVAL, SK_ECUDA. */
int sk_count_pairs_by_path(sk_ctx *ctx, const sk_kern *k, int64_t *out3);

/* The same counts split by the launch that sums them: out4[0] belt, out4[1] polar
 * caps with narrow windows (the main cap launch), out4[2] polar caps with wide or
 * whole-ring windows (the rings nearest the poles, summed on a side stream),
 * out4[3] per-pair general path.  Blocks until done.  Errors: SK_EINVAL,
 * SK_EUNSUPPORTED (no plan), SK_ECUDA. */
int sk_count_pairs_by_launch(sk_ctx *ctx, const sk_kern *k, int64_t *out4);

/* In-cut pairs of each output ring (out: rings entries, RING order) and, if path is not
 * NULL, each ring's path (rings entries: 0 belt, 1 cap, 2 per-pair, 3 cap with wide
 * windows) -- the costs a ring-band decomposition balances.  Blocks until done.
 * Errors: SK_EINVAL, SK_EUNSUPPORTED (path asked for without a plan), SK_ECUDA. */
int sk_count_pairs_by_ring(sk_ctx *ctx, const sk_kern *k, int64_t *out, uint8_t *path);

/* ---- convolution --------------------------------------------------------- */

/* y = A x for `batch` maps (the real-space convolution above).
 * d_in, d_out: [batch][map_stride] FP32 device buffers.  batch >= 0 (0 is a
 * no-op).  Inputs should be finite: some sums multiply pixels just outside an
 * output's window by a zero weight, so a NaN or Inf can reach outputs beyond its
 * cut -- within theta_cut plus a few pixels of it (the union windows of the caps and
 * of the belt's ring pairs, the tensor belt's 16-ring tiles); farther outputs are
 * unaffected.  Uses the context workspace.  Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA. */
int sk_convolve(sk_ctx *ctx, const sk_kern *k, const float *d_in, float *d_out,
                int64_t batch, int64_t map_stride, void *stream);

/* Same, choosing a path (SK_PATH_AUTO, SK_PATH_GENERAL or SK_PATH_TENSOR). */
int sk_convolve_path(sk_ctx *ctx, const sk_kern *k, const float *d_in, float *d_out,
                     int64_t batch, int64_t map_stride, int path, void *stream);

/* The outputs of rings [ring_lo, ring_hi) (0-based RING rings) of y = A x, for a
 * ring-band decomposition of one map over several devices (each device owns a band
 * of output rings and needs the input rings within theta_cut of it, a halo; the
 * rest of d_in may hold any finite values -- zeros, say -- but no NaN or Inf: some
 * sums multiply pixels outside an output's window by a zero weight, and 0 times NaN
 * is NaN).  Runs the work items that write those rings;
 * items that also write rings outside the range (a belt ring group across its
 * edge, the other hemisphere of a cap ring) write values there that depend on
 * inputs outside the halo: the caller keeps only its band.  In the range the
 * results are bit-identical to sk_convolve.  Arguments as sk_convolve.
 * Errors: SK_EINVAL (also a ring range outside [0, rings)), SK_ENOMEM, SK_ECUDA. */
int sk_convolve_rings(sk_ctx *ctx, const sk_kern *k, const float *d_in, float *d_out, int64_t batch,
                      int64_t map_stride, int ring_lo, int ring_hi, void *stream);

/* Planning: the first call for a ring range (and belt tile width) builds the range's
 * work-item lists on the device, which allocates and synchronises the device -- make
 * it before any stream capture.  The lists are kept on the operator for up to 256
 * ranges; the next new range then synchronises the device and drops them all (so
 * callers that vary the band edges do not grow device memory without bound).  Calls
 * for ranges of one operator from several host threads must not overlap with that
 * drop: plan every range once from one thread first. */

/* The same for rings [ring_lo, ring_hi) together with their mirror rings about the
 * equator, [rings - ring_hi, rings - ring_lo): a band made of a northern range and its
 * southern image.  A polar-cap work item sums a ring and its mirror at once, so a
 * symmetric band runs each such item once, where two one-sided bands would both run it.
 * The halo is the input rings within theta_cut of either range.  Otherwise as
 * sk_convolve_rings (the two ranges may overlap at the equator). */
int sk_convolve_rings_sym(sk_ctx *ctx, const sk_kern *k, const float *d_in, float *d_out, int64_t batch,
                          int64_t map_stride, int ring_lo, int ring_hi, void *stream);

/* Re-orientation of maps by a rotation (nearest-centre resampling), for partial-sky
 * maps moved onto the polar cap, where they occupy few rings and the real-space sums
 * touch only those (Sec. 4; with sk_convolve_rings).  For every output pixel p of
 * rings [ring_lo, ring_hi) (0-based): i = the pixel whose centre is nearest to the
 * direction M v_p (v_p the centre of p; ties to the lower index), and
 * d_out[b][p] = d_in[b][i] if ring(i) < src_ring_hi, else 0.  Other output pixels
 * are not written.  h_rot: host array of 9 doubles, M row-major, a rotation
 * (orthonormal to 1e-9).  Rotating the pole frame onto a field at (theta0, phi0)
 * and back: M and its transpose.  All geometry in FP64; the index decisions are
 * exact.  Maps as in sk_convolve (FP32, stride >= npix); d_in and d_out must not
 * overlap.  Errors: SK_EINVAL (also a ring range outside [0, rings], a matrix that
 * is not orthogonal, overlapping maps), SK_ECUDA. */
int sk_resample(sk_ctx *ctx, const sk_geom *g, const float *d_in, float *d_out, int64_t batch,
                int64_t map_stride, const double *h_rot, int ring_lo, int ring_hi, int src_ring_hi,
                void *stream);

/* Plan of a partial-sky field convolved on the polar cap (Sec. 4: a field re-oriented
 * onto the pole spans few rings).  Writes the rotation M = R_z(phi0) R_y(theta0) that
 * takes the pole to the field centre (theta0, phi0) (rot9, row-major FP64; resampling by
 * M moves the field onto the pole, by its transpose back), and four ring indices
 * (rings4, 0-based, ends exclusive): [0] out_hi -- the cap's output rings [0, out_hi)
 * reach colatitude radius plus two pixels (every sky pixel of the field has its nearest
 * rotated centre among them); [1] in_hi -- input rings [0, in_hi) within theta_cut of
 * those (1e-6 relative margin); [2], [3] sky_lo, sky_hi -- the sky rings that hold the
 * field (its colatitude band widened by one pixel, clamped to the poles).  With g NULL
 * only the rotation is written.  Host arithmetic (FP64); no device work.
 * Errors: SK_EINVAL (rot9 or rings4 NULL, radius <= 0, theta_cut <= 0). */
int sk_field_plan(const sk_geom *g, double theta0, double phi0, double radius, double theta_cut, double *rot9,
                  int32_t *rings4);

/* The same resampling planned once: the nearest-centre search depends on the
 * geometry, the rotation and the ring ranges only, so the plan keeps the kept
 * (output, source) pixel pairs (8 bytes each, on the device) and every apply is a
 * gather.  sk_resample_plan_apply(p, x, y) writes exactly what
 * sk_resample(.., x, y, .., same rotation and ranges) writes (masked outputs of the
 * ring range are cleared, then the pairs gathered).  The plan refers to the
 * geometry, which must outlive it.  info: out3[0] = kept pairs, out3[1] = output
 * pixels of the ring range, out3[2] = device bytes held.
 * Errors: as sk_resample; SK_ENOMEM when the pairs do not fit. */
typedef struct sk_resample_plan sk_resample_plan;
int sk_resample_plan_create(sk_ctx *ctx, const sk_geom *g, const double *h_rot, int ring_lo, int ring_hi,
                            int src_ring_hi, sk_resample_plan **out);
int sk_resample_plan_destroy(sk_resample_plan *p);
int sk_resample_plan_info(const sk_resample_plan *p, int64_t *out3);
int sk_resample_plan_apply(const sk_resample_plan *p, const float *d_in, float *d_out, int64_t batch,
                           int64_t map_stride, void *stream);

/* x_bar = A^T y_bar.  The kernel is radial, so A_oi = dOmega K_lin(gamma(o,i))
 * is symmetric and the transpose, written as a gather over the inputs of each
 * output, is the forward gather.  Same arguments and errors as sk_convolve. */
int sk_convolve_adjoint(sk_ctx *ctx, const sk_kern *k, const float *d_gy, float *d_gx,
                        int64_t batch, int64_t map_stride, void *stream);

/* Gradient of a loss with respect to the table nodes, given the input maps x
 * and dL/dy:  d_gtable[n] = dOmega sum_b sum_o gy_bo sum_{i in cut} x_bi dK_lin/dV_n,
 * dK_lin/dV_k = 1 - f, dK_lin/dV_{k+1} = f (linear interpolation, Sec. 3).
 * d_gtable: n_nodes FP32 device buffer (overwritten).  Partial sums are FP32
 * per block and reduced in FP64.  Uses the context workspace: the FP64 bins, the
 * caps' input rings in their symmetric layout (16 bytes per pixel and map), the
 * belt's ring-pair sums and, with more than four maps, a per-warp cache of the cap
 * pairs' node intervals (8 bytes per step of the longest cap walk, at most 2048
 * steps, x 32 lanes x 16 warps per SM; about 150 MB at Nside 1024, 30').
 * Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA. */
int sk_grad_table(sk_ctx *ctx, const sk_kern *k, const float *d_x, const float *d_gy,
                  int64_t batch, int64_t map_stride, float *d_gtable, void *stream);

/* The same table gradient without any device allocation.  There is no
 * counterpart in the paper: it exists for callers that cannot let a library
 * allocate device memory -- hosts whose device memory belongs to their own
 * allocator or budget, and latency-critical loops in which cudaMalloc or
 * cudaFree would synchronise the device.  Instead of the context workspace it
 * accumulates in a fixed FP64 array of 16384 entries compiled into the
 * library (128 KiB, held on every GPU that loads the library until the
 * process exits).  It always runs the per-pixel gradient kernel on every ring
 * (the belt and cap gradient kernels need workspace), so at large sizes it is
 * several times slower than sk_grad_table; results agree within rounding.  Arguments as sk_grad_table; n_nodes above 16384 is
 * rejected with SK_EINVAL.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  Every call clears the array before
 * using it, and all calls on a device share it: two calls whose work overlaps
 * on the GPU (e.g. on unordered streams) race and give wrong results.
 * Errors: SK_EINVAL, SK_ECUDA, SK_EUNSUPPORTED (device index above 63). */
int sk_grad_table_noalloc(sk_ctx *ctx, const sk_kern *k, const float *d_x, const float *d_gy,
                          int64_t batch, int64_t map_stride, float *d_gtable, void *stream);

/* End-to-end convolution from and to host memory: copies `batch` maps from
 * h_in to the context workspace, convolves, copies the result to h_out, and
 * synchronises `stream`.  h_in/h_out: [batch][map_stride] FP32 host buffers
 * (page-locked memory lets the copies overlap the sums).  The maps move in 16
 * ring bands ordered by distance from the poles: the sums of a band start once
 * the bands its windows reach have arrived, and a band's outputs go back once
 * the sums writing them are done, on two copy streams of the context beside
 * `stream`.  The bands' sums run the FP32 belt whatever the operator's belt form (a
 * band's few ring groups would underfill the tensor-core form, and the sums hide behind
 * the copies): the results are bit for bit those of sk_convolve_path with SK_PATH_FP32
 * on device buffers.  Uses the context workspace.  Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA. */
int sk_convolve_host(sk_ctx *ctx, const sk_kern *k, const float *h_in, float *h_out,
                     int64_t batch, int64_t map_stride, void *stream);

/* ---- many jobs in one launch, CUDA graphs -------------------------------- */

typedef struct {
    const sk_kern *k;      /* operator (its geometry decides Npix)             */
    const float *d_in;     /* [batch][map_stride] FP32 device                   */
    float *d_out;          /* [batch][map_stride] FP32 device                   */
    int64_t batch;
    int64_t map_stride;
} sk_job;

/* Convolve several jobs (mixed Nside, kernels, batch sizes) with one
 * persistent launch per path family that pulls (job, tile) items from a
 * device work queue, largest items first.  flags: SK_PATH_AUTO or
 * SK_PATH_GENERAL.  Uses the context workspace.
 * Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA. */
int sk_convolve_jobs(sk_ctx *ctx, const sk_job *jobs, int n_jobs, int flags, void *stream);

/* Capture the launches of sk_convolve_jobs(jobs) into a CUDA graph and
 * instantiate it; *graph_exec receives an opaque handle.  Replaying it with
 * sk_graph_launch runs the same jobs on the same buffers.  The work list the
 * graph reads is owned by the handle; free it with sk_graph_destroy. */
int sk_graph_capture(sk_ctx *ctx, const sk_job *jobs, int n_jobs, int flags, void *stream,
                     void **graph_exec);
int sk_graph_launch(void *graph_exec, void *stream);
int sk_graph_destroy(void *graph_exec);

/* ---- measurement ---------------------------------------------------------- */

/* Turn per-launch timing on or off for the context.  While on, every kernel the
 * library launches is bracketed by CUDA events on its stream (no work changes). */
int sk_profile_enable(sk_ctx *ctx, int on);

/* Collect the recorded launches (synchronising on their events) and clear
 * them: per kernel name, total milliseconds and launch count.  names receives
 * up to max_kernels NUL-terminated names of 32 bytes each.  *n_kernels is the
 * number of distinct kernels seen. */
int sk_profile_read(sk_ctx *ctx, int max_kernels, char *names, double *ms, int *launches,
                    int *n_kernels);

/* ---- measured peaks (denominators of the roofline fractions) -------------- */

/* Arithmetic forms whose peak rate sk_measure_peak measures. */
#define SK_PEAK_FFMA   0   /* FP32 fma.rn.f32: independent FMA chains in registers, 2 flop each      */
#define SK_PEAK_FFMA2  1   /* FP32 fma.rn.f32x2 (two FMAs per instruction), 2 flop per FMA          */
#define SK_PEAK_TF32   2   /* tcgen05.mma.kind::tf32, 128 x 256 x 8 per MMA from shared memory into  */
                           /* tensor memory, one block per SM, 2 flop per multiply-add              */

/* Measure the device's peak rate of one arithmetic form (no counterpart in the
 * paper; the rate the convolution's useful flops are compared against): runs
 * launches of a fixed amount of that arithmetic on `stream` for about
 * `seconds` (0 < seconds <= 60) and writes TFLOP/s to *tflops (CUDA-event time;
 * synchronises `stream`).  The clock the GPU ran at is the caller's to record.
 * Errors: SK_EINVAL (NULL, bad kind or seconds), SK_ENOMEM, SK_ECUDA; a
 * bounded wait of the TF32 form that gives up is reported by sk_get_status. */
int sk_measure_peak(sk_ctx *ctx, int kind, double seconds, double *tflops, void *stream);

/* Device properties the benchmark's peaks and grids use: out4[0] = SM count,
 * out4[1] = maximum SM clock in kHz, out4[2] = opt-in shared memory per block in
 * bytes, out4[3] = L2 bytes.  Errors: SK_EINVAL, SK_ECUDA. */
int sk_device_info(sk_ctx *ctx, int64_t *out4);

/* ---- tuning -------------------------------------------------------------- */

/* Set the tile parameters of operator k: belt_p = outputs per thread along a
 * belt ring (one of 5, 7, 9, 11, 13, 15, 17), cap_t = output pixels per cap tile
 * (64 or 128).  0 keeps the current value.  Used by the autotuner; not safe
 * while a launch with k is being issued from another thread.
 * Errors: SK_EINVAL. */
int sk_kernel_set_tiles(sk_kern *k, int belt_p, int cap_t);
int sk_kernel_get_tiles(const sk_kern *k, int *belt_p, int *cap_t);

/* Belt form of operator k used by SK_PATH_AUTO: SK_BELT_FP32 (the default),
 * SK_BELT_TENSOR or SK_BELT_BF16X3.  Choosing a tensor form evaluates its stored
 * weight tiles (synchronises the device; they follow later table updates).  Not safe
 * while a launch with k is being issued from another thread.
 * Errors: SK_EINVAL (bad form, or the operator has no such form: no belt, a ring
 * shorter than 128 pixels, or windows wider than the form's 64-column tiles allow),
 * SK_ENOMEM (the tiles do not fit), SK_ECUDA. */
int sk_kernel_set_belt_form(sk_kern *k, int form);

/* The operator's tuned settings: out4[0] = belt tile width P of the FP32 form,
 * out4[1] = belt form (SK_BELT_*), out4[2] = 1 if the cap weights are stored,
 * out4[3] = bit 0: the operator has the 3xTF32 tensor form, bit 1: the BF16x3 form.
 * Errors: SK_EINVAL. */
int sk_kernel_get_config(const sk_kern *k, int64_t *out4);

/* Autotuner: times, on the caller's maps (d_in -> d_out, `batch` maps), every
 * belt form -- the FP32 kernel with each tile width P and the tensor-core kernel
 * where the operator has one -- and then stored against evaluated cap weights
 * where the weights fit; keeps the fastest combination in k (read it back with
 * sk_kernel_get_config) and returns the FP32 tile width in *chosen.  If
 * cache_path is not NULL, a text file of "key P form capw" lines keyed by GPU
 * name, Nside, cut, node count, layout and batch is consulted first and appended
 * to after tuning.  Synchronises `stream`.  Not safe while k is used from
 * another thread.  Errors: as sk_convolve. */
int sk_kernel_autotune(sk_ctx *ctx, sk_kern *k, const float *d_in, float *d_out, int64_t batch,
                       int64_t map_stride, const char *cache_path, void *stream, int *chosen);

/* ---- self-test of device-side failure reporting --------------------------- */

/* Launch a kernel whose bounded wait on an mbarrier can never complete: after
 * `seconds` (0 < seconds <= 2) it records SK_ETIMEOUT in the context's status
 * word and returns, as the library's pipelined kernels do when a copy never
 * lands.  sk_get_status then reports SK_ETIMEOUT and the context stays usable.
 * Errors: SK_EINVAL, SK_ECUDA. */
int sk_selftest_wait_timeout(sk_ctx *ctx, double seconds, void *stream);

/* Self-test of the tensor-core building blocks the batched path uses: one block
 * computes D = A B^T (A: 128 x k, B: n x k, D: 128 x n, all row-major FP32 device
 * buffers) with tcgen05 TF32 MMAs from 128-byte-swizzled K-major shared-memory
 * operands into tensor memory; passes = 1 multiplies the TF32 parts only,
 * passes = 3 adds the hi*lo and lo*hi products (3xTF32).  n a multiple of 16 in
 * [16, 256], k a multiple of 32 in [32, 128].  Errors: SK_EINVAL, SK_ECUDA. */
int sk_selftest_tc_gemm(sk_ctx *ctx, const float *d_a, const float *d_b, float *d_d, int n, int k,
                        int passes, void *stream);

/* Self-test of the operand form of the tensor-core belt: one block computes
 * D[r][s] = sum_{k < K} A[r][k] x[8 s + k + off] (A: 128 x k row-major, x: at least
 * 8 (n + k/8 + 2) floats, D: 128 x n row-major; FP32 device buffers) with 3xTF32
 * tcgen05 MMAs from no-swizzle K-major shared-memory operands, x read as sliding
 * rows of three 16-byte-row planes.  n a multiple of 16 in [16, 256], k a multiple
 * of 8 in [8, 64], off 0 or 4.  Errors: SK_EINVAL, SK_ECUDA. */
int sk_selftest_tc_sliding(sk_ctx *ctx, const float *d_a, const float *d_x, float *d_d, int n, int k, int off,
                           void *stream);

/* The same product in the BF16x3 form of the tensor-core belt: A and x split into BF16
 * hi/lo parts, three kind::f16 MMAs of K = 16 per k-step, x read as sliding rows of one
 * plane of 8-value (16-byte) rows.  D[r][s] = sum_{k < K} A[r][k] x[8 s + k]; x at least
 * 8 (n + k/8) floats; n a multiple of 16 in [16, 256], k a multiple of 16 in [16, 64].
 * Errors: SK_EINVAL, SK_ECUDA. */
int sk_selftest_tc_sliding_bf16(sk_ctx *ctx, const float *d_a, const float *d_x, float *d_d, int n, int k,
                                void *stream);

/* ---- harmonic half of the split (Sec. 2, Eq. 1: the l <= l_cut part) ----
 *
 * The split convolution adds to the real-space sum above the harmonic part
 *
 *   y_p += sum_{l=0}^{L} sum_{m=-l}^{l} K^_l a_lm Y_lm(p),  a_lm = dOmega sum_q x_q Y*_lm(q),
 *
 * with L = l_cut and K^_l = K_l - R_l the l-space kernel the paper hands to a
 * spherical harmonic transform (R_l: the Legendre coefficients of the
 * real-space part).  The transform is a ring-based one on the same RING maps:
 * ring DFTs (cuFFT for the 2N+1 rings of 4N pixels, direct sums for the polar
 * cap rings), and Legendre sums against a table of the orthonormal associated
 * Legendre functions lambda_lm(theta_r), built once per handle (FP64
 * recurrence, stored FP32: (L+1)(L+2)/2 * 2N floats on the device).  Arithmetic
 * of the transforms is FP32. */
typedef struct sk_harm sk_harm;
#define SK_HARM_MAX_NSIDE 4096

/* Legendre coefficients of the real-space part, the R_l of K^_l = K_l - R_l
 * (Sec. 3: the l-space kernel is adjusted so that the two halves add up to K_l
 * for l <= l_cut): R_l = 2 pi int_0^theta_cut K_lin(theta) P_l(cos theta)
 * sin theta dtheta for l = 0..lmax, by 8-point Gauss-Legendre quadrature on
 * every node interval (exact for K_lin P_l sin up to the quadrature's degree),
 * FP64, into the host array h_R[lmax + 1] (synchronous).  lmax <= 65535.
 * Errors: SK_EINVAL, SK_ENOMEM, SK_ECUDA. */
int sk_kernel_response(sk_ctx *ctx, const sk_kern *k, int lmax, double *h_R);

/* The real-space part as a least-squares fit (Sec. 3: the real-space kernel
 * K^_theta is fit so that its harmonic transform matches K_l above l_cut; the
 * paper does not say how).  Unknowns: the values c_k of a piecewise-linear
 * kernel on the uniform nodes k theta_cut/(n_basis-1), k < n_basis-1, zero at
 * theta_cut.  Objective:
 *   sum_{l=0}^{lfit} w_l (2l+1) (R_l(c) - K_l)^2 + lam |c|^2,
 *   w_l = 1 for l > lcut, low_weight for l <= lcut (K^_l = K_l - R_l carries
 *   those; a small weight keeps the halves from carrying large cancelling parts),
 *   lam = reg * trace(normal matrix) / (n_basis - 1),
 * with R_l(c) by 8-point Gauss-Legendre per node interval (FP64 on the device),
 * solved by Cholesky of the normal equations (FP64, host).  h_kl[0..lfit]: K_l.
 * Output: h_V[nt_out] node values on nt_out uniform nodes of [0, theta_cut]
 * ((nt_out-1) a multiple of (n_basis-1): the table represents the fitted kernel
 * exactly), and *h_sigma_rms (may be NULL) =
 *   sqrt(sum_{l>lcut}^{lfit} (2l+1)(R_l - K_l)^2 / sum_{l<=lfit} (2l+1) K_l^2),
 * Eq. 2's sigma_rms relative to the kernel (without its factor alpha).
 * Errors: SK_EINVAL (ranges; a normal matrix that is not positive definite:
 * raise reg), SK_ENOMEM, SK_ECUDA. */
int sk_fit_real_kernel(sk_ctx *ctx, const double *h_kl, int lfit, int lcut, double theta_cut, int n_basis,
                       int nt_out, double low_weight, double reg, double *h_V, double *h_sigma_rms);

/* Builds the harmonic operator for geometry g: copies h_kl[0..lmax] (FP64
 * host array, K^_l) and tabulates lambda_lm on the device.
 * Errors: SK_EINVAL (NULL, lmax outside [0, 2 nside - 1]), SK_EUNSUPPORTED
 * (nside outside [2, SK_HARM_MAX_NSIDE]), SK_ENOMEM (the table does not fit),
 * SK_ECUDA.  *out is NULL on error. */
int sk_harmonic_create(sk_ctx *ctx, const sk_geom *g, const double *h_kl, int lmax, sk_harm **out);
int sk_harmonic_destroy(sk_harm *h);
/* Device bytes of the lambda table (for capacity planning). */
int sk_harmonic_table_bytes(const sk_harm *h, int64_t *bytes);
/* d_out = H d_in (accumulate = 0) or d_out += H d_in (accumulate != 0) for
 * `batch` maps [batch][map_stride]; H is the harmonic operator above.  Uses the
 * handle's own buffers (grown on demand): calls with one handle must not
 * overlap on the GPU.  Errors: SK_EINVAL (NULL, stride < Npix, misaligned,
 * aliasing), SK_ENOMEM, SK_ECUDA. */
int sk_harmonic_apply(sk_ctx *ctx, const sk_harm *h, const float *d_in, float *d_out, int64_t batch,
                      int64_t map_stride, int accumulate, void *stream);

/* Power spectra of maps by the handle's analysis (the spectra the paper extracts from
 * convolved uniform-noise maps to judge a split, Sec. 3):
 *   d_cl[b][l] = (|a_l0|^2 + 2 sum_{m=1}^{l} |a_lm|^2) / (2l + 1),  l = 0..lmax,
 * with a_lm = dOmega sum_q x_q Y*_lm(q) of map b, accumulated in FP64 from the FP32
 * transform.  d_cl: FP64 device [batch][lmax + 1].  Uses the handle's buffers: calls
 * with one handle must not overlap on the GPU.  Errors: as sk_harmonic_apply. */
int sk_harmonic_spectrum(sk_ctx *ctx, const sk_harm *h, const float *d_in, int64_t batch, int64_t map_stride,
                         double *d_cl, void *stream);

/* ---- ring-pair Fourier form of the belt, for wide theta_cut --------------- */

/* In the equatorial zone (rings of 4 Nside pixels) the real-space sum between
 * two rings is a circular correlation along the ring, diagonal in the ring's
 * Fourier modes m: Y_o(m) = sum_i W_oi(m) X_i(m) (the paper's Eq. 3 cost model
 * is linear in theta_cut; direct sums grow with its square).  The handle holds
 * W_oi(m) (as real G_oi(m) and a phase) for every output ring whose whole
 * window lies in the zone and every input ring of its window, built once from
 * FP64 weights through FP32 FFTs; the other rings (polar caps, rings whose
 * window leaves the zone) run through the kernel's direct paths.  Same
 * operator as sk_convolve (FP32 FFTs and mode sums: rms differences ~1e-7).
 * Device memory: f_nb (2H+1) (2 Nside + 1) floats for G, see sk_fourier_info.
 * Errors: SK_EINVAL (NULL), SK_ENOMEM, SK_ECUDA.  *out is NULL on error. */
typedef struct sk_fourier sk_fourier;
int sk_fourier_create(sk_ctx *ctx, const sk_kern *k, sk_fourier **out);
int sk_fourier_destroy(sk_fourier *f);
/* out4[0] = first output ring of the Fourier form (0-based), out4[1] = its number
 * of rings (0: none qualifies, all rings run direct), out4[2] = H (ring offsets
 * -H..H), out4[3] = device bytes of G. */
int sk_fourier_info(const sk_fourier *f, int64_t *out4);
/* d_out = A d_in for `batch` maps [batch][map_stride] (as sk_convolve), the zone
 * rings by the Fourier form.  Uses the handle's buffers: calls with one handle
 * must not overlap on the GPU.  Errors: as sk_convolve. */
int sk_fourier_apply(sk_ctx *ctx, const sk_fourier *f, const float *d_in, float *d_out, int64_t batch,
                     int64_t map_stride, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SKCONV_H */
