// patch.cu -- re-orientation of a map by a rotation, for partial-sky maps moved onto the
// polar cap.
//
// A survey that covers a small part of the sky can be rotated so that it sits on the
// north pole: there it occupies the first few HEALPix rings, and the real-space sums
// of its pixels (the in-cut neighbours of an output lie within theta_cut in
// colatitude) touch only those rings (Sec. 4).  The kernel is radial, so convolving
// the rotated map and rotating the result back is the convolution of the original
// map, up to the resampling of the pixel grid under the rotation.
//
// Resampling here is nearest-centre: output pixel p of rings [r_lo, r_hi) takes the
// value of the input pixel whose centre is nearest to the direction M v_p (v_p the
// centre of p, M a rotation), or 0 if that pixel lies on a ring at or beyond
// src_ring_hi.  The nearest centre is searched on the five rings around the
// direction's colatitude (ring spacing and in-ring pixel spacing are both below
// 1.3 / Nside rad, so the nearest centre is never more than two rings away from the
// ring closest in z), one candidate per ring: the pixel nearest in phi.  All in FP64;
// ties in distance go to the lower pixel index.  Index work is bit-exact; FP64 decides
// it.
//
// Outputs that can only land beyond the source limit skip the search: with c the third
// row of M, w_z = c . v_p, and every direction with w_z below the z of (continuous)
// ring src_ring_hi + 4 has all five candidate rings at or beyond the limit.  On an
// output ring those directions are the pixels farther than delta from the longitude of
// c, delta from one acos per block; two pixels of margin absorb its rounding.
//
// The search depends on the geometry and the rotation only, so a plan stores its result
// once (the (output, source) pairs that are kept, compacted with warp-aggregated
// atomics) and each application is a gather: HBM-bound, a few bytes per pixel.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "skconv.h"
#include "skconv_host.h"

namespace {

struct Rot {
    double m[9];
};

// 1-based ring whose z is nearest to zw (continuous estimate, within a ring).
__device__ __forceinline__ double ring_estimate(double zw, double N) {
    if (zw > 2.0 / 3.0) return N * sqrt(3.0 * (1.0 - zw));
    if (zw < -2.0 / 3.0) return 4.0 * N - N * sqrt(3.0 * (1.0 + zw));
    return N * (2.0 - 1.5 * zw);
}

// Index of the pixel whose centre is nearest to unit vector w.
__device__ long long nearest_pixel(double wx, double wy, double wz, long long N, int nr, const RingDev *rings,
                                   const double *z, const double *rho) {
    wz = fmin(1.0, fmax(-1.0, wz));
    const double rw = sqrt(wx * wx + wy * wy);
    double phw = atan2(wy, wx);
    if (phw < 0.0) phw += 2.0 * M_PI;
    const long long rc = llrint(ring_estimate(wz, (double)N));
    const int a = (int)max(1LL, rc - 2), b = (int)min((long long)nr, rc + 2);
    long long best = -1;
    double bestd = -2.0;
    for (int r = a; r <= b; ++r) {
        const RingDev R = rings[r - 1];
        // pixel j sits at phi = pi (2 j + s) / n: nearest j in phi
        const double jf = phw * R.n / (2.0 * M_PI) - 0.5 * R.s;
        long long j = llrint(jf);
        j %= R.n;
        if (j < 0) j += R.n;
        const double dph = phw - M_PI * (double)(2 * j + R.s) / R.n;
        const double d = wz * z[r - 1] + rw * rho[r - 1] * cos(dph);
        const long long p = R.start + j;
        if (d > bestd || (d == bestd && p < best)) {
            bestd = d;
            best = p;
        }
    }
    return best;
}

// Ring of pixel p (0-based), by bisection over the ring starts.
__device__ __forceinline__ int ring_of_pixel(long long p, int nr, const RingDev *rings) {
    int lo = 0, hi = nr - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rings[mid].start <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// z of the continuous (1-based) ring index rc: the inverse of ring_estimate.
__host__ __device__ inline double z_of_ring(double rc, double N) {
    if (rc <= N) return 1.0 - rc * rc / (3.0 * N * N);
    if (rc <= 3.0 * N) return 4.0 / 3.0 - 2.0 * rc / (3.0 * N);
    const double rs = 4.0 * N - rc;
    return -(1.0 - rs * rs / (3.0 * N * N));
}

// Half-width in phi, about the longitude of c, of the pixels of ring r whose direction
// can reach w_z >= zthr (negative: none; >= pi: all).
__device__ double reach_halfwidth(const Rot &M, double zr, double rr, double zthr) {
    const double cx = M.m[6], cy = M.m[7], cz = M.m[8];
    const double cr = sqrt(cx * cx + cy * cy);
    const double den = rr * cr;
    if (den < 1e-300) return cz * zr >= zthr ? 4.0 : -1.0;
    const double kap = (zthr - cz * zr) / den;
    if (kap > 1.0) return -1.0;
    if (kap < -1.0) return 4.0;
    return acos(kap);
}

// Source pixel of output pixel j of ring r (0-based), or -1 when it is masked.
struct Search {
    Rot M;
    long long N;
    int nr, src_hi;
    double zthr;          // w_z below this: masked without a search
    const RingDev *rings;
    const double *z, *rho;
};

__device__ long long source_of(const Search &S, int r, int j, const RingDev &R, double delta, double phic) {
    const double ph = M_PI * (double)(2 * j + R.s) / R.n;
    if (delta < M_PI) {
        double d = fabs(ph - phic);
        d = d > M_PI ? 2.0 * M_PI - d : d;
        if (delta < 0.0 || d > delta + 4.0 * M_PI / R.n) return -1;
    }
    double sp, cp;
    sincospi((double)(2 * j + R.s) / R.n, &sp, &cp);
    const double vx = S.rho[r] * cp, vy = S.rho[r] * sp, vz = S.z[r];
    const double *m = S.M.m;
    const double wx = m[0] * vx + m[1] * vy + m[2] * vz;
    const double wy = m[3] * vx + m[4] * vy + m[5] * vz;
    const double wz = m[6] * vx + m[7] * vy + m[8] * vz;
    // the rotation keeps |w| = 1 up to rounding: renormalise before the search
    const double inv = rsqrt(wx * wx + wy * wy + wz * wz);
    const long long src = nearest_pixel(wx * inv, wy * inv, wz * inv, S.N, S.nr, S.rings, S.z, S.rho);
    return ring_of_pixel(src, S.nr, S.rings) < S.src_hi ? src : -1;
}

// The block's ring, and the phi window of its pixels that need a search.
__device__ __forceinline__ void block_window(const Search &S, int r, double &delta, double &phic) {
    __shared__ double s_win[2];
    if (threadIdx.x == 0) {
        s_win[0] = S.zthr > -2.0 ? reach_halfwidth(S.M, S.z[r], S.rho[r], S.zthr) : 4.0;
        s_win[1] = atan2(S.M.m[7], S.M.m[6]);
    }
    __syncthreads();
    delta = s_win[0];
    phic = s_win[1] < 0.0 ? s_win[1] + 2.0 * M_PI : s_win[1];
}

// grid: (pixel blocks of the widest ring, rings r0 .. r0 + gridDim.y - 1)
__global__ void k_resample(const Search S, const float *x, float *y, long long batch, long long stride, int r0) {
    const int r = r0 + blockIdx.y;
    const RingDev R = S.rings[r];
    double delta, phic;
    block_window(S, r, delta, phic);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= R.n) return;
    const long long src = source_of(S, r, j, R, delta, phic);
    const long long dst = R.start + j;
    for (long long b = 0; b < batch; ++b) y[b * stride + dst] = src >= 0 ? x[b * stride + src] : 0.0f;
}

// The kept (output, source) pairs of the plan, compacted (a warp reserves its slots with
// one atomic, so a warp's pairs stay in pixel order).
__global__ void k_resample_pairs(const Search S, int r0, int2 *pairs, unsigned long long *count, long long p0) {
    const int r = r0 + blockIdx.y;
    const RingDev R = S.rings[r];
    double delta, phic;
    block_window(S, r, delta, phic);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const long long src = j < R.n ? source_of(S, r, j, R, delta, phic) : -1;
    const unsigned keep = __ballot_sync(0xffffffffu, src >= 0);
    if (!keep) return;
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == __ffs(keep) - 1) base = atomicAdd(count, (unsigned long long)__popc(keep));
    base = __shfl_sync(0xffffffffu, base, __ffs(keep) - 1);
    if (src >= 0) {
        const unsigned long long slot = base + __popc(keep & ((1u << lane) - 1u));
        pairs[slot] = make_int2((int)(R.start + j - p0), (int)src);
    }
}

// y[b][p0 + pair.x] = x[b][pair.y] for every kept pair and map.
__global__ void k_resample_gather(const int2 *__restrict__ pairs, long long n, const float *__restrict__ x,
                                  float *__restrict__ y, long long batch, long long stride, long long p0) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int2 pr = pairs[i];
        for (long long b = 0; b < batch; ++b) y[b * stride + p0 + pr.x] = __ldg(x + b * stride + pr.y);
    }
}

}  // namespace

static int check_rot(const double *h_rot, const char *who) {
    // a rotation: orthonormal rows (checked loosely: the caller's matrix is FP64)
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            const double d = h_rot[3 * i] * h_rot[3 * k] + h_rot[3 * i + 1] * h_rot[3 * k + 1] + h_rot[3 * i + 2] * h_rot[3 * k + 2];
            if (fabs(d - (i == k ? 1.0 : 0.0)) > 1e-9) return sk_fail(SK_EINVAL, "%s: matrix is not orthogonal", who);
        }
    return SK_OK;
}

static int check_range(const sk_geom *g, int ring_lo, int ring_hi, int src_ring_hi, const char *who) {
    if (ring_lo < 0 || ring_hi > g->nr || ring_lo > ring_hi || src_ring_hi < 0 || src_ring_hi > g->nr)
        return sk_fail(SK_EINVAL, "%s: ring range [%d, %d) or source limit %d outside [0, %d]", who, ring_lo, ring_hi,
                       src_ring_hi, g->nr);
    return SK_OK;
}

static Search make_search(const sk_geom *g, const double *h_rot, int src_ring_hi) {
    Search S;
    for (int i = 0; i < 9; ++i) S.M.m[i] = h_rot[i];
    S.N = g->nside;
    S.nr = g->nr;
    S.src_hi = src_ring_hi;
    // masked for sure below the z of ring src_ring_hi + 4 (1-based, continuous)
    S.zthr = src_ring_hi + 4 < g->nr ? z_of_ring(src_ring_hi + 4.0, (double)g->nside) : -4.0;
    S.rings = g->d_rings;
    S.z = g->d_z;
    S.rho = g->d_rho;
    return S;
}

static int widest_ring(const sk_geom *g, int lo, int hi) {
    int nmax = 0;
    for (int r = lo; r < hi; ++r) nmax = std::max(nmax, g->h_rings[r].n);
    return nmax;
}

extern "C" int sk_resample(sk_ctx *ctx, const sk_geom *g, const float *d_in, float *d_out, int64_t batch,
                           int64_t map_stride, const double *h_rot, int ring_lo, int ring_hi, int src_ring_hi,
                           void *stream) {
    if (!ctx || !g || !h_rot) return sk_fail(SK_EINVAL, "sk_resample: NULL argument");
    if (batch < 0 || map_stride < g->npix) return sk_fail(SK_EINVAL, "sk_resample: batch %lld, stride %lld below npix %lld",
                                                        (long long)batch, (long long)map_stride, g->npix);
    int rc = check_range(g, ring_lo, ring_hi, src_ring_hi, "sk_resample");
    if (!rc) rc = check_rot(h_rot, "sk_resample");
    if (rc) return rc;
    if (batch == 0 || ring_lo == ring_hi) return SK_OK;
    if (!d_in || !d_out) return sk_fail(SK_EINVAL, "sk_resample: NULL map");
    // the maps must not overlap: every output reads an arbitrary input pixel
    const char *a0 = (const char *)d_in, *a1 = a0 + sizeof(float) * (size_t)(map_stride * (batch - 1) + g->npix);
    const char *b0 = (const char *)d_out, *b1 = b0 + sizeof(float) * (size_t)(map_stride * (batch - 1) + g->npix);
    if (a0 < b1 && b0 < a1) return sk_fail(SK_EINVAL, "sk_resample: input and output overlap");
    SK_CU(cudaSetDevice(ctx->device));
    const Search S = make_search(g, h_rot, src_ring_hi);
    const int nmax = widest_ring(g, ring_lo, ring_hi);
    const int threads = 256;
    const cudaStream_t st = (cudaStream_t)stream;
    // grid.y is at most 65535 rings per launch
    for (int r0 = ring_lo; r0 < ring_hi; r0 += 65535) {
        const int nr = std::min(65535, ring_hi - r0);
        k_resample<<<dim3((nmax + threads - 1) / threads, nr), threads, 0, st>>>(S, d_in, d_out, batch, map_stride, r0);
        SK_CU(cudaGetLastError());
    }
    return SK_OK;
}

struct sk_resample_plan {
    sk_ctx *ctx = nullptr;
    int device = 0;                 // the context's device (the handle may outlive the context)
    const sk_geom *g = nullptr;
    int ring_lo = 0, ring_hi = 0;
    long long p0 = 0, p1 = 0;       // pixel range of the output rings
    int2 *d_pairs = nullptr;
    long long n_pairs = 0;
};

extern "C" int sk_resample_plan_create(sk_ctx *ctx, const sk_geom *g, const double *h_rot, int ring_lo, int ring_hi,
                                       int src_ring_hi, sk_resample_plan **out) {
    if (!ctx || !g || !h_rot || !out) return sk_fail(SK_EINVAL, "sk_resample_plan_create: NULL argument");
    *out = nullptr;
    int rc = check_range(g, ring_lo, ring_hi, src_ring_hi, "sk_resample_plan_create");
    if (!rc) rc = check_rot(h_rot, "sk_resample_plan_create");
    if (rc) return rc;
    SK_CU(cudaSetDevice(ctx->device));
    sk_resample_plan *p = new sk_resample_plan();
    p->ctx = ctx;
    p->device = ctx->device;
    p->g = g;
    p->ring_lo = ring_lo;
    p->ring_hi = ring_hi;
    p->p0 = ring_lo < g->nr ? g->h_rings[ring_lo].start : g->npix;
    p->p1 = ring_hi < g->nr ? g->h_rings[ring_hi].start : g->npix;
    const long long cap = p->p1 - p->p0;
    if (cap > 0) {
        int2 *tmp = nullptr;
        unsigned long long *d_count = nullptr, count = 0;
        cudaError_t e = cudaMalloc(&tmp, sizeof(int2) * cap);
        if (e == cudaSuccess) e = cudaMalloc(&d_count, sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemset(d_count, 0, sizeof(unsigned long long));
        const Search S = make_search(g, h_rot, src_ring_hi);
        const int nmax = widest_ring(g, ring_lo, ring_hi), threads = 256;
        for (int r0 = ring_lo; e == cudaSuccess && r0 < ring_hi; r0 += 65535) {
            const int nr = std::min(65535, ring_hi - r0);
            k_resample_pairs<<<dim3((nmax + threads - 1) / threads, nr), threads>>>(S, r0, tmp, d_count, p->p0);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpy(&count, d_count, sizeof count, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && count > 0) e = cudaMalloc(&p->d_pairs, sizeof(int2) * count);
        if (e == cudaSuccess && count > 0) e = cudaMemcpy(p->d_pairs, tmp, sizeof(int2) * count, cudaMemcpyDeviceToDevice);
        cudaFree(tmp);
        cudaFree(d_count);
        if (e != cudaSuccess) {
            cudaFree(p->d_pairs);
            delete p;
            return sk_fail(e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA, "sk_resample_plan_create: %s",
                           cudaGetErrorString(e));
        }
        p->n_pairs = (long long)count;
    }
    *out = p;
    return SK_OK;
}

extern "C" int sk_resample_plan_destroy(sk_resample_plan *p) {
    if (!p) return SK_OK;
    cudaSetDevice(p->device);
    cudaFree(p->d_pairs);
    delete p;
    return SK_OK;
}

extern "C" int sk_resample_plan_info(const sk_resample_plan *p, int64_t *out3) {
    if (!p || !out3) return sk_fail(SK_EINVAL, "sk_resample_plan_info: NULL argument");
    out3[0] = p->n_pairs;
    out3[1] = p->p1 - p->p0;
    out3[2] = (int64_t)sizeof(int2) * p->n_pairs;
    return SK_OK;
}

extern "C" int sk_resample_plan_apply(const sk_resample_plan *p, const float *d_in, float *d_out, int64_t batch,
                                      int64_t map_stride, void *stream) {
    if (!p) return sk_fail(SK_EINVAL, "sk_resample_plan_apply: NULL plan");
    const sk_geom *g = p->g;
    if (batch < 0 || map_stride < g->npix)
        return sk_fail(SK_EINVAL, "sk_resample_plan_apply: batch %lld, stride %lld below npix %lld", (long long)batch,
                       (long long)map_stride, g->npix);
    if (batch == 0 || p->p1 == p->p0) return SK_OK;
    if (!d_in || !d_out) return sk_fail(SK_EINVAL, "sk_resample_plan_apply: NULL map");
    const char *a0 = (const char *)d_in, *a1 = a0 + sizeof(float) * (size_t)(map_stride * (batch - 1) + g->npix);
    const char *b0 = (const char *)d_out, *b1 = b0 + sizeof(float) * (size_t)(map_stride * (batch - 1) + g->npix);
    if (a0 < b1 && b0 < a1) return sk_fail(SK_EINVAL, "sk_resample_plan_apply: input and output overlap");
    SK_CU(cudaSetDevice(p->ctx->device));
    const cudaStream_t st = (cudaStream_t)stream;
    // masked outputs are 0: clear the ring range of every map, then scatter the kept pairs
    if (p->n_pairs < p->p1 - p->p0)
        SK_CU(cudaMemset2DAsync(d_out + p->p0, sizeof(float) * (size_t)map_stride, 0,
                                sizeof(float) * (size_t)(p->p1 - p->p0), (size_t)batch, st));
    if (p->n_pairs > 0) {
        const long long blocks = std::min<long long>((p->n_pairs + 255) / 256, 148LL * 16);
        k_resample_gather<<<(int)blocks, 256, 0, st>>>(p->d_pairs, p->n_pairs, d_in, d_out, batch, map_stride, p->p0);
        SK_CU(cudaGetLastError());
    }
    return SK_OK;
}

// Colatitude of ring r (0-based) of the RING scheme (Sec. 2's pixelisation), FP64.
static double ring_theta(long long N, int r) {
    const long long i = r + 1;
    double z;
    if (i < N) z = 1.0 - (double)(i * i) / (3.0 * (double)N * (double)N);
    else if (i <= 3 * N) z = 4.0 / 3.0 - 2.0 * (double)i / (3.0 * (double)N);
    else {
        const long long ii = 4 * N - i;
        z = -(1.0 - (double)(ii * ii) / (3.0 * (double)N * (double)N));
    }
    return acos(fmin(1.0, fmax(-1.0, z)));
}

extern "C" int sk_field_plan(const sk_geom *g, double theta0, double phi0, double radius, double theta_cut,
                             double *rot9, int32_t *rings4) {
    if (!rot9 || !rings4) return sk_fail(SK_EINVAL, "sk_field_plan: NULL argument");
    if (!(radius > 0.0) || !(theta_cut > 0.0)) return sk_fail(SK_EINVAL, "sk_field_plan: radius and theta_cut > 0");
    const double ct = cos(theta0), st = sin(theta0), cp = cos(phi0), sp = sin(phi0);
    // R_z(phi0) R_y(theta0)
    const double m[9] = {cp * ct, -sp, cp * st, sp * ct, cp, sp * st, -st, 0.0, ct};
    for (int i = 0; i < 9; ++i) rot9[i] = m[i];
    if (!g) return SK_OK;
    const int nr = g->nr;
    const long long N = g->nside;
    const double pix = sqrt(4.0 * SK_PI / (double)g->npix);
    // the first ring whose colatitude exceeds t (rings are in increasing colatitude)
    auto upper = [&](double t) {
        int lo = 0, hi = nr;
        while (lo < hi) {
            const int mid = (lo + hi) / 2;
            if (ring_theta(N, mid) <= t) lo = mid + 1; else hi = mid;
        }
        return lo;
    };
    auto lower = [&](double t) {          // the first ring whose colatitude is at least t
        int lo = 0, hi = nr;
        while (lo < hi) {
            const int mid = (lo + hi) / 2;
            if (ring_theta(N, mid) < t) lo = mid + 1; else hi = mid;
        }
        return lo;
    };
    int out_hi = std::max(1, std::min(upper(radius + 2.0 * pix), nr));
    const double reach = ring_theta(N, out_hi - 1) + theta_cut + 1e-6 * std::max(1.0, theta_cut);
    int in_hi = std::max(out_hi, std::min(nr, upper(reach)));
    const double lo_t = theta0 - ring_theta(N, out_hi - 1), hi_t = theta0 + ring_theta(N, out_hi - 1);
    int sky_lo = std::max(0, lower(lo_t - pix)), sky_hi = std::min(nr, upper(hi_t + pix));
    if (lo_t <= 0.0) sky_lo = 0;
    if (hi_t >= SK_PI) sky_hi = nr;
    rings4[0] = out_hi;
    rings4[1] = in_hi;
    rings4[2] = sky_lo;
    rings4[3] = sky_hi;
    return SK_OK;
}
