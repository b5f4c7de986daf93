/*
 * skoracle.c -- FP64 CPU oracle for the real-space spherical convolution.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product imports, links or runs this
 * file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant with the CUDA
 * path.
 *
 * What it computes (the plain definition, FP64 throughout):
 *
 *   y_o = dOmega * sum_{i : gamma(o,i) <= theta_cut} K_lin(gamma(o,i)) * x_i,
 *   dOmega = 4 pi / Npix,
 *   gamma(o,i) = 2 asin(|p_o - p_i| / 2), p = unit vector of a pixel centre,
 *
 * i.e. the real-space half of the split convolution of Sec. 2, Eq. 1 (the
 * truncated real-space kernel K^_theta applied to a pixelised map), with the
 * kernel represented by nodes interpolated linearly in theta as described in
 * Sec. 3 (tabulated kernel, optional node bias putting half of the nodes in
 * the first 1/16 of the support).  Pixels are HEALPix RING-ordered (the paper's
 * data layout, Sec. 2; Gorski et al. 2005 for the pixelisation formulas).
 *
 * K_lin(theta): u = node coordinate of theta, k = min(floor(u), n-2),
 * f = u - k, K = V[k] + f (V[k+1] - V[k]).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846264338327950288

/* ---------------------------------------------------------------------- */
/* HEALPix RING geometry (Gorski et al. 2005), written from the definition. */
/* Rings r = 1 .. 4N-1; pixel j = 0 .. n_r-1 on a ring; phi = pi (2j + s) / n_r */
/* with s = 1 on shifted rings (all cap rings, belt rings with r - N even) and  */
/* s = 0 otherwise, so the first pixel of an unshifted ring sits at phi = 0    */
/* (the numbering of the HEALPix library: pixel 4 of Nside 1 is at phi = 0).  */
/* ---------------------------------------------------------------------- */

int64_t or_npix(int64_t nside) { return 12 * nside * nside; }

/* Ring r (1-based): number of pixels, first pixel index, phi shift s (0/1),
 * z = cos(theta), sin(theta). */
void or_ring_info(int64_t nside, int64_t r, int64_t *n, int64_t *start, int *s,
                  double *z, double *sinth)
{
    const int64_t N = nside, npix = 12 * N * N;
    const double N2 = (double)N * (double)N;
    if (r < N) {                       /* north polar cap */
        *n = 4 * r;
        *start = 2 * r * (r - 1);
        *s = 1;
        double omz = (double)(r * r) / (3.0 * N2);          /* 1 - z, exact form */
        *z = 1.0 - omz;
        *sinth = sqrt(omz * (2.0 - omz));
    } else if (r <= 3 * N) {           /* equatorial belt */
        *n = 4 * N;
        *start = 2 * N * (N - 1) + 4 * N * (r - N);
        *s = (int)((r - N + 1) % 2);
        *z = (double)(2 * (2 * N - r)) / (3.0 * (double)N);   /* 4/3 - 2r/(3N) */
        *sinth = sqrt((1.0 - *z) * (1.0 + *z));
    } else {                           /* south polar cap: mirror of 4N - r */
        int64_t rp = 4 * N - r;
        *n = 4 * rp;
        *start = npix - 2 * rp * (rp + 1);
        *s = 1;
        double omz = (double)(rp * rp) / (3.0 * N2);
        *z = -(1.0 - omz);
        *sinth = sqrt(omz * (2.0 - omz));
    }
}

/* Ring (1-based) and in-ring index (0-based) of pixel p, by direct search on
 * the ring starts (plain, not fast). */
void or_pix2ring(int64_t nside, int64_t p, int64_t *ring, int64_t *j)
{
    int64_t lo = 1, hi = 4 * nside - 1;
    while (lo < hi) {                  /* largest r with start(r) <= p */
        int64_t mid = (lo + hi + 1) / 2, n, st; int s; double z, st2;
        or_ring_info(nside, mid, &n, &st, &s, &z, &st2);
        if (st <= p) lo = mid; else hi = mid - 1;
    }
    int64_t n, st; int s; double z, sn;
    or_ring_info(nside, lo, &n, &st, &s, &z, &sn);
    *ring = lo;
    *j = p - st;
}

void or_pix2ang(int64_t nside, int64_t p, double *theta, double *phi)
{
    int64_t r, j, n, st; int s; double z, sn;
    or_pix2ring(nside, p, &r, &j);
    or_ring_info(nside, r, &n, &st, &s, &z, &sn);
    *theta = atan2(sn, z);
    *phi = OR_PI * (double)(2 * j + s) / (double)n;
}

void or_pix2vec(int64_t nside, int64_t p, double *v)
{
    int64_t r, j, n, st; int s; double z, sn;
    or_pix2ring(nside, p, &r, &j);
    or_ring_info(nside, r, &n, &st, &s, &z, &sn);
    double phi = OR_PI * (double)(2 * j + s) / (double)n;
    v[0] = sn * cos(phi);
    v[1] = sn * sin(phi);
    v[2] = z;
}

/* Unit vectors of all pixels, [npix][3]. */
void or_all_vecs(int64_t nside, double *v)
{
    const int64_t nr = 4 * nside - 1;
    for (int64_t r = 1; r <= nr; ++r) {
        int64_t n, st; int s; double z, sn;
        or_ring_info(nside, r, &n, &st, &s, &z, &sn);
        for (int64_t j = 0; j < n; ++j) {
            double phi = OR_PI * (double)(2 * j + s) / (double)n;
            double *q = v + 3 * (st + j);
            q[0] = sn * cos(phi); q[1] = sn * sin(phi); q[2] = z;
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Tabulated kernel (Sec. 3): node coordinate and linear interpolation.      */
/* layout 0: n uniform nodes theta_k = k theta_cut / (n-1).                   */
/* layout 1: half of the nodes on the first 1/16 of the support: nodes        */
/*   0..M (M = n/2) uniform on [0, theta_cut/16], nodes M..n-1 uniform on     */
/*   [theta_cut/16, theta_cut].                                               */
/* ---------------------------------------------------------------------- */

double or_node_theta(int64_t k, int64_t nt, double tc, int layout)
{
    if (layout == 0) return (double)k * tc / (double)(nt - 1);
    int64_t M = nt / 2;
    double t1 = tc / 16.0;
    if (k <= M) return (double)k * t1 / (double)M;
    return t1 + (double)(k - M) * (tc - t1) / (double)(nt - 1 - M);
}

double or_node_coord(double theta, int64_t nt, double tc, int layout)
{
    if (layout == 0) return theta * (double)(nt - 1) / tc;
    int64_t M = nt / 2;
    double t1 = tc / 16.0;
    if (theta <= t1) return theta * (double)M / t1;
    return (double)M + (theta - t1) * (double)(nt - 1 - M) / (tc - t1);
}

/* Interval k and fraction f of theta (theta <= theta_cut). */
void or_node_kf(double theta, int64_t nt, double tc, int layout, int64_t *kout, double *fout)
{
    double u = or_node_coord(theta, nt, tc, layout);
    int64_t k = (int64_t)floor(u);
    if (k > nt - 2) k = nt - 2;
    if (k < 0) k = 0;
    *kout = k;
    *fout = u - (double)k;
}

/* K_lin(theta); 0 beyond the cut. */
double or_klin(const double *V, int64_t nt, double tc, int layout, double theta)
{
    if (theta > tc) return 0.0;
    int64_t k; double f;
    or_node_kf(theta, nt, tc, layout, &k, &f);
    return V[k] + f * (V[k + 1] - V[k]);
}

static double pair_angle(const double *a, const double *b)
{
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    double c = sqrt(dx * dx + dy * dy + dz * dz);
    double h = 0.5 * c;
    if (h > 1.0) h = 1.0;
    return 2.0 * asin(h);
}

static int nthreads_or_default(int nthreads)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads; return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Brute force over all (o, i) pairs.  Plain definition; small Nside.     */
/* x, y: [npix].                                                             */
/* ---------------------------------------------------------------------- */
void or_conv_brute(int64_t nside, const double *V, int64_t nt, double tc, int layout,
                   const double *x, double *y, int nthreads)
{
    const int64_t npix = 12 * nside * nside;
    const double dOmega = 4.0 * OR_PI / (double)npix;
    double *vec = (double *)malloc(sizeof(double) * 3 * npix);
    or_all_vecs(nside, vec);
    int nth = nthreads_or_default(nthreads);
    #pragma omp parallel for schedule(dynamic, 16) num_threads(nth)
    for (int64_t o = 0; o < npix; ++o) {
        double acc = 0.0;
        for (int64_t i = 0; i < npix; ++i) {
            double g = pair_angle(vec + 3 * o, vec + 3 * i);
            if (g <= tc) acc += or_klin(V, nt, tc, layout, g) * x[i];
        }
        y[o] = dOmega * acc;
    }
    free(vec);
}

/* ---------------------------------------------------------------------- */
/* The same sum restricted to a conservative window.  For output o only  */
/* rings with |theta_o - theta_i| <= theta_cut can hold in-cut pixels, and    */
/* on such a ring only pixels with |phi_i - phi_o| <= dphi_max, where          */
/*   cos dphi_max = (cos theta_cut - z_o z_i) / (sin th_o sin th_i).            */
/* Three pixels of padding on each side; every candidate is then tested with  */
/* the exact FP64 angle, so the set of summed pairs equals the brute force.   */
/* ---------------------------------------------------------------------- */

typedef struct {
    int64_t n, start; int s; double z, sn, theta;
} or_ring;

static or_ring *make_rings(int64_t nside)
{
    const int64_t nr = 4 * nside - 1;
    or_ring *R = (or_ring *)malloc(sizeof(or_ring) * (nr + 1));
    for (int64_t r = 1; r <= nr; ++r) {
        or_ring_info(nside, r, &R[r].n, &R[r].start, &R[r].s, &R[r].z, &R[r].sn);
        R[r].theta = atan2(R[r].sn, R[r].z);
    }
    return R;
}

/* Visit every in-cut input pixel of output (ro, jo); callback-free: the
 * caller passes what to do through `mode`. */
typedef struct {
    const double *V; int64_t nt; double tc; int layout;
    const double *x;              /* input map */
    double gy;                    /* upstream gradient of this output (grad mode) */
    double *gV;                   /* table gradient accumulator (grad mode) */
    double acc;                   /* sum (conv mode) */
    int64_t count;                /* pair count */
} or_visit;

enum { OR_CONV = 0, OR_COUNT = 1, OR_GRAD = 2 };

static void visit_output(int64_t nside, const or_ring *R, int64_t ro, int64_t jo,
                         or_visit *st, int mode)
{
    const int64_t nr = 4 * nside - 1;
    const or_ring *Ro = &R[ro];
    double phio = OR_PI * (double)(2 * jo + Ro->s) / (double)Ro->n;
    double vo[3] = { Ro->sn * cos(phio), Ro->sn * sin(phio), Ro->z };
    double ctc = cos(st->tc);
    /* rings ordered by theta; walk outward from ro */
    for (int dir = -1; dir <= 1; dir += 2) {
        for (int64_t ri = (dir < 0 ? ro : ro + 1); ri >= 1 && ri <= nr; ri += dir) {
            const or_ring *Ri = &R[ri];
            if (fabs(Ri->theta - Ro->theta) > st->tc + 1e-12) break;
            double den = Ro->sn * Ri->sn;
            double cdp = (ctc - Ro->z * Ri->z) / den;
            int64_t n = Ri->n;
            int64_t jlo, cnt;
            if (cdp <= -1.0) {
                jlo = 0; cnt = n;
            } else {
                double dpm = acos(cdp > 1.0 ? 1.0 : cdp);
                /* phi_i(j) = pi (2j + s) / n  ->  j = phi n / (2 pi) - s/2 */
                double jc_lo = (phio - dpm) * (double)n / (2.0 * OR_PI) - 0.5 * Ri->s;
                double jc_hi = (phio + dpm) * (double)n / (2.0 * OR_PI) - 0.5 * Ri->s;
                jlo = (int64_t)floor(jc_lo) - 3;
                int64_t jhi = (int64_t)ceil(jc_hi) + 3;
                cnt = jhi - jlo + 1;
                if (cnt >= n) { jlo = 0; cnt = n; }
            }
            for (int64_t m = 0; m < cnt; ++m) {
                int64_t j = jlo + m;
                j %= n; if (j < 0) j += n;
                double phii = OR_PI * (double)(2 * j + Ri->s) / (double)n;
                double vi[3] = { Ri->sn * cos(phii), Ri->sn * sin(phii), Ri->z };
                double g = pair_angle(vo, vi);
                if (g > st->tc) continue;
                int64_t pidx = Ri->start + j;
                if (mode == OR_COUNT) { st->count++; continue; }
                if (mode == OR_CONV) {
                    st->acc += or_klin(st->V, st->nt, st->tc, st->layout, g) * st->x[pidx];
                } else {
                    int64_t k; double f;
                    or_node_kf(g, st->nt, st->tc, st->layout, &k, &f);
                    double v = st->gy * st->x[pidx];
                    st->gV[k] += (1.0 - f) * v;
                    st->gV[k + 1] += f * v;
                }
                st->count++;
            }
        }
    }
}

/* y[outs[t]] for t < nouts (all outputs when outs == NULL; then y is [npix]
 * indexed by pixel, else y is [nouts]). */
void or_conv_window(int64_t nside, const double *V, int64_t nt, double tc, int layout,
                    const double *x, const int64_t *outs, int64_t nouts, double *y,
                    int nthreads)
{
    const int64_t npix = 12 * nside * nside;
    const double dOmega = 4.0 * OR_PI / (double)npix;
    or_ring *R = make_rings(nside);
    int64_t total = outs ? nouts : npix;
    int nth = nthreads_or_default(nthreads);
    #pragma omp parallel for schedule(dynamic, 64) num_threads(nth)
    for (int64_t t = 0; t < total; ++t) {
        int64_t o = outs ? outs[t] : t;
        int64_t ro, jo;
        or_pix2ring(nside, o, &ro, &jo);
        or_visit st; memset(&st, 0, sizeof st);
        st.V = V; st.nt = nt; st.tc = tc; st.layout = layout; st.x = x;
        visit_output(nside, R, ro, jo, &st, OR_CONV);
        y[t] = dOmega * st.acc;
    }
    free(R);
}

/* Number of ordered in-cut pairs (o, i) with o in outs (all when NULL). */
int64_t or_count_pairs(int64_t nside, double tc, const int64_t *outs, int64_t nouts,
                       int nthreads)
{
    const int64_t npix = 12 * nside * nside;
    or_ring *R = make_rings(nside);
    int64_t total = outs ? nouts : npix;
    int64_t sum = 0;
    int nth = nthreads_or_default(nthreads);
    #pragma omp parallel for schedule(dynamic, 256) num_threads(nth) reduction(+:sum)
    for (int64_t t = 0; t < total; ++t) {
        int64_t o = outs ? outs[t] : t;
        int64_t ro, jo;
        or_pix2ring(nside, o, &ro, &jo);
        or_visit st; memset(&st, 0, sizeof st);
        st.tc = tc;
        visit_output(nside, R, ro, jo, &st, OR_COUNT);
        sum += st.count;
    }
    free(R);
    return sum;
}

/* Gradient of L with respect to the table nodes, given gy = dL/dy:
 *   dL/dV_n = dOmega sum_o gy_o sum_{i in cut} x_i dK_lin/dV_n(gamma_oi),
 * dK_lin/dV_k = 1 - f, dK_lin/dV_{k+1} = f.  gV: [nt], overwritten. */
void or_grad_table(int64_t nside, int64_t nt, double tc, int layout, const double *x,
                   const double *gy, double *gV, int nthreads)
{
    const int64_t npix = 12 * nside * nside;
    const double dOmega = 4.0 * OR_PI / (double)npix;
    or_ring *R = make_rings(nside);
    int nth = nthreads_or_default(nthreads);
    double *part = (double *)calloc((size_t)nth * nt, sizeof(double));
    #pragma omp parallel num_threads(nth)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mine = part + (size_t)tid * nt;
        #pragma omp for schedule(dynamic, 64)
        for (int64_t o = 0; o < npix; ++o) {
            if (gy[o] == 0.0) continue;
            int64_t ro, jo;
            or_pix2ring(nside, o, &ro, &jo);
            or_visit st; memset(&st, 0, sizeof st);
            st.nt = nt; st.tc = tc; st.layout = layout; st.x = x;
            st.gy = gy[o]; st.gV = mine;
            visit_output(nside, R, ro, jo, &st, OR_GRAD);
        }
    }
    for (int64_t n = 0; n < nt; ++n) {
        double s = 0.0;
        for (int t = 0; t < nth; ++t) s += part[(size_t)t * nt + n];
        gV[n] = dOmega * s;
    }
    free(part);
    free(R);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
