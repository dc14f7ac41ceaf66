/*
 * pg_oracle.c -- plain FP64 CPU oracle for the Phantom-GRAPE pairwise force
 * loop (Tanikawa, Yoshikawa, Nitadori & Okamoto, arXiv:1203.4037).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this file. It shares no code, header,
 * table or constant with the CUDA library, and the library never calls it.
 *
 * Conventions used throughout:
 *   - positions are double[n][3] row-major, masses double[n];
 *   - d_ij = x_j - x_i (j acts on i), G = 1;
 *   - each i sums its j in ascending j order with Neumaier-compensated FP64
 *     accumulation; i is spread over POSIX threads;
 *   - skip[i] (optional) names one j that i leaves out (its own index in
 *     all-pairs mode); a negative entry leaves nothing out.
 *
 * Functions and the passages they follow:
 *   orc_newton, orc_newton_groups   Eq. (1): softened Newton acceleration;
 *                                   potential with the sign of the Newton
 *                                   listing (phi = -sum m/r_hat, Section 3.3).
 *   orc_s_max, orc_knot, orc_bin    Section 3.4.1: affine map of r^2 to s,
 *                                   s_max, knot formula s_{bE,bF}, index
 *                                   k = 2^F bE + bF, computed arithmetically.
 *   orc_shape                       closed-form g(r) = f(r)/r: Newton,
 *                                   TreePM Gaussian split, S2 PP shape
 *                                   (Eq. s2pp / s2), a linear-in-r^2 test shape.
 *   orc_table_*                     Section 3.4.1 table contents G0, G1 and the
 *                                   interpolation of Section 3.4.2, steps 1-6.
 *   orc_table_forces, orc_shape_forces   Eq. (2) with the table / closed form.
 *   orc_grad_*, orc_fd_*            gradients of L = sum_i w_i . a_i (an
 *                                   extension; the paper has no backward pass)
 *                                   and incremental central differences.
 *
 * Parity pins for every function are in tests/test_oracle_*.py.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* compensated sum                                                      */
/* ------------------------------------------------------------------ */
typedef struct { double s, c; } nsum;

static inline void nadd(nsum *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static inline double nval(const nsum *a) { return a->s + a->c; }

/* ------------------------------------------------------------------ */
/* parallel for over [0, n) with dynamic chunks                          */
/* ------------------------------------------------------------------ */
typedef void (*body_fn)(long long lo, long long hi, void *ctx);
typedef struct { long long n, chunk; long long next; body_fn fn; void *ctx; } pfor_t;

static void *pfor_worker(void *p)
{
    pfor_t *pf = (pfor_t *)p;
    for (;;) {
        long long lo = __atomic_fetch_add(&pf->next, pf->chunk, __ATOMIC_RELAXED);
        if (lo >= pf->n) break;
        long long hi = lo + pf->chunk < pf->n ? lo + pf->chunk : pf->n;
        pf->fn(lo, hi, pf->ctx);
    }
    return NULL;
}

static void parallel_for(long long n, int nthreads, body_fn fn, void *ctx)
{
    if (n <= 0) return;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pfor_t pf;
    pf.n = n; pf.fn = fn; pf.ctx = ctx; pf.next = 0;
    pf.chunk = n / (8LL * nthreads);
    if (pf.chunk < 1) pf.chunk = 1;
    if (nthreads == 1) { fn(0, n, ctx); return; }
    pthread_t th[256];
    int started = 0;
    for (int t = 0; t < nthreads - 1; ++t)
        if (pthread_create(&th[started], NULL, pfor_worker, &pf) == 0) ++started;
    pfor_worker(&pf);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
}

/* minimum-image difference along one axis for a periodic box (box > 0) */
static inline double wrap(double d, double box)
{
    if (box > 0.0) d -= box * nearbyint(d / box);
    return d;
}

/* ------------------------------------------------------------------ */
/* Newton, Eq. (1)                                                      */
/* ------------------------------------------------------------------ */
typedef struct {
    const double *xi; const long long *skip; long long nj;
    const double *xj; const double *mj; double eps2;
    double *acc; double *pot;
    const double *eps_i;   /* per-i softening (Section 3.1), or NULL: eps2 */
} newton_ctx;

static void newton_body(long long lo, long long hi, void *p)
{
    newton_ctx *c = (newton_ctx *)p;
    for (long long i = lo; i < hi; ++i) {
        nsum ax = {0, 0}, ay = {0, 0}, az = {0, 0}, ph = {0, 0};
        long long sk = c->skip ? c->skip[i] : -1;
        double xi = c->xi[3 * i], yi = c->xi[3 * i + 1], zi = c->xi[3 * i + 2];
        /* the softening belongs to the i-particle: its own eps in the i record */
        double e2 = c->eps_i ? c->eps_i[i] * c->eps_i[i] : c->eps2;
        for (long long j = 0; j < c->nj; ++j) {
            if (j == sk) continue;
            double dx = c->xj[3 * j] - xi;
            double dy = c->xj[3 * j + 1] - yi;
            double dz = c->xj[3 * j + 2] - zi;
            double rh2 = dx * dx + dy * dy + dz * dz + e2;        /* r^2 + eps_i^2 */
            double rh = sqrt(rh2);
            double m = c->mj[j];
            double k3 = m / (rh2 * rh);                           /* m / r_hat^3 */
            nadd(&ax, k3 * dx);
            nadd(&ay, k3 * dy);
            nadd(&az, k3 * dz);
            nadd(&ph, -m / rh);
        }
        c->acc[3 * i] = nval(&ax);
        c->acc[3 * i + 1] = nval(&ay);
        c->acc[3 * i + 2] = nval(&az);
        if (c->pot) c->pot[i] = nval(&ph);
    }
}

/* a_i = sum_{j != skip[i]} m_j d_ij / (|d_ij|^2 + eps^2)^{3/2},
 * phi_i = -sum_{j != skip[i]} m_j / (|d_ij|^2 + eps^2)^{1/2}.   Eq. (1), G = 1. */
int orc_newton(long long ni, const double *xi, const long long *skip,
               long long nj, const double *xj, const double *mj, double eps,
               double *acc, double *pot, int nthreads)
{
    if (ni < 0 || nj < 0 || eps < 0) return -1;
    newton_ctx c = {xi, skip, nj, xj, mj, eps * eps, acc, pot, NULL};
    parallel_for(ni, nthreads, newton_body, &c);
    return 0;
}

/* Eq. (1) with the softening of each i-particle: the i-particle structure
 * of Section 3.1 carries eps^2 per i, and the kernel of Section 3.3 adds the
 * i-particle's eps^2 to |d|^2.  a_i = sum_j m_j d_ij / (|d_ij|^2 + eps_i^2)^{3/2},
 * phi_i = -sum_j m_j / (|d_ij|^2 + eps_i^2)^{1/2}, j != skip[i]. */
int orc_newton_epsi(long long ni, const double *xi, const double *eps_i, const long long *skip,
                    long long nj, const double *xj, const double *mj,
                    double *acc, double *pot, int nthreads)
{
    if (ni < 0 || nj < 0 || !eps_i) return -1;
    for (long long i = 0; i < ni; ++i)
        if (!(eps_i[i] >= 0)) return -1;
    newton_ctx c = {xi, skip, nj, xj, mj, 0.0, acc, pot, eps_i};
    parallel_for(ni, nthreads, newton_body, &c);
    return 0;
}

/* list mode: group g's i-particles [i_off[g], i_off[g+1]) each sum exactly the
 * j listed in jlist[j_off[g] .. j_off[g+1]) (tree usage, Section 5.1). */
typedef struct {
    const long long *i_off, *j_off; const int *jlist;
    const double *xi, *xj, *mj; double eps2; double *acc, *pot;
} groups_ctx;

static void groups_body(long long lo, long long hi, void *p)
{
    groups_ctx *c = (groups_ctx *)p;
    for (long long g = lo; g < hi; ++g) {
        for (long long i = c->i_off[g]; i < c->i_off[g + 1]; ++i) {
            nsum ax = {0, 0}, ay = {0, 0}, az = {0, 0}, ph = {0, 0};
            double xi = c->xi[3 * i], yi = c->xi[3 * i + 1], zi = c->xi[3 * i + 2];
            for (long long t = c->j_off[g]; t < c->j_off[g + 1]; ++t) {
                long long j = c->jlist[t];
                double dx = c->xj[3 * j] - xi;
                double dy = c->xj[3 * j + 1] - yi;
                double dz = c->xj[3 * j + 2] - zi;
                double rh2 = dx * dx + dy * dy + dz * dz + c->eps2;
                double rh = sqrt(rh2);
                double m = c->mj[j];
                double k3 = m / (rh2 * rh);
                nadd(&ax, k3 * dx);
                nadd(&ay, k3 * dy);
                nadd(&az, k3 * dz);
                nadd(&ph, -m / rh);
            }
            c->acc[3 * i] = nval(&ax);
            c->acc[3 * i + 1] = nval(&ay);
            c->acc[3 * i + 2] = nval(&az);
            if (c->pot) c->pot[i] = nval(&ph);
        }
    }
}

int orc_newton_groups(long long ngroups, const long long *i_off, const long long *j_off,
                      const int *jlist, const double *xi, const double *xj,
                      const double *mj, double eps, double *acc, double *pot,
                      int nthreads)
{
    if (ngroups < 0 || eps < 0) return -1;
    groups_ctx c = {i_off, j_off, jlist, xi, xj, mj, eps * eps, acc, pot};
    parallel_for(ngroups, nthreads, groups_body, &c);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Table geometry, Section 3.4.1                                        */
/* ------------------------------------------------------------------ */

/* s_max = 2^(2^E) (2 - 2^-F) */
double orc_s_max(int E, int F)
{
    return ldexp(1.0, 1 << E) * (2.0 - ldexp(1.0, -F));
}

/* number of table entries, 2^(E+F) */
long long orc_table_size(int E, int F) { return 1LL << (E + F); }

/* knot k = 2^F bE + bF sits at s = 2^(bE+1) (1 + bF / 2^F) */
double orc_knot(int E, int F, long long k)
{
    (void)E;
    long long nF = 1LL << F;
    long long bE = k / nF, bF = k % nF;
    return ldexp(1.0 + (double)bF / (double)nF, (int)bE + 1);
}

/* index of the bin holding s in [2, s_max]: bE = floor(log2 s) - 1,
 * bF = floor((s / 2^(bE+1) - 1) 2^F), k = 2^F bE + bF. */
long long orc_bin(int E, int F, double s)
{
    (void)E;
    int e;
    frexp(s, &e);                 /* s = f 2^e with f in [1/2, 1): floor(log2 s) = e - 1 */
    int bE = e - 2;
    double frac = ldexp(s, -(bE + 1)) - 1.0;   /* in [0, 1), exact */
    long long bF = (long long)floor(ldexp(frac, F));
    return ((long long)bE << F) + bF;
}

/* scale^2 = (s_max - 2) / r_cut^2, so s = scale^2 r^2 + 2 (Section 3.4.1) */
double orc_scale2(int E, int F, double r_cut)
{
    return (orc_s_max(E, F) - 2.0) / (r_cut * r_cut);
}

/* ------------------------------------------------------------------ */
/* closed-form force shapes g(r) = f(r) / r                             */
/* ------------------------------------------------------------------ */
enum { ORC_SHAPE_NEWTON = 0, ORC_SHAPE_GAUSS_SPLIT = 1, ORC_SHAPE_S2PP = 2,
       ORC_SHAPE_LINEAR = 3, ORC_SHAPE_NEWTON_POT = 4 };

/* S2 force profile of Hockney & Eastwood divided by r (Eq. s2), with
 * xi = 2 r / a and the 35 a^2 denominator in both polynomial branches. */
static double s2_over_r(double r, double a)
{
    double xi = 2.0 * r / a;
    if (xi < 1.0) {
        /* R / r = 2 (224 - 224 xi^2 + 70 xi^3 + 48 xi^4 - 21 xi^5) / (35 a^3) */
        double x2 = xi * xi, x3 = x2 * xi, x4 = x3 * xi, x5 = x4 * xi;
        return 2.0 * (224.0 - 224.0 * x2 + 70.0 * x3 + 48.0 * x4 - 21.0 * x5) /
               (35.0 * a * a * a);
    }
    if (xi < 2.0) {
        double x2 = xi * xi, x3 = x2 * xi, x4 = x3 * xi, x5 = x4 * xi, x6 = x5 * xi;
        double R = (12.0 / x2 - 224.0 + 896.0 * xi - 840.0 * x2 + 224.0 * x3 +
                    70.0 * x4 - 48.0 * x5 + 7.0 * x6) / (35.0 * a * a);
        return R / r;
    }
    return 1.0 / (r * r * r);
}

/* the S2 profile itself, R(r, a) (Eq. s2) */
double orc_s2_profile(double r, double a)
{
    return s2_over_r(r, a) * r;
}

/* g(r) = f(r)/r for the shape selected by id:
 *   NEWTON       par = {eps}:      (r^2 + eps^2)^(-3/2)
 *   GAUSS_SPLIT  par = {r_s, eps}: [erfc(r / 2 r_s) + r/(r_s sqrt(pi)) exp(-r^2 / 4 r_s^2)]
 *                                   (r^2 + eps^2)^(-3/2)   (TreePM short-range part)
 *   S2PP         par = {eps, r_cut}: [R(r, eps) - R(r, r_cut)] / r   (Eq. s2pp)
 *   LINEAR       par = {alpha, beta}: alpha + beta r^2
 *   NEWTON_POT   par = {eps}: -(r^2 + eps^2)^(-1/2), a potential rather than f/r
 *                (tabulated the same way for the table-mode potential) */
double orc_shape(int id, const double *par, double r)
{
    switch (id) {
    case ORC_SHAPE_NEWTON: {
        double rh2 = r * r + par[0] * par[0];
        return 1.0 / (rh2 * sqrt(rh2));
    }
    case ORC_SHAPE_GAUSS_SPLIT: {
        double rs = par[0], eps = par[1];
        double u = r / (2.0 * rs);
        double w = erfc(u) + (r / (rs * sqrt(M_PI))) * exp(-u * u);
        double rh2 = r * r + eps * eps;
        return w / (rh2 * sqrt(rh2));
    }
    case ORC_SHAPE_S2PP:
        return s2_over_r(r, par[0]) - s2_over_r(r, par[1]);
    case ORC_SHAPE_LINEAR:
        return par[0] + par[1] * r * r;
    case ORC_SHAPE_NEWTON_POT:
        return -1.0 / sqrt(r * r + par[0] * par[0]);
    default:
        return NAN;
    }
}

/* ------------------------------------------------------------------ */
/* table contents                                                       */
/* ------------------------------------------------------------------ */

/* From knot values v_0 .. v_{n-1} (v_{n-1} = g at r_cut approached from
 * below) build the stored pair per knot:
 *   G0_k = v_k for k < n-1, G0_{n-1} = 0  (zero force at and beyond r_cut);
 *   G1_k = (v_{k+1} - v_k) / (s_{k+1} - s_k) for k < n-1, G1_{n-1} = 0.
 * The differences and quotients are taken in FP64 and rounded once to FP32;
 * the knot spacing is a power of two, so the quotient is exact. */
int orc_table_from_values(int E, int F, const float *v, float *G0, float *G1)
{
    long long n = orc_table_size(E, F);
    for (long long k = 0; k < n; ++k) {
        if (k < n - 1) {
            double ds = orc_knot(E, F, k + 1) - orc_knot(E, F, k);
            G0[k] = v[k];
            G1[k] = (float)(((double)v[k + 1] - (double)v[k]) / ds);
        } else {
            G0[k] = 0.0f;
            G1[k] = 0.0f;
        }
    }
    return 0;
}

/* knot values of a closed-form shape: v_k = fp32(g(r_k)) with
 * r_k = sqrt((s_k - 2) / scale^2), evaluated in FP64 (r_0 = 0). */
int orc_table_values(int E, int F, double r_cut, int shape, const double *par, float *v)
{
    long long n = orc_table_size(E, F);
    double sc2 = orc_scale2(E, F, r_cut);
    for (long long k = 0; k < n; ++k) {
        double r = sqrt((orc_knot(E, F, k) - 2.0) / sc2);
        v[k] = (float)orc_shape(shape, par, r);
    }
    return 0;
}

int orc_table_build(int E, int F, double r_cut, int shape, const double *par,
                    float *G0, float *G1)
{
    long long n = orc_table_size(E, F);
    float *v = (float *)malloc(sizeof(float) * (size_t)n);
    if (!v) return -2;
    orc_table_values(E, F, r_cut, shape, par, v);
    orc_table_from_values(E, F, v, G0, G1);
    free(v);
    return 0;
}

/* the interpolant of Section 3.4.2 as a function of s (FP64):
 * s is clamped to s_max, k = bin(s), g = G0_k + (s - s_k) G1_k. */
static inline double table_eval_s(int E, int F, double smax, const float *G0,
                                  const float *G1, double s, long long *kout)
{
    if (s > smax) s = smax;
    long long k = orc_bin(E, F, s);
    if (kout) *kout = k;
    return (double)G0[k] + (s - orc_knot(E, F, k)) * (double)G1[k];
}

double orc_table_eval(int E, int F, double r_cut, const float *G0, const float *G1,
                      double r2)
{
    double s = r2 * orc_scale2(E, F, r_cut) + 2.0;
    return table_eval_s(E, F, orc_s_max(E, F), G0, G1, s, NULL);
}

/* ------------------------------------------------------------------ */
/* Eq. (2) with the table (O-T2) or the closed form (O-T1)              */
/* ------------------------------------------------------------------ */
typedef struct {
    const double *xi; const long long *skip; long long nj;
    const double *xj; const double *mj; double box;
    /* table */
    int E, F; double sc2, smax; const float *G0, *G1;
    /* closed form */
    int shape; const double *par; double r_cut;
    double window; double *acc; double *amb; double *absum;
} tab_ctx;

static void table_body(long long lo, long long hi, void *p)
{
    tab_ctx *c = (tab_ctx *)p;
    long long nlast = orc_table_size(c->E, c->F) - 1;
    double s_prev = orc_knot(c->E, c->F, nlast - 1);
    for (long long i = lo; i < hi; ++i) {
        nsum ax = {0, 0}, ay = {0, 0}, az = {0, 0}, am = {0, 0};
        long long sk = c->skip ? c->skip[i] : -1;
        for (long long j = 0; j < c->nj; ++j) {
            if (j == sk) continue;
            double dx = wrap(c->xj[3 * j] - c->xi[3 * i], c->box);
            double dy = wrap(c->xj[3 * j + 1] - c->xi[3 * i + 1], c->box);
            double dz = wrap(c->xj[3 * j + 2] - c->xi[3 * i + 2], c->box);
            double r2 = dx * dx + dy * dy + dz * dz;
            double s = r2 * c->sc2 + 2.0;
            double g = table_eval_s(c->E, c->F, c->smax, c->G0, c->G1, s, NULL);
            double m = c->mj[j];
            nadd(&ax, m * g * dx);
            nadd(&ay, m * g * dy);
            nadd(&az, m * g * dz);
            if (c->amb && fabs(s - c->smax) <= c->window * c->smax) {
                /* either side of the cutoff is a correct reading at this
                 * rounding distance: record the size of the left-limit term */
                double sl = s < c->smax ? s : c->smax;
                double gl = (double)c->G0[nlast - 1] + (sl - s_prev) * (double)c->G1[nlast - 1];
                nadd(&am, m * fabs(gl) * sqrt(r2));
            }
        }
        c->acc[3 * i] = nval(&ax);
        c->acc[3 * i + 1] = nval(&ay);
        c->acc[3 * i + 2] = nval(&az);
        if (c->amb) c->amb[i] = nval(&am);
    }
}

/* O-T2: a_i = sum_{j != skip[i]} m_j g_tab(s_ij) d_ij with the table's
 * interpolant; box > 0 selects minimum-image periodic differences.
 * amb (optional) receives, per i, the summed magnitude of pair terms whose
 * s lies within a relative `window` of s_max. */
int orc_table_forces(long long ni, const double *xi, const long long *skip,
                     long long nj, const double *xj, const double *mj,
                     int E, int F, double r_cut, const float *G0, const float *G1,
                     double box, double window, double *acc, double *amb, int nthreads)
{
    if (ni < 0 || nj < 0 || r_cut <= 0 || E < 0 || F < 0 || E + F > 20) return -1;
    tab_ctx c;
    memset(&c, 0, sizeof c);
    c.xi = xi; c.skip = skip; c.nj = nj; c.xj = xj; c.mj = mj; c.box = box;
    c.E = E; c.F = F; c.sc2 = orc_scale2(E, F, r_cut); c.smax = orc_s_max(E, F);
    c.G0 = G0; c.G1 = G1; c.window = window; c.acc = acc; c.amb = amb;
    parallel_for(ni, nthreads, table_body, &c);
    return 0;
}

/* Table-mode potential, an extension: the tabulated kernel of Section 3.4.2
 * stores accelerations only. A second table of the same layout holds a
 * potential shape psi(r) (P0, P1 built from its knot values exactly as G0,
 * G1 are, so it too is zero at and beyond r_cut), and
 *   phi_i = sum_{j != skip[i]} m_j psi~(s_ij),
 * psi~ the same interpolant in s as the force's g~. amb[i] receives the size
 * of the terms within window relative distance of s_max in s (either side of
 * the cutoff is a correct reading at rounding distance). */
static void tpot_body(long long lo, long long hi, void *p)
{
    tab_ctx *c = (tab_ctx *)p;
    long long nlast = orc_table_size(c->E, c->F) - 1;
    double s_prev = orc_knot(c->E, c->F, nlast - 1);
    for (long long i = lo; i < hi; ++i) {
        nsum ph = {0, 0}, am = {0, 0};
        long long sk = c->skip ? c->skip[i] : -1;
        for (long long j = 0; j < c->nj; ++j) {
            if (j == sk) continue;
            double dx = wrap(c->xj[3 * j] - c->xi[3 * i], c->box);
            double dy = wrap(c->xj[3 * j + 1] - c->xi[3 * i + 1], c->box);
            double dz = wrap(c->xj[3 * j + 2] - c->xi[3 * i + 2], c->box);
            double s = (dx * dx + dy * dy + dz * dz) * c->sc2 + 2.0;
            double m = c->mj[j];
            nadd(&ph, m * table_eval_s(c->E, c->F, c->smax, c->G0, c->G1, s, NULL));
            if (c->amb && fabs(s - c->smax) <= c->window * c->smax) {
                double sl = s < c->smax ? s : c->smax;
                double pl = (double)c->G0[nlast - 1] + (sl - s_prev) * (double)c->G1[nlast - 1];
                nadd(&am, m * fabs(pl));
            }
        }
        c->acc[i] = nval(&ph);
        if (c->amb) c->amb[i] = nval(&am);
    }
}

int orc_table_potential(long long ni, const double *xi, const long long *skip,
                        long long nj, const double *xj, const double *mj,
                        int E, int F, double r_cut, const float *P0, const float *P1,
                        double box, double window, double *phi, double *amb, int nthreads)
{
    if (ni < 0 || nj < 0 || r_cut <= 0 || E < 0 || F < 0 || E + F > 20) return -1;
    tab_ctx c;
    memset(&c, 0, sizeof c);
    c.xi = xi; c.skip = skip; c.nj = nj; c.xj = xj; c.mj = mj; c.box = box;
    c.E = E; c.F = F; c.sc2 = orc_scale2(E, F, r_cut); c.smax = orc_s_max(E, F);
    c.G0 = P0; c.G1 = P1; c.window = window; c.acc = phi; c.amb = amb;
    parallel_for(ni, nthreads, tpot_body, &c);
    return 0;
}

static void shape_body(long long lo, long long hi, void *p)
{
    tab_ctx *c = (tab_ctx *)p;
    double rc2 = c->r_cut * c->r_cut;
    for (long long i = lo; i < hi; ++i) {
        nsum ax = {0, 0}, ay = {0, 0}, az = {0, 0}, am = {0, 0}, ab = {0, 0};
        long long sk = c->skip ? c->skip[i] : -1;
        for (long long j = 0; j < c->nj; ++j) {
            if (j == sk) continue;
            double dx = wrap(c->xj[3 * j] - c->xi[3 * i], c->box);
            double dy = wrap(c->xj[3 * j + 1] - c->xi[3 * i + 1], c->box);
            double dz = wrap(c->xj[3 * j + 2] - c->xi[3 * i + 2], c->box);
            double r2 = dx * dx + dy * dy + dz * dz;
            double r = sqrt(r2);
            double m = c->mj[j];
            if (c->amb && fabs(r2 - rc2) <= c->window * rc2)
                nadd(&am, m * fabs(orc_shape(c->shape, c->par, r)) * r);
            if (r2 >= rc2) continue;
            double g = orc_shape(c->shape, c->par, r);
            nadd(&ax, m * g * dx);
            nadd(&ay, m * g * dy);
            nadd(&az, m * g * dz);
            nadd(&ab, m * fabs(g) * r);
        }
        c->acc[3 * i] = nval(&ax);
        c->acc[3 * i + 1] = nval(&ay);
        c->acc[3 * i + 2] = nval(&az);
        if (c->amb) c->amb[i] = nval(&am);
        if (c->absum) c->absum[i] = nval(&ab);
    }
}

/* O-T1: Eq. (2) with the closed-form shape, pairs with r < r_cut only.
 * absum (optional) receives sum_j |m_j g(r_ij) d_ij| per i: a per-pair
 * relative table error bound (Section 4.2) bounds a per-particle error by
 * that fraction of this sum. */
int orc_shape_forces(long long ni, const double *xi, const long long *skip,
                     long long nj, const double *xj, const double *mj,
                     int shape, const double *par, double r_cut, double box,
                     double window, double *acc, double *amb, double *absum, int nthreads)
{
    if (ni < 0 || nj < 0 || r_cut <= 0) return -1;
    tab_ctx c;
    memset(&c, 0, sizeof c);
    c.xi = xi; c.skip = skip; c.nj = nj; c.xj = xj; c.mj = mj; c.box = box;
    c.shape = shape; c.par = par; c.r_cut = r_cut; c.window = window;
    c.acc = acc; c.amb = amb; c.absum = absum;
    parallel_for(ni, nthreads, shape_body, &c);
    return 0;
}

/* ------------------------------------------------------------------ */
/* gradients of L = sum_i w_i . a_i                                     */
/* ------------------------------------------------------------------ */
/* A pair (i, j), i != j, contributes T_ij = m_j K(r_ij^2) w_i . d_ij with
 * d_ij = x_j - x_i. K is the Newton kernel (r^2 + eps^2)^(-3/2) or the
 * table interpolant g(s(r^2)). With K' = dK/d(r^2):
 *   dT_ij/dx_j = m_j [K w_i + 2 K' (w_i . d_ij) d_ij] = -dT_ij/dx_i,
 *   dT_ij/dm_j = K w_i . d_ij,
 *   dT_ij/dv_b = m_j (w_i . d_ij) dg/dv_b  (table knot values v_b). */

typedef struct {
    long long n; const double *x, *m, *w; double box;
    int table; double eps2;
    int E, F; double sc2, smax; const double *v;   /* table in FP64 knot values */
} lmodel;

/* kernel value K and derivative K' = dK/d(r^2) of one pair; for the table,
 * also the bin k and the position t in [0, 1] inside it (k < 0: no bin). */
static inline void pair_kernel(const lmodel *M, double r2, double *K, double *Kp,
                               long long *kb, double *t)
{
    if (!M->table) {
        double rh2 = r2 + M->eps2;
        double rh = sqrt(rh2);
        *K = 1.0 / (rh2 * rh);
        *Kp = -1.5 * (*K) / rh2;
        *kb = -1; *t = 0;
        return;
    }
    double s = r2 * M->sc2 + 2.0;
    long long n = 1LL << (M->E + M->F);
    if (s >= M->smax) { *K = 0; *Kp = 0; *kb = -1; *t = 0; return; }
    long long k = orc_bin(M->E, M->F, s);
    if (k >= n - 1) { *K = 0; *Kp = 0; *kb = -1; *t = 0; return; }
    double s0 = orc_knot(M->E, M->F, k), s1 = orc_knot(M->E, M->F, k + 1);
    double slope = (M->v[k + 1] - M->v[k]) / (s1 - s0);
    *K = M->v[k] + (s - s0) * slope;
    *Kp = slope * M->sc2;
    *kb = k; *t = (s - s0) / (s1 - s0);
}

static inline void pair_d(const lmodel *M, long long i, long long j, double d[3])
{
    for (int c = 0; c < 3; ++c) d[c] = wrap(M->x[3 * j + c] - M->x[3 * i + c], M->box);
}

typedef struct { const lmodel *M; double *dx, *dm, *Lpart; } grad_ctx;

/* dL/dx_k and dL/dm_k for k in [lo, hi): every pair with k as j, then as i. */
static void grad_body(long long lo, long long hi, void *p)
{
    grad_ctx *c = (grad_ctx *)p;
    const lmodel *M = c->M;
    for (long long k = lo; k < hi; ++k) {
        nsum gx[3] = {{0, 0}, {0, 0}, {0, 0}}, gm = {0, 0}, Lk = {0, 0};
        const double *wk = M->w + 3 * k;
        for (long long o = 0; o < M->n; ++o) {
            if (o == k) continue;
            double d[3], K, Kp, t;
            long long kb;
            /* k acts as j on i = o: T_ok, d_ok = x_k - x_o */
            pair_d(M, o, k, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            pair_kernel(M, r2, &K, &Kp, &kb, &t);
            const double *wo = M->w + 3 * o;
            double wd = wo[0] * d[0] + wo[1] * d[1] + wo[2] * d[2];
            for (int q = 0; q < 3; ++q)
                nadd(&gx[q], M->m[k] * (K * wo[q] + 2.0 * Kp * wd * d[q]));
            nadd(&gm, K * wd);
            /* k acts as i with j = o: T_ko, d_ko = x_o - x_k = -d_ok (K even) */
            double wkd = -(wk[0] * d[0] + wk[1] * d[1] + wk[2] * d[2]);
            for (int q = 0; q < 3; ++q)
                nadd(&gx[q], -M->m[o] * (K * wk[q] + 2.0 * Kp * wkd * (-d[q])));
            nadd(&Lk, M->m[o] * K * wkd);
        }
        if (c->dx) for (int q = 0; q < 3; ++q) c->dx[3 * k + q] = nval(&gx[q]);
        if (c->dm) c->dm[k] = nval(&gm);
        if (c->Lpart) c->Lpart[k] = nval(&Lk);
    }
}

static void setup_model(lmodel *M, long long n, const double *x, const double *m,
                        const double *w, double box)
{
    memset(M, 0, sizeof *M);
    M->n = n; M->x = x; M->m = m; M->w = w; M->box = box;
}

static double sum_parts(const double *p, long long n)
{
    nsum s = {0, 0};
    for (long long i = 0; i < n; ++i) nadd(&s, p[i]);
    return nval(&s);
}

/* Newton: all-pairs analytic dL/dx (n x 3), dL/dm (n) and L. */
int orc_grad_newton(long long n, const double *x, const double *m, const double *w,
                    double eps, double *dx, double *dm, double *L, int nthreads)
{
    lmodel M;
    setup_model(&M, n, x, m, w, 0.0);
    M.eps2 = eps * eps;
    double *Lp = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!Lp) return -2;
    grad_ctx c = {&M, dx, dm, Lp};
    parallel_for(n, nthreads, grad_body, &c);
    if (L) *L = sum_parts(Lp, n);
    free(Lp);
    return 0;
}

/* the same for the subset `idx` of k (dx: nidx x 3, dm: nidx). */
typedef struct { const lmodel *M; const long long *idx; double *dx, *dm; } gsub_ctx;
static void gsub_body(long long lo, long long hi, void *p)
{
    gsub_ctx *c = (gsub_ctx *)p;
    for (long long q = lo; q < hi; ++q) {
        double gx[3], gm;
        grad_ctx one = {c->M, gx, &gm, NULL};
        /* grad_body writes at index k: shift the output pointers */
        long long k = c->idx[q];
        one.dx = gx - 3 * k;
        one.dm = &gm - k;
        grad_body(k, k + 1, &one);
        for (int t = 0; t < 3; ++t) c->dx[3 * q + t] = gx[t];
        c->dm[q] = gm;
    }
}

int orc_grad_newton_at(long long n, const double *x, const double *m, const double *w,
                       double eps, long long nidx, const long long *idx,
                       double *dx, double *dm, int nthreads)
{
    lmodel M;
    setup_model(&M, n, x, m, w, 0.0);
    M.eps2 = eps * eps;
    gsub_ctx c = {&M, idx, dx, dm};
    parallel_for(nidx, nthreads, gsub_body, &c);
    return 0;
}

static int table_model(lmodel *M, long long n, const double *x, const double *m,
                       const double *w, double box, int E, int F, double r_cut,
                       const float *v, double **vd)
{
    setup_model(M, n, x, m, w, box);
    M->table = 1; M->E = E; M->F = F;
    M->sc2 = orc_scale2(E, F, r_cut); M->smax = orc_s_max(E, F);
    long long nt = orc_table_size(E, F);
    *vd = (double *)malloc(sizeof(double) * (size_t)nt);
    if (!*vd) return -2;
    for (long long k = 0; k < nt; ++k) (*vd)[k] = v[k];
    M->v = *vd;
    return 0;
}

int orc_grad_table_at(long long n, const double *x, const double *m, const double *w,
                      double box, int E, int F, double r_cut, const float *v,
                      long long nidx, const long long *idx, double *dx, double *dm,
                      int nthreads)
{
    lmodel M;
    double *vd;
    if (table_model(&M, n, x, m, w, box, E, F, r_cut, v, &vd)) return -2;
    gsub_ctx c = {&M, idx, dx, dm};
    parallel_for(nidx, nthreads, gsub_body, &c);
    free(vd);
    return 0;
}

int orc_grad_table(long long n, const double *x, const double *m, const double *w,
                   double box, int E, int F, double r_cut, const float *v,
                   double *dx, double *dm, double *L, int nthreads)
{
    lmodel M;
    double *vd;
    if (table_model(&M, n, x, m, w, box, E, F, r_cut, v, &vd)) return -2;
    double *Lp = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!Lp) { free(vd); return -2; }
    grad_ctx c = {&M, dx, dm, Lp};
    parallel_for(n, nthreads, grad_body, &c);
    if (L) *L = sum_parts(Lp, n);
    free(Lp);
    free(vd);
    return 0;
}

/* dL/dv_b for every knot b: sum over pairs of m_j (w_i . d_ij) times the
 * hat weights (1 - t) on the bin's left knot and t on its right knot.
 * Threads own blocks of i and keep private per-knot sums. */
typedef struct { const lmodel *M; int nthreads; double *part; long long nt; long long blk; } dv_ctx;
static void dv_body(long long lo, long long hi, void *p)
{
    dv_ctx *c = (dv_ctx *)p;
    const lmodel *M = c->M;
    for (long long b = lo; b < hi; ++b) {
        long long i0 = b * c->blk, i1 = i0 + c->blk < M->n ? i0 + c->blk : M->n;
        double *acc = c->part + (size_t)b * (size_t)c->nt;
        for (long long i = i0; i < i1; ++i) {
            const double *wi = M->w + 3 * i;
            for (long long j = 0; j < M->n; ++j) {
                if (j == i) continue;
                double d[3], K, Kp, t;
                long long kb;
                pair_d(M, i, j, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                pair_kernel(M, r2, &K, &Kp, &kb, &t);
                if (kb < 0) continue;
                double pw = M->m[j] * (wi[0] * d[0] + wi[1] * d[1] + wi[2] * d[2]);
                acc[kb] += pw * (1.0 - t);
                acc[kb + 1] += pw * t;
            }
        }
    }
}

int orc_grad_table_v(long long n, const double *x, const double *m, const double *w,
                     double box, int E, int F, double r_cut, const float *v,
                     double *dv, int nthreads)
{
    lmodel M;
    double *vd;
    if (table_model(&M, n, x, m, w, box, E, F, r_cut, v, &vd)) return -2;
    long long nt = orc_table_size(E, F);
    long long nblk = 64LL * (nthreads > 0 ? nthreads : 1);
    if (nblk > n) nblk = n > 0 ? n : 1;
    long long blk = (n + nblk - 1) / nblk;
    if (blk < 1) blk = 1;
    nblk = (n + blk - 1) / blk;
    double *part = (double *)calloc((size_t)(nblk > 0 ? nblk : 1) * (size_t)nt, sizeof(double));
    if (!part) { free(vd); return -2; }
    dv_ctx c = {&M, nthreads, part, nt, blk};
    parallel_for(nblk, nthreads, dv_body, &c);
    for (long long k = 0; k < nt; ++k) {
        nsum s = {0, 0};
        for (long long b = 0; b < nblk; ++b) nadd(&s, part[(size_t)b * (size_t)nt + k]);
        dv[k] = nval(&s);
    }
    free(part);
    free(vd);
    return 0;
}

/* ------------------------------------------------------------------ */
/* incremental central differences                                      */
/* ------------------------------------------------------------------ */
/* The part of L that involves particle k: sum over o != k of T_ko + T_ok.
 * Central differences of L in a coordinate of x_k, in m_k, or in a knot
 * value only need this part; each pair's change is formed before summing,
 * so the FP64 sum of the full L never cancels. `kinked` is set when a pair
 * changes bin, or crosses the cutoff, between the two probes. */
static void pair_terms(const lmodel *M, long long k, const double xk[3], double mk,
                       long long o, double *T, long long *bin)
{
    double d[3];
    for (int c = 0; c < 3; ++c) d[c] = wrap(M->x[3 * o + c] - xk[c], M->box);   /* d_ko */
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double K, Kp, t;
    long long kb;
    pair_kernel(M, r2, &K, &Kp, &kb, &t);
    const double *wk = M->w + 3 * k, *wo = M->w + 3 * o;
    double Tko = M->m[o] * K * (wk[0] * d[0] + wk[1] * d[1] + wk[2] * d[2]);
    double Tok = mk * K * -(wo[0] * d[0] + wo[1] * d[1] + wo[2] * d[2]);
    *T = Tko + Tok;
    *bin = kb;
}

static double fd_x(const lmodel *M, long long k, int comp, double h, int *kinked)
{
    double xp[3], xm[3];
    for (int c = 0; c < 3; ++c) xp[c] = xm[c] = M->x[3 * k + c];
    xp[comp] += h;
    xm[comp] -= h;
    nsum s = {0, 0};
    int kink = 0;
    for (long long o = 0; o < M->n; ++o) {
        if (o == k) continue;
        double Tp, Tm;
        long long bp, bm;
        pair_terms(M, k, xp, M->m[k], o, &Tp, &bp);
        pair_terms(M, k, xm, M->m[k], o, &Tm, &bm);
        if (bp != bm) kink = 1;
        nadd(&s, Tp - Tm);
    }
    if (kinked) *kinked = kink;
    return nval(&s) / (2.0 * h);
}

static double fd_m(const lmodel *M, long long k, double h)
{
    const double *xk = M->x + 3 * k;
    nsum s = {0, 0};
    for (long long o = 0; o < M->n; ++o) {
        if (o == k) continue;
        double Tp, Tm;
        long long b;
        pair_terms(M, k, xk, M->m[k] + h, o, &Tp, &b);
        pair_terms(M, k, xk, M->m[k] - h, o, &Tm, &b);
        nadd(&s, Tp - Tm);
    }
    return nval(&s) / (2.0 * h);
}

int orc_fd_newton(long long n, const double *x, const double *m, const double *w,
                  double eps, long long k, int what, double h, double *out)
{
    lmodel M;
    setup_model(&M, n, x, m, w, 0.0);
    M.eps2 = eps * eps;
    if (what >= 0 && what < 3) *out = fd_x(&M, k, what, h, NULL);
    else if (what == 3) *out = fd_m(&M, k, h);
    else return -1;
    return 0;
}

int orc_fd_table(long long n, const double *x, const double *m, const double *w,
                 double box, int E, int F, double r_cut, const float *v,
                 long long k, int what, double h, double *out, int *kinked)
{
    lmodel M;
    double *vd;
    if (table_model(&M, n, x, m, w, box, E, F, r_cut, v, &vd)) return -2;
    int rc = 0;
    if (kinked) *kinked = 0;
    if (what >= 0 && what < 3) *out = fd_x(&M, k, what, h, kinked);
    else if (what == 3) *out = fd_m(&M, k, h);
    else rc = -1;
    free(vd);
    return rc;
}

/* central differences in knot values v_b, b in bidx[0..nb): one pass over
 * pairs; a pair whose bin touches a probed knot adds
 * (T(v_b + h_b) - T(v_b - h_b)) / 2h_b to that probe, h_b = h max(1, |v_b|). Threads own blocks of i and
 * keep private per-probe sums. */
typedef struct { const lmodel *M; const long long *slot; long long nb; double h;
                 double *part; long long blk; } fdv_ctx;

/* interpolant in bin k with knot value v_b shifted by dv */
static inline double interp_shift(const lmodel *M, long long k, double s,
                                  long long b, double dv)
{
    double vk = M->v[k] + (b == k ? dv : 0.0);
    double vk1 = M->v[k + 1] + (b == k + 1 ? dv : 0.0);
    double s0 = orc_knot(M->E, M->F, k), s1 = orc_knot(M->E, M->F, k + 1);
    return vk + (s - s0) * ((vk1 - vk) / (s1 - s0));
}

static void fdv_body(long long lo, long long hi, void *p)
{
    fdv_ctx *c = (fdv_ctx *)p;
    const lmodel *M = c->M;
    long long nt = 1LL << (M->E + M->F);
    for (long long blk = lo; blk < hi; ++blk) {
        long long i0 = blk * c->blk, i1 = i0 + c->blk < M->n ? i0 + c->blk : M->n;
        double *acc = c->part + (size_t)blk * (size_t)c->nb;
        for (long long i = i0; i < i1; ++i) {
            const double *wi = M->w + 3 * i;
            for (long long j = 0; j < M->n; ++j) {
                if (j == i) continue;
                double d[3];
                pair_d(M, i, j, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                double s_ = r2 * M->sc2 + 2.0;
                if (s_ >= M->smax) continue;
                long long k = orc_bin(M->E, M->F, s_);
                if (k >= nt - 1) continue;
                double pw = M->m[j] * (wi[0] * d[0] + wi[1] * d[1] + wi[2] * d[2]);
                for (long long b = k; b <= k + 1; ++b) {
                    long long q = c->slot[b];
                    if (q < 0) continue;
                    /* step relative to the knot's size: v reaches 1/eps^3 */
                    double hb = c->h * (fabs(M->v[b]) > 1.0 ? fabs(M->v[b]) : 1.0);
                    double gp = interp_shift(M, k, s_, b, hb);
                    double gm = interp_shift(M, k, s_, b, -hb);
                    acc[q] += pw * (gp - gm) / (2.0 * hb);
                }
            }
        }
    }
}

int orc_fd_table_v(long long n, const double *x, const double *m, const double *w,
                   double box, int E, int F, double r_cut, const float *v,
                   long long nb, const long long *bidx, double h, double *out,
                   int nthreads)
{
    lmodel M;
    double *vd;
    if (table_model(&M, n, x, m, w, box, E, F, r_cut, v, &vd)) return -2;
    long long nt = orc_table_size(E, F);
    long long *slot = (long long *)malloc(sizeof(long long) * (size_t)nt);
    if (!slot) { free(vd); return -2; }
    for (long long k = 0; k < nt; ++k) slot[k] = -1;
    for (long long q = 0; q < nb; ++q)
        if (bidx[q] >= 0 && bidx[q] < nt) slot[bidx[q]] = q;
    long long nblk = 64LL * (nthreads > 0 ? nthreads : 1);
    if (nblk > n) nblk = n > 0 ? n : 1;
    long long blk = (n + nblk - 1) / nblk;
    if (blk < 1) blk = 1;
    nblk = (n + blk - 1) / blk;
    double *part = (double *)calloc((size_t)(nblk > 0 ? nblk : 1) * (size_t)(nb > 0 ? nb : 1),
                                    sizeof(double));
    if (!part) { free(slot); free(vd); return -2; }
    fdv_ctx c = {&M, slot, nb, h, part, blk};
    parallel_for(nblk, nthreads, fdv_body, &c);
    for (long long q = 0; q < nb; ++q) {
        nsum s = {0, 0};
        for (long long b = 0; b < nblk; ++b) nadd(&s, part[(size_t)b * (size_t)nb + q]);
        out[q] = nval(&s);
    }
    free(part);
    free(slot);
    free(vd);
    return 0;
}
