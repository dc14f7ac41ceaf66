/* pg_tree.c -- FP64 CPU oracle of the tree front end: a Barnes-Hut tree
 * whose i-particles are taken in groups that traverse the tree once and
 * share the resulting interaction list (the tree usage of Section 5.1,
 * vacuum boundary, monopole moments), and the forces of all particles from
 * those lists.
 *
 * TEST INFRASTRUCTURE: only the tests, the smoke check and the CPU baseline
 * of the bench use it. It shares no code with the CUDA library.
 *
 * Readings (the paper names the method, not these details):
 *  - the root is the smallest axis-aligned cube holding all particles, with
 *    its low corner at the per-axis minimum and side span = the largest
 *    extent (1 if all particles coincide);
 *  - 10 bits per axis: q_a = floor((x_a - lo_a) / span * 1024), clamped to
 *    1023, interleaved with bit b of x at bit 3b+2 of the key; a node of
 *    level L (0 .. 10) is a run of particles, in key order, with equal
 *    3L-bit key prefix, and its side is span / 2^L;
 *  - monopoles: M = sum of m, S = sum of m x, summed from the particles in
 *    key order for level 10 and from the children in order above it; the
 *    centre of mass is S / M;
 *  - groups: the nodes with at most ncrit particles whose parent has more
 *    (the root if it has at most ncrit), and the level-10 nodes whose
 *    parent has more than ncrit; in particle order;
 *  - opening: a group with bounding box [blo, bhi] accepts node N as one
 *    pseudo-particle if N holds none of the group's particles and
 *    side(N)^2 < theta^2 d^2, d the distance from N's centre of mass to the
 *    box (0 inside it); otherwise a leaf (at most nleaf particles, or level
 *    10) gives its particles and an internal node is opened (a node holding
 *    the group is always opened: its centre of mass may lie far from the
 *    group when the mass is elsewhere);
 *  - list order: breadth first. Every node of level L is decided before any
 *    node of level L + 1, the nodes of one level in key order, and each
 *    decision appends its entries (the node, or a leaf's particles in key
 *    order). The paper fixes the list as a set; the order only changes the
 *    rounding of the sums;
 *  - list entries: k < n is sorted particle k; n + P t + q is pseudo-particle
 *    q of node t, with nodes numbered level by level and in key order within
 *    a level and P pseudo-particles per node;
 *  - monopole (P = 1): one pseudo-particle of mass M at the centre of mass c;
 *  - quadrupole (P = 3; the pseudo-particle multipole method of Kawai and
 *    Makino that the paper cites for its quadrupole runs): with
 *    T = sum m (x - c)(x - c)^T over the node's particles, its eigenvalues
 *    l1 >= l2 >= l3 and unit eigenvectors e1, e2, a = sqrt(2 (l1 - l3) / M)
 *    and b = sqrt(2 (l2 - l3) / M), three pseudo-particles of mass M / 3 at
 *    c + a e1 and c - a/2 e1 +- (sqrt 3 / 2) b e2. They carry the node's
 *    mass, a zero dipole about c and T - l3 I, whose trace-free part is
 *    T's: the potential is the node's through the quadrupole term. e1's
 *    sign makes its largest-magnitude component positive (the lower axis on
 *    a tie); e2's sign does not change the set. With l1 = l2 > l3 exactly
 *    the angle of the triangle in its plane is the eigen-solver's choice.
 * Every FP64 operation is written out (separate multiply and add), so that
 * an implementation that rounds each operation the same way takes the same
 * decisions; the file is compiled without contraction. */
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { TREE_LEVELS = 11, TREE_BITS = 10 };

typedef struct {
    long long n, nnodes, ngroups, nlist;
    long long *perm;        /* key order -> input index */
    unsigned *key;          /* keys in key order */
    double *xs, *ms;        /* particles in key order */
    long long lev_off[TREE_LEVELS + 1];   /* node index range of each level */
    long long *nfirst, *ncount, *nchild0, *nchildn;
    int *nlevel;
    double *nM, *nS;        /* mass, first moment (3 per node) */
    double *nT;             /* second moment about the centre of mass (6 per node:
                             * xx, xy, xz, yy, yz, zz) */
    int npseudo;            /* pseudo-particles per node: 1 or 3 */
    double *pseudo;         /* 4 per pseudo-particle: x, y, z, m */
    double span, lo[3];
    long long *g_node, *g_i0, *g_ni;      /* groups */
    long long *j_off, *jlist;
} orc_tree_t;

static unsigned spread10(unsigned v)
{
    unsigned r = 0;
    for (int b = 0; b < TREE_BITS; ++b) r |= ((v >> b) & 1u) << (3 * b);
    return r;
}

typedef struct { unsigned key; long long idx; } kv_t;

static int kv_cmp(const void *a, const void *b)
{
    const kv_t *x = (const kv_t *)a, *y = (const kv_t *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : x->idx > y->idx;
}

void orc_tree_free(orc_tree_t *t)
{
    if (!t) return;
    free(t->perm); free(t->key); free(t->xs); free(t->ms);
    free(t->nfirst); free(t->ncount); free(t->nchild0); free(t->nchildn); free(t->nlevel);
    free(t->nM); free(t->nS); free(t->nT); free(t->pseudo);
    free(t->g_node); free(t->g_i0); free(t->g_ni); free(t->j_off); free(t->jlist);
    free(t);
}

/* squared distance from point c to the box [lo, hi] */
static double box_d2(const double c[3], const double lo[3], const double hi[3])
{
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double d = 0.0;
        if (c[a] < lo[a]) d = lo[a] - c[a];
        else if (c[a] > hi[a]) d = c[a] - hi[a];
        double dd = d * d;
        d2 = d2 + dd;
    }
    return d2;
}

static int is_leaf(const orc_tree_t *t, long long k, int nleaf)
{
    return t->nlevel[k] == TREE_LEVELS - 1 || t->ncount[k] <= nleaf;
}

/* eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations
 * (each rotation zeroes one off-diagonal element; sweeps repeat until the
 * off-diagonal part is negligible): A = V diag(lam) V^T, V's columns the
 * eigenvectors. A is overwritten. */
static void sym3_eig(double A[3][3], double V[3][3], double lam[3])
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) V[a][b] = a == b ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
        double diag = fabs(A[0][0]) + fabs(A[1][1]) + fabs(A[2][2]);
        if (off == 0.0 || off <= 1e-300 || off <= 1e-18 * diag) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                /* rotation angle phi with tan(2 phi) = 2 A_pq / (A_qq - A_pp);
                 * t = tan(phi) is the smaller root of t^2 + 2 h t - 1 = 0 */
                double h = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double tt = (h >= 0.0 ? 1.0 : -1.0) / (fabs(h) + sqrt(h * h + 1.0));
                double c = 1.0 / sqrt(tt * tt + 1.0), sn = tt * c;
                /* A <- J^T A J with J the rotation in the (p, q) plane */
                for (int k = 0; k < 3; ++k) {
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - sn * akq;
                    A[k][q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - sn * aqk;
                    A[q][k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - sn * vkq;
                    V[k][q] = sn * vkp + c * vkq;
                }
            }
    }
    for (int a = 0; a < 3; ++a) lam[a] = A[a][a];
}

/* second moments about each node's centre of mass, from the definition
 * (the node's particles), and the pseudo-particles */
static int make_pseudo(orc_tree_t *t)
{
    long long nn = t->nnodes;
    t->nT = (double *)calloc((size_t)(6 * nn), sizeof(double));
    t->pseudo = (double *)calloc((size_t)(4 * t->npseudo * nn), sizeof(double));
    if (!t->nT || !t->pseudo) return -1;
    for (long long k = 0; k < nn; ++k) {
        double M = t->nM[k], c[3];
        for (int a = 0; a < 3; ++a) c[a] = t->nS[3 * k + a] / M;
        double T[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (long long i = t->nfirst[k]; i < t->nfirst[k] + t->ncount[k]; ++i) {
            double y[3];
            for (int a = 0; a < 3; ++a) y[a] = t->xs[3 * i + a] - c[a];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) T[a][b] += t->ms[i] * y[a] * y[b];
        }
        double *nt = t->nT + 6 * k;
        nt[0] = T[0][0]; nt[1] = T[0][1]; nt[2] = T[0][2];
        nt[3] = T[1][1]; nt[4] = T[1][2]; nt[5] = T[2][2];
        double *ps = t->pseudo + 4 * t->npseudo * k;
        if (t->npseudo == 1) {
            for (int a = 0; a < 3; ++a) ps[a] = c[a];
            ps[3] = M;
            continue;
        }
        double A[3][3], V[3][3], lam[3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) A[a][b] = T[a][b];
        sym3_eig(A, V, lam);
        /* order: i1 the largest eigenvalue, i3 the smallest, i2 the other */
        int i1 = 0, i3 = 0;
        for (int e = 1; e < 3; ++e) {
            if (lam[e] > lam[i1]) i1 = e;
            if (lam[e] < lam[i3]) i3 = e;
        }
        if (i1 == i3) i3 = (i1 + 1) % 3;      /* all equal */
        int i2 = 3 - i1 - i3;
        double e1[3], e2[3];
        for (int a = 0; a < 3; ++a) { e1[a] = V[a][i1]; e2[a] = V[a][i2]; }
        int big = 0;
        for (int a = 1; a < 3; ++a)
            if (fabs(e1[a]) > fabs(e1[big])) big = a;
        if (e1[big] < 0.0)
            for (int a = 0; a < 3; ++a) e1[a] = -e1[a];
        double d13 = lam[i1] - lam[i3], d23 = lam[i2] - lam[i3];
        double al = sqrt(2.0 * (d13 > 0.0 ? d13 : 0.0) / M);
        double be = sqrt(2.0 * (d23 > 0.0 ? d23 : 0.0) / M);
        double h = sqrt(3.0) / 2.0;
        for (int a = 0; a < 3; ++a) {
            ps[a] = c[a] + al * e1[a];
            ps[4 + a] = c[a] - 0.5 * al * e1[a] + h * be * e2[a];
            ps[8 + a] = c[a] - 0.5 * al * e1[a] - h * be * e2[a];
        }
        ps[3] = ps[7] = ps[11] = M / 3.0;
    }
    return 0;
}

/* the walk of group g, breadth first through a FIFO queue (children are
 * queued in key order, so the queue runs level by level and in key order
 * within a level); writes the entries to out when given and returns their
 * count. queue has room for every node: each enters at most once. */
static long long walk(const orc_tree_t *t, long long g, double theta2, int nleaf,
                      long long *queue, long long *out)
{
    long long i0 = t->g_i0[g], ni = t->g_ni[g];
    double blo[3], bhi[3];
    for (int a = 0; a < 3; ++a) { blo[a] = t->xs[3 * i0 + a]; bhi[a] = blo[a]; }
    for (long long i = i0; i < i0 + ni; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = t->xs[3 * i + a];
            if (v < blo[a]) blo[a] = v;
            if (v > bhi[a]) bhi[a] = v;
        }
    long long head = 0, tail = 0, cnt = 0;
    queue[tail++] = 0;  /* the root */
    while (head < tail) {
        long long k = queue[head++];
        double c[3];
        for (int a = 0; a < 3; ++a) c[a] = t->nS[3 * k + a] / t->nM[k];
        double side = ldexp(t->span, -t->nlevel[k]);
        double side2 = side * side;
        double d2 = box_d2(c, blo, bhi);
        double lim = theta2 * d2;
        int holds = t->nfirst[k] <= i0 && i0 < t->nfirst[k] + t->ncount[k];
        if (!holds && side2 < lim) {
            for (int q = 0; q < t->npseudo; ++q) {
                if (out) out[cnt] = t->n + t->npseudo * k + q;
                ++cnt;
            }
        } else if (is_leaf(t, k, nleaf)) {
            for (long long j = t->nfirst[k]; j < t->nfirst[k] + t->ncount[k]; ++j) {
                if (out) out[cnt] = j;
                ++cnt;
            }
        } else {
            for (long long ch = t->nchild0[k]; ch < t->nchild0[k] + t->nchildn[k]; ++ch)
                queue[tail++] = ch;
        }
    }
    return cnt;
}

orc_tree_t *orc_tree_build(long long n, const double *x, const double *m, double theta,
                           int ncrit, int nleaf, int quadrupole)
{
    if (n <= 0 || !(theta >= 0.0) || ncrit < 1 || nleaf < 1) return NULL;
    orc_tree_t *t = (orc_tree_t *)calloc(1, sizeof *t);
    if (!t) return NULL;
    t->n = n;
    t->npseudo = quadrupole ? 3 : 1;
    /* root cube */
    double hi[3];
    for (int a = 0; a < 3; ++a) { t->lo[a] = x[a]; hi[a] = x[a]; }
    for (long long i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            if (x[3 * i + a] < t->lo[a]) t->lo[a] = x[3 * i + a];
            if (x[3 * i + a] > hi[a]) hi[a] = x[3 * i + a];
        }
    double span = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = hi[a] - t->lo[a];
        if (e > span) span = e;
    }
    if (!(span > 0.0)) span = 1.0;
    t->span = span;
    /* keys and stable order */
    kv_t *kv = (kv_t *)malloc(sizeof(kv_t) * (size_t)n);
    t->perm = (long long *)malloc(sizeof(long long) * (size_t)n);
    t->key = (unsigned *)malloc(sizeof(unsigned) * (size_t)n);
    t->xs = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    t->ms = (double *)malloc(sizeof(double) * (size_t)n);
    if (!kv || !t->perm || !t->key || !t->xs || !t->ms) { free(kv); orc_tree_free(t); return NULL; }
    for (long long i = 0; i < n; ++i) {
        unsigned k = 0;
        for (int a = 0; a < 3; ++a) {
            double u = (x[3 * i + a] - t->lo[a]) / span;
            double s = u * 1024.0;
            double f = floor(s);
            unsigned q = f >= 1023.0 ? 1023u : (unsigned)f;
            k |= spread10(q) << (2 - a);
        }
        kv[i].key = k;
        kv[i].idx = i;
    }
    qsort(kv, (size_t)n, sizeof(kv_t), kv_cmp);
    for (long long i = 0; i < n; ++i) {
        t->perm[i] = kv[i].idx;
        t->key[i] = kv[i].key;
        for (int a = 0; a < 3; ++a) t->xs[3 * i + a] = x[3 * kv[i].idx + a];
        t->ms[i] = m[kv[i].idx];
    }
    free(kv);
    /* nodes: runs of equal prefix at every level */
    long long total = 0;
    for (int L = 0; L < TREE_LEVELS; ++L) {
        int sh = 3 * (TREE_BITS - L);
        long long runs = 0;
        for (long long i = 0; i < n; ++i)
            if (i == 0 || (t->key[i] >> sh) != (t->key[i - 1] >> sh)) ++runs;
        t->lev_off[L] = total;
        total += runs;
    }
    t->lev_off[TREE_LEVELS] = total;
    t->nnodes = total;
    t->nfirst = (long long *)malloc(sizeof(long long) * (size_t)total);
    t->ncount = (long long *)malloc(sizeof(long long) * (size_t)total);
    t->nchild0 = (long long *)calloc((size_t)total, sizeof(long long));
    t->nchildn = (long long *)calloc((size_t)total, sizeof(long long));
    t->nlevel = (int *)malloc(sizeof(int) * (size_t)total);
    t->nM = (double *)malloc(sizeof(double) * (size_t)total);
    t->nS = (double *)malloc(sizeof(double) * 3 * (size_t)total);
    if (!t->nfirst || !t->ncount || !t->nchild0 || !t->nchildn || !t->nlevel || !t->nM || !t->nS) {
        orc_tree_free(t);
        return NULL;
    }
    for (int L = 0; L < TREE_LEVELS; ++L) {
        int sh = 3 * (TREE_BITS - L);
        long long k = t->lev_off[L] - 1;
        for (long long i = 0; i < n; ++i) {
            if (i == 0 || (t->key[i] >> sh) != (t->key[i - 1] >> sh)) {
                ++k;
                t->nfirst[k] = i;
                t->ncount[k] = 0;
                t->nlevel[k] = L;
            }
            ++t->ncount[k];
        }
    }
    /* children: the runs of the next level inside each node */
    for (int L = 0; L + 1 < TREE_LEVELS; ++L) {
        long long c = t->lev_off[L + 1];
        for (long long k = t->lev_off[L]; k < t->lev_off[L + 1]; ++k) {
            t->nchild0[k] = c;
            long long end = t->nfirst[k] + t->ncount[k];
            while (c < t->lev_off[L + 2] && t->nfirst[c] < end) ++c;
            t->nchildn[k] = c - t->nchild0[k];
        }
    }
    /* monopoles, bottom-up */
    for (long long k = t->lev_off[TREE_LEVELS - 1]; k < total; ++k) {
        double M = 0.0, S[3] = {0.0, 0.0, 0.0};
        for (long long i = t->nfirst[k]; i < t->nfirst[k] + t->ncount[k]; ++i) {
            M = M + t->ms[i];
            for (int a = 0; a < 3; ++a) {
                double p = t->ms[i] * t->xs[3 * i + a];
                S[a] = S[a] + p;
            }
        }
        t->nM[k] = M;
        for (int a = 0; a < 3; ++a) t->nS[3 * k + a] = S[a];
    }
    for (int L = TREE_LEVELS - 2; L >= 0; --L)
        for (long long k = t->lev_off[L]; k < t->lev_off[L + 1]; ++k) {
            double M = 0.0, S[3] = {0.0, 0.0, 0.0};
            for (long long ch = t->nchild0[k]; ch < t->nchild0[k] + t->nchildn[k]; ++ch) {
                M = M + t->nM[ch];
                for (int a = 0; a < 3; ++a) S[a] = S[a] + t->nS[3 * ch + a];
            }
            t->nM[k] = M;
            for (int a = 0; a < 3; ++a) t->nS[3 * k + a] = S[a];
        }
    if (make_pseudo(t)) { orc_tree_free(t); return NULL; }
    /* groups, in particle order */
    long long ng = 0;
    t->g_node = (long long *)malloc(sizeof(long long) * (size_t)n);
    t->g_i0 = (long long *)malloc(sizeof(long long) * (size_t)n);
    t->g_ni = (long long *)malloc(sizeof(long long) * (size_t)n);
    if (!t->g_node || !t->g_i0 || !t->g_ni) { orc_tree_free(t); return NULL; }
    {
        long long *gat = (long long *)malloc(sizeof(long long) * (size_t)n);
        if (!gat) { orc_tree_free(t); return NULL; }
        for (long long i = 0; i < n; ++i) gat[i] = -1;
        /* parent of each node: the node of the previous level holding its
         * first particle (runs are nested and in order: one pass per level) */
        for (int L = 0; L < TREE_LEVELS; ++L) {
            long long p = L > 0 ? t->lev_off[L - 1] : 0;
            for (long long k = t->lev_off[L]; k < t->lev_off[L + 1]; ++k) {
                long long pc = -1;
                if (L > 0) {
                    while (t->nfirst[p] + t->ncount[p] <= t->nfirst[k]) ++p;
                    pc = t->ncount[p];
                }
                int grp = (t->ncount[k] <= ncrit && (L == 0 || pc > ncrit)) ||
                          (L == TREE_LEVELS - 1 && pc > ncrit);
                if (grp) gat[t->nfirst[k]] = k;
            }
        }
        for (long long i = 0; i < n; ++i)
            if (gat[i] >= 0) {
                t->g_node[ng] = gat[i];
                t->g_i0[ng] = i;
                t->g_ni[ng] = t->ncount[gat[i]];
                ++ng;
            }
        free(gat);
    }
    t->ngroups = ng;
    /* lists: counts, offsets, entries */
    double theta2 = theta * theta;
    t->j_off = (long long *)malloc(sizeof(long long) * (size_t)(ng + 1));
    if (!t->j_off) { orc_tree_free(t); return NULL; }
    long long *queue = (long long *)malloc(sizeof(long long) * (size_t)t->nnodes);
    if (!queue) { orc_tree_free(t); return NULL; }
    t->j_off[0] = 0;
    for (long long g = 0; g < ng; ++g)
        t->j_off[g + 1] = t->j_off[g] + walk(t, g, theta2, nleaf, queue, NULL);
    t->nlist = t->j_off[ng];
    t->jlist = (long long *)malloc(sizeof(long long) * (size_t)(t->nlist > 0 ? t->nlist : 1));
    if (!t->jlist) { free(queue); orc_tree_free(t); return NULL; }
    for (long long g = 0; g < ng; ++g) walk(t, g, theta2, nleaf, queue, t->jlist + t->j_off[g]);
    free(queue);
    return t;
}

void orc_tree_sizes(const orc_tree_t *t, long long *out5)
{
    out5[0] = t->n;
    out5[1] = t->nnodes;
    out5[2] = t->ngroups;
    out5[3] = t->nlist;
    out5[4] = t->npseudo;
}

/* copies out per node: first particle and count [nnodes], second moment
 * [6 nnodes], and the pseudo-particles [4 npseudo nnodes] */
void orc_tree_get_nodes(const orc_tree_t *t, long long *nfirst, long long *ncount, double *nT,
                        double *pseudo)
{
    memcpy(nfirst, t->nfirst, sizeof(long long) * (size_t)t->nnodes);
    memcpy(ncount, t->ncount, sizeof(long long) * (size_t)t->nnodes);
    memcpy(nT, t->nT, sizeof(double) * 6 * (size_t)t->nnodes);
    memcpy(pseudo, t->pseudo, sizeof(double) * 4 * (size_t)(t->npseudo * t->nnodes));
}

/* copies out: perm[n], group i0/ni/node [ngroups], j_off[ngroups + 1],
 * jlist[nlist], node mass, first moment and level [nnodes], [3 nnodes], [nnodes] */
void orc_tree_get(const orc_tree_t *t, long long *perm, long long *g_i0, long long *g_ni,
                  long long *g_node, long long *j_off, long long *jlist, double *nM, double *nS,
                  int *nlevel)
{
    memcpy(nlevel, t->nlevel, sizeof(int) * (size_t)t->nnodes);
    memcpy(perm, t->perm, sizeof(long long) * (size_t)t->n);
    memcpy(g_i0, t->g_i0, sizeof(long long) * (size_t)t->ngroups);
    memcpy(g_ni, t->g_ni, sizeof(long long) * (size_t)t->ngroups);
    memcpy(g_node, t->g_node, sizeof(long long) * (size_t)t->ngroups);
    memcpy(j_off, t->j_off, sizeof(long long) * (size_t)(t->ngroups + 1));
    memcpy(jlist, t->jlist, sizeof(long long) * (size_t)t->nlist);
    memcpy(nM, t->nM, sizeof(double) * (size_t)t->nnodes);
    memcpy(nS, t->nS, sizeof(double) * 3 * (size_t)t->nnodes);
}

/* Eq. (1) over each group's list, in input order: a particle's own entry
 * (d = 0) is left out; pseudo-particles as the build placed them. FP64,
 * list order, Neumaier-compensated. */
int orc_tree_forces(const orc_tree_t *t, double eps, double *acc, double *pot)
{
    if (!(eps >= 0.0)) return -1;
    double e2 = eps * eps;
    for (long long g = 0; g < t->ngroups; ++g)
        for (long long i = t->g_i0[g]; i < t->g_i0[g] + t->g_ni[g]; ++i) {
            double s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
            for (long long e = t->j_off[g]; e < t->j_off[g + 1]; ++e) {
                long long j = t->jlist[e];
                if (j == i) continue;
                double xj[3], mj;
                if (j < t->n) {
                    for (int a = 0; a < 3; ++a) xj[a] = t->xs[3 * j + a];
                    mj = t->ms[j];
                } else {
                    const double *ps = t->pseudo + 4 * (j - t->n);
                    for (int a = 0; a < 3; ++a) xj[a] = ps[a];
                    mj = ps[3];
                }
                double d[3], r2 = e2;
                for (int a = 0; a < 3; ++a) {
                    d[a] = xj[a] - t->xs[3 * i + a];
                    r2 += d[a] * d[a];
                }
                double rh = sqrt(r2);
                double v[4] = {mj * d[0] / (r2 * rh), mj * d[1] / (r2 * rh), mj * d[2] / (r2 * rh),
                               -mj / rh};
                for (int q = 0; q < 4; ++q) {       /* Neumaier */
                    double tt = s[q] + v[q];
                    if (fabs(s[q]) >= fabs(v[q])) c[q] += (s[q] - tt) + v[q];
                    else c[q] += (v[q] - tt) + s[q];
                    s[q] = tt;
                }
            }
            long long o = t->perm[i];
            for (int a = 0; a < 3; ++a) acc[3 * o + a] = s[a] + c[a];
            if (pot) pot[o] = s[3] + c[3];
        }
    return 0;
}
