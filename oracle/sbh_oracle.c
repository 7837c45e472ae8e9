/*
 * sbh_oracle.c -- the plain, slow, FP64 CPU oracle for the stochastic Barnes-Hut hot path
 * (Madan, Sharp, Williams, Museth, Levin: "Stochastic Barnes-Hut Approximation for Fast
 * Summation on the GPU", SIGGRAPH 2025).
 *
 * THIS IS TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg load it. It shares no code, header, table or helper with the CUDA library: the
 * two are written independently from the paper, and the only thing they have in common is the
 * seeded input generator that feeds both.
 *
 * What it computes, each function citing the passage it follows:
 *   - brute-force kernel sum F(q) = sum_i m_i f(p_i, q)                     (Sec. 3, Eq. 1)
 *   - the octree-like tree with per-dimension branching d (2 or 4), node aggregate mass and
 *     centre of mass (Sec. 3.1), built from its plain recursive definition
 *   - Barnes-Hut, Algorithm 1 (Sec. 3.1, Eq. 2; supplemental "Pseudocode")
 *   - a replay of the stratified path estimator, Algorithm 2, with Russian roulette Eq. 5,
 *     contribution swap Eq. 6 and the one-path estimator Eq. 7 (Sec. 3.3, 3.3.1)
 *   - the exact mean and variance of that estimator by enumerating every outcome of the path
 *     sampler on small trees: the operational form of the unbiasedness proof (Appendix A).
 *
 * Precision. Sums, kernel values and estimator weights are FP64. The decisions that turn a
 * floating-point value into a discrete choice -- the Morton quantisation of a point, the child a
 * path steps into, and the Russian-roulette continue/stop -- are taken in FP32, the precision the
 * paper states for its implementation (Sec. 4.1), with every operation a single IEEE
 * round-to-nearest step (this file must be compiled with -ffp-contract=off), so that the GPU
 * kernels can reproduce them bit for bit.
 *
 * Readings where the paper is silent (each is also listed in the design notes):
 *   - |B_a| is the diagonal of the node's octree cell, sqrt(3) * side * d^-level.
 *   - A node whose points all fall in one child cell is replaced by that child (single-child
 *     chains collapse); the kept node keeps its own level.
 *   - The subdomains are the root's children (Sec. 3.3.1).
 *   Three alternatives are kept as build options of the oracle alone, to measure what each
 *   reading does to the estimator (sbho_tree_build_ex): |B_a| as the diagonal of the tight
 *   axis-aligned box of the node's points (Sec. 3.1's wording), with zero-extent nodes taking
 *   their cell's diagonal (box mode 1) or literally 0, so that Eq. 5 gives p = 0 into one-point
 *   nodes and the estimator is truncated there (box mode 2); single-child chains kept as nodes;
 *   and the subdomains taken one or more generations deeper ("other choices are also possible",
 *   Sec. 3.3.1).
 *   - A node is a leaf when it holds <= leaf_size points or sits at the deepest level; a leaf
 *     with more than one point has its points as children, one level deeper.
 *   - The path index I is drawn lazily, one child per level, child c of T with probability
 *     m_c / m_T (or |T_c| / |T| for the paper's count-uniform choice), which gives
 *     p(I in T_{I,k}) = m_{I,k} / m_a exactly as drawing I up front with p(I=i) = m_i / m_a.
 *   - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = (seed low 32,
 *     seed high 32). A decision needs two independent uniforms and a block gives four, so one
 *     block serves two consecutive depths: the decision at depth k uses the block of counter
 *     (query index, subdomain index, sample index, k - k mod 2), words 0 and 1 at even k, words
 *     2 and 3 at odd k. The first of the two words picks the child, the second drives Russian
 *     roulette; u = (x >> 8) * 2^-24.
 *   - Child pick: the stored FP32 prefix fraction cdf_c = (sum_{c'<=c} m_c') / m_T (the last
 *     child's is exactly 1); the chosen child is the number of children c < last with
 *     cdf_c <= u.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define SBHO_API __attribute__((visibility("default")))

enum { K_COULOMB = 0, K_WINDING = 1, K_SMOOTHDIST = 2, K_AFFINE = 3 };
enum { SAMPLE_MASS = 0, SAMPLE_COUNT = 1 };
enum { RR_PAPER = 0, RR_OFF = 1, RR_HALF = 2 };

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition (Salmon et al., SC'11, Sec. 4 and Table 2):     */
/* ten rounds of two 32x32->64 multiplies with Feistel-style mixing; the key is bumped by the   */
/* Weyl constants (golden ratio, sqrt(3)-1) before every round but the first.                  */
/* ------------------------------------------------------------------------------------------ */
SBHO_API void sbho_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += weyl0; k1 += weyl1; }
        uint64_t prod0 = (uint64_t)mul0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)mul1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* uniform in [0,1) with 24 random bits: exactly representable in FP32 and FP64 */
static float unit24f(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

/* The two random words of the decision at depth k of the path (query index qc, subdomain ai,    */
/* sample s): block (qc, ai, s, k - k mod 2), words 0 and 1 at even k, 2 and 3 at odd k.         */
static void decision_words(const uint32_t key[2], uint32_t qc, uint32_t ai, uint32_t s, uint32_t k, uint32_t w[2])
{
    const uint32_t ctr[4] = {qc, ai, s, k & ~1u};
    uint32_t x[4];
    sbho_philox4x32_10(ctr, key, x);
    w[0] = x[2 * (k & 1u)];
    w[1] = x[2 * (k & 1u) + 1];
}

/* ------------------------------------------------------------------------------------------ */
/* Kernels f(p, q) times the source weight, in FP64 (Sec. 3 Eq. 1; Sec. 4.2 Coulomb-like       */
/* potential; Sec. 4.3.2 winding numbers; Sec. 4.3.3 smooth distance).                        */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t kind;
    double softening;  /* Coulomb: f = 1 / sqrt(r^2 + eps^2) */
    double alpha;      /* smooth distance: f = exp(-alpha r) */
    double affine[3];  /* test kernel: f = 1 + g . (p - q), affine in p */
} sbho_kernel;

/* weight * f(p, q); dip is the node's dipole sum_j m_j n_j (used by the winding kernel only) */
static double term(const sbho_kernel *k, const double p[3], double m, const double dip[3],
                   const double q[3])
{
    double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
    double r2 = dx * dx + dy * dy + dz * dz;
    switch (k->kind) {
    case K_COULOMB:
        return m / sqrt(r2 + k->softening * k->softening);
    case K_WINDING: {
        if (r2 == 0.0) return 0.0;
        double r = sqrt(r2);
        return (dx * dip[0] + dy * dip[1] + dz * dip[2]) / (4.0 * M_PI * r2 * r);
    }
    case K_SMOOTHDIST:
        return m * exp(-k->alpha * sqrt(r2));
    case K_AFFINE:
        return m * (1.0 + k->affine[0] * dx + k->affine[1] * dy + k->affine[2] * dz);
    }
    return 0.0;
}

/* Gradient with respect to the query q of weight * f(p, q), with d = p - q, r = |d|:
 *   Coulomb   m d / (r^2 + eps^2)^(3/2)
 *   winding   (-N / r^3 + 3 (d . N) d / r^5) / (4 pi), 0 at r = 0
 *   smooth    alpha m exp(-alpha r) d / r, 0 at r = 0
 *   affine    -m g                                                                              */
static void term_grad(const sbho_kernel *k, const double p[3], double m, const double dip[3],
                      const double q[3], double g[3])
{
    double d[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double c = 0.0;
    switch (k->kind) {
    case K_COULOMB: {
        double e = r2 + k->softening * k->softening;
        c = m / (e * sqrt(e));
        for (int a = 0; a < 3; ++a) g[a] = c * d[a];
        return;
    }
    case K_WINDING: {
        if (r2 == 0.0) { g[0] = g[1] = g[2] = 0.0; return; }
        double r = sqrt(r2), r3 = r2 * r, r5 = r3 * r2;
        double dn = d[0] * dip[0] + d[1] * dip[1] + d[2] * dip[2];
        for (int a = 0; a < 3; ++a) g[a] = (-dip[a] / r3 + 3.0 * dn * d[a] / r5) / (4.0 * M_PI);
        return;
    }
    case K_SMOOTHDIST: {
        if (r2 == 0.0) { g[0] = g[1] = g[2] = 0.0; return; }
        double r = sqrt(r2);
        c = k->alpha * m * exp(-k->alpha * r) / r;
        for (int a = 0; a < 3; ++a) g[a] = c * d[a];
        return;
    }
    case K_AFFINE:
        for (int a = 0; a < 3; ++a) g[a] = -m * k->affine[a];
        return;
    }
    g[0] = g[1] = g[2] = 0.0;
}

/* ------------------------------------------------------------------------------------------ */
/* Brute force, Eq. 1: F(q) = sum_i m_i f(p_i, q). Neumaier-compensated FP64 summation.        */
/* ------------------------------------------------------------------------------------------ */
static double point_term(const sbho_kernel *k, const float *pts, const float *w, const float *nrm,
                         int64_t i, const double q[3])
{
    double p[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
    double m = w[i];
    double dip[3] = {0, 0, 0};
    if (nrm) {
        dip[0] = m * (double)nrm[3 * i];
        dip[1] = m * (double)nrm[3 * i + 1];
        dip[2] = m * (double)nrm[3 * i + 2];
    }
    return term(k, p, m, dip, q);
}

SBHO_API void sbho_brute(const sbho_kernel *k, const float *pts, const float *w, const float *nrm,
                         int64_t n, const float *queries, int64_t nq, double *out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < nq; ++j) {
        double q[3] = {queries[3 * j], queries[3 * j + 1], queries[3 * j + 2]};
        double sum = 0.0, comp = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double t = point_term(k, pts, w, nrm, i, q);
            double s = sum + t;
            if (fabs(sum) >= fabs(t)) comp += (sum - s) + t;
            else comp += (t - s) + sum;
            sum = s;
        }
        out[j] = sum + comp;
    }
}

/* grad[3 j + a] = dF/dq_a (q_j) = sum_i d(m_i f(p_i, q))/dq_a, compensated FP64 sums */
SBHO_API void sbho_brute_grad(const sbho_kernel *k, const float *pts, const float *w, const float *nrm,
                              int64_t n, const float *queries, int64_t nq, double *grad)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < nq; ++j) {
        double q[3] = {queries[3 * j], queries[3 * j + 1], queries[3 * j + 2]};
        double sum[3] = {0, 0, 0}, comp[3] = {0, 0, 0};
        for (int64_t i = 0; i < n; ++i) {
            double p[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
            double m = w[i], dip[3] = {0, 0, 0}, g[3];
            if (nrm)
                for (int a = 0; a < 3; ++a) dip[a] = m * (double)nrm[3 * i + a];
            term_grad(k, p, m, dip, q, g);
            for (int a = 0; a < 3; ++a) {
                double t = g[a], s2 = sum[a] + t;
                if (fabs(sum[a]) >= fabs(t)) comp[a] += (sum[a] - s2) + t;
                else comp[a] += (t - s2) + sum[a];
                sum[a] = s2;
            }
        }
        for (int a = 0; a < 3; ++a) grad[3 * j + a] = sum[a] + comp[a];
    }
}

/* ------------------------------------------------------------------------------------------ */
/* The tree (Sec. 3.1): an octree-like subdivision of the root cube with per-dimension         */
/* branching d; every node stores its point set (a range of the Morton-sorted points), its     */
/* aggregate mass m_a = sum m_b and centre of mass p_a = sum m_b p_b / m_a.                     */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    int32_t d;          /* per-dimension branching: 2 or 4 */
    int32_t bits;       /* Morton bits per level: log2(d^3) = 3 or 6 */
    int32_t max_level;  /* 20 (d=2) or 10 (d=4): 60-bit codes */
    int32_t leaf_size;
    int32_t has_normals;
    float lo[3], side, diam0;  /* root cube corner and edge; cell diagonal at level 0 (FP32) */
    int64_t *perm;   /* [n] original index of the i-th point in Morton order */
    uint64_t *code;  /* [n] sorted Morton codes */
    int64_t n_nodes;
    int64_t *begin, *end, *first_child, *parent;
    int32_t *nchild, *level;
    double *mass, *com, *dip;      /* FP64 aggregates: [N], [3N], [3N] */
    float *mass32, *com32, *cdf;   /* FP32 roundings used by the FP32 decisions: [N], [3N], [N] */
    int64_t n_sub;                 /* subdomains (Sec. 3.3.1): the root's children, or the root */
    int64_t first_sub;
    int64_t *subs;                 /* [n_sub] subdomain node ids */
    int32_t box_mode;              /* |B_a|: 0 cell diagonal, 1 tight box (cell if zero extent), 2 tight box */
    int32_t collapse;              /* 1: single-child chains collapse */
    double *bd;                    /* [N] |B_a| in FP64 for box modes 1 and 2 */
} otree;

/* Quantise one coordinate to a 20-bit cell index: floor((x - lo) * (2^20 / side)), clamped.
 * FP32, one rounding per operation, no contraction. */
static uint32_t quant20(float x, float lo, float scale)
{
    float t = (x - lo) * scale;
    float f = floorf(t);
    uint32_t c = (f <= 0.0f) ? 0u : (uint32_t)f;
    return c > 1048575u ? 1048575u : c;
}

/* Morton interleave, x bit first within each (x, y, z) triple, most significant triple first */
static uint64_t morton60(uint32_t cx, uint32_t cy, uint32_t cz)
{
    uint64_t code = 0;
    for (int b = 19; b >= 0; --b) {
        code = (code << 3) | ((uint64_t)((cx >> b) & 1u) << 2) | ((uint64_t)((cy >> b) & 1u) << 1) |
               (uint64_t)((cz >> b) & 1u);
    }
    return code;
}

typedef struct { uint64_t code; int64_t idx; } keyed;
static int cmp_keyed(const void *a, const void *b)
{
    const keyed *x = (const keyed *)a, *y = (const keyed *)b;
    if (x->code != y->code) return x->code < y->code ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);  /* ties keep the input order */
}

/* child cell digit of code at level (1-based): the bits-wide group below level-1 */
static uint32_t digit_at(const otree *t, uint64_t code, int level)
{
    int shift = 60 - t->bits * level;
    return (uint32_t)((code >> shift) & ((1u << t->bits) - 1u));
}

/* A node under construction, before breadth-first numbering */
typedef struct tnode {
    int64_t begin, end;
    int32_t level;
    int32_t nchild;
    struct tnode **child;
} tnode;

static tnode *new_tnode(int64_t b, int64_t e, int level)
{
    tnode *x = (tnode *)calloc(1, sizeof(tnode));
    x->begin = b; x->end = e; x->level = level;
    return x;
}

/* Points [b, e) as children of a multi-point leaf, one level below it */
static void attach_points(tnode *x)
{
    int64_t cnt = x->end - x->begin;
    x->nchild = (int32_t)cnt;
    x->child = (tnode **)calloc((size_t)cnt, sizeof(tnode *));
    for (int64_t i = 0; i < cnt; ++i) x->child[i] = new_tnode(x->begin + i, x->begin + i + 1, x->level + 1);
}

/* The node holding the points [b, e), which first appear as one run at `level`. */
static tnode *make_node(const otree *t, int64_t b, int64_t e, int level)
{
    tnode *x = new_tnode(b, e, level);
    int64_t cnt = e - b;
    if (cnt == 1) return x;                                   /* a source point */
    if (cnt <= t->leaf_size) { attach_points(x); return x; }  /* small leaf */
    for (;;) {
        if (x->level == t->max_level) { attach_points(x); return x; }  /* deepest level */
        /* split into runs of equal digits one level down */
        int runs = 1;
        for (int64_t i = b + 1; i < e; ++i)
            if (digit_at(t, t->code[i], x->level + 1) != digit_at(t, t->code[i - 1], x->level + 1)) ++runs;
        if (runs == 1 && t->collapse) { x->level += 1; continue; }  /* single child: collapse into it */
        if (runs == 1) {  /* single child kept as a node one level down (collapse off) */
            x->nchild = 1;
            x->child = (tnode **)calloc(1, sizeof(tnode *));
            x->child[0] = make_node(t, b, e, x->level + 1);
            return x;
        }
        x->nchild = runs;
        x->child = (tnode **)calloc((size_t)runs, sizeof(tnode *));
        int64_t s = b; int c = 0;
        for (int64_t i = b + 1; i <= e; ++i) {
            if (i == e || digit_at(t, t->code[i], x->level + 1) != digit_at(t, t->code[i - 1], x->level + 1)) {
                x->child[c++] = make_node(t, s, i, x->level + 1);
                s = i;
            }
        }
        return x;
    }
}

static void free_tnode(tnode *x)
{
    for (int i = 0; i < x->nchild; ++i) free_tnode(x->child[i]);
    free(x->child);
    free(x);
}

static int64_t count_tnodes(const tnode *x)
{
    int64_t c = 1;
    for (int i = 0; i < x->nchild; ++i) c += count_tnodes(x->child[i]);
    return c;
}

/* The tree with the default readings when box_mode = 0, collapse = 1, sub_gen = 1. Otherwise:
 * box_mode 1 or 2 takes |B_a| from the tight box of the node's points (see the file header),
 * collapse = 0 keeps single-child chains, and sub_gen = g takes as subdomains the nodes g
 * generations below the root (and any leaf above that generation), which still cover every
 * point once, as Sec. 3.3.1 requires. */
SBHO_API void *sbho_tree_build_ex(const float *pts, const float *w, const float *nrm, int64_t n,
                                  int32_t leaf_size, int32_t d, int32_t box_mode, int32_t collapse,
                                  int32_t sub_gen)
{
    if (n < 1 || leaf_size < 1 || (d != 2 && d != 4)) return NULL;
    if (box_mode < 0 || box_mode > 2 || sub_gen < 1) return NULL;
    otree *t = (otree *)calloc(1, sizeof(otree));
    t->n = n; t->d = d; t->bits = (d == 4) ? 6 : 3; t->max_level = 60 / t->bits;
    t->leaf_size = leaf_size; t->has_normals = nrm != NULL;
    t->box_mode = box_mode; t->collapse = collapse != 0;

    /* root cube: lower corner = per-axis minimum, edge = largest extent (1 if all coincide) */
    float mn[3], mx[3];
    for (int a = 0; a < 3; ++a) { mn[a] = pts[a]; mx[a] = pts[a]; }
    for (int64_t i = 1; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            float v = pts[3 * i + a];
            if (v < mn[a]) mn[a] = v;
            if (v > mx[a]) mx[a] = v;
        }
    float side = 0.0f;
    for (int a = 0; a < 3; ++a) {
        float ext = mx[a] - mn[a];
        if (ext > side) side = ext;
        t->lo[a] = mn[a];
    }
    if (side == 0.0f) side = 1.0f;
    t->side = side;
    t->diam0 = 1.7320508075688772f * side;
    float scale = 1048576.0f / side;

    keyed *kv = (keyed *)malloc((size_t)n * sizeof(keyed));
    for (int64_t i = 0; i < n; ++i) {
        uint32_t cx = quant20(pts[3 * i], t->lo[0], scale);
        uint32_t cy = quant20(pts[3 * i + 1], t->lo[1], scale);
        uint32_t cz = quant20(pts[3 * i + 2], t->lo[2], scale);
        kv[i].code = morton60(cx, cy, cz);
        kv[i].idx = i;
    }
    qsort(kv, (size_t)n, sizeof(keyed), cmp_keyed);
    t->perm = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    t->code = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    for (int64_t i = 0; i < n; ++i) { t->perm[i] = kv[i].idx; t->code[i] = kv[i].code; }
    free(kv);

    tnode *root = make_node(t, 0, n, 0);
    int64_t N = count_tnodes(root);
    t->n_nodes = N;
    t->begin = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    t->end = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    t->first_child = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    t->parent = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    t->nchild = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    t->level = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    t->mass = (double *)calloc((size_t)N, sizeof(double));
    t->com = (double *)calloc((size_t)N * 3, sizeof(double));
    t->dip = (double *)calloc((size_t)N * 3, sizeof(double));
    t->mass32 = (float *)malloc((size_t)N * sizeof(float));
    t->com32 = (float *)malloc((size_t)N * 3 * sizeof(float));
    t->cdf = (float *)malloc((size_t)N * sizeof(float));

    /* breadth-first numbering: the children of a node get consecutive indices, in Morton order */
    tnode **queue = (tnode **)malloc((size_t)N * sizeof(tnode *));
    int64_t head = 0, tail = 0;
    queue[tail++] = root;
    t->parent[0] = -1;
    while (head < tail) {
        int64_t id = head;
        tnode *x = queue[head++];
        t->begin[id] = x->begin; t->end[id] = x->end; t->level[id] = x->level;
        t->nchild[id] = x->nchild;
        t->first_child[id] = x->nchild ? tail : -1;
        for (int c = 0; c < x->nchild; ++c) {
            t->parent[tail] = id;
            queue[tail++] = x->child[c];
        }
    }
    free(queue);
    free_tnode(root);

    /* aggregates (Sec. 3.1): direct FP64 sums over each node's points */
    for (int64_t v = 0; v < N; ++v) {
        double m = 0, s[3] = {0, 0, 0}, nd[3] = {0, 0, 0};
        for (int64_t i = t->begin[v]; i < t->end[v]; ++i) {
            int64_t j = t->perm[i];
            double mj = w[j];
            m += mj;
            for (int a = 0; a < 3; ++a) s[a] += mj * (double)pts[3 * j + a];
            if (nrm)
                for (int a = 0; a < 3; ++a) nd[a] += mj * (double)nrm[3 * j + a];
        }
        t->mass[v] = m;
        for (int a = 0; a < 3; ++a) {
            t->com[3 * v + a] = s[a] / m;
            t->dip[3 * v + a] = nd[a];
            t->com32[3 * v + a] = (float)t->com[3 * v + a];
        }
        t->mass32[v] = (float)m;
    }
    /* child-pick prefix fractions within each parent */
    t->cdf[0] = 1.0f;
    for (int64_t v = 0; v < N; ++v) {
        int nc = t->nchild[v];
        if (!nc) continue;
        int64_t fc = t->first_child[v];
        double tot = 0;
        for (int c = 0; c < nc; ++c) tot += t->mass[fc + c];
        double pre = 0;
        for (int c = 0; c < nc; ++c) {
            pre += t->mass[fc + c];
            t->cdf[fc + c] = (c == nc - 1) ? 1.0f : (float)(pre / tot);
        }
    }
    if (t->nchild[0] > 0) { t->first_sub = t->first_child[0]; t->n_sub = t->nchild[0]; }
    else { t->first_sub = 0; t->n_sub = 1; }

    /* subdomains: generation sub_gen below the root, plus the leaves above it */
    t->subs = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    if (N == 1) {
        t->subs[0] = 0; t->n_sub = 1;
    } else {
        int32_t *gen = (int32_t *)calloc((size_t)N, sizeof(int32_t));
        t->n_sub = 0;
        for (int64_t v = 1; v < N; ++v) {
            gen[v] = gen[t->parent[v]] + 1;
            if (gen[v] == sub_gen || (gen[v] < sub_gen && t->nchild[v] == 0)) t->subs[t->n_sub++] = v;
        }
        free(gen);
        t->first_sub = t->subs[0];
    }

    /* |B_a| of the tight box of each node's points, for box modes 1 and 2 */
    if (box_mode != 0) {
        t->bd = (double *)malloc((size_t)N * sizeof(double));
        for (int64_t v = 0; v < N; ++v) {
            double lo[3], hi[3], s2 = 0.0;
            for (int a = 0; a < 3; ++a) { lo[a] = INFINITY; hi[a] = -INFINITY; }
            for (int64_t i = t->begin[v]; i < t->end[v]; ++i)
                for (int a = 0; a < 3; ++a) {
                    double x = pts[3 * t->perm[i] + a];
                    if (x < lo[a]) lo[a] = x;
                    if (x > hi[a]) hi[a] = x;
                }
            for (int a = 0; a < 3; ++a) s2 += (hi[a] - lo[a]) * (hi[a] - lo[a]);
            double b = sqrt(s2);
            if (b == 0.0 && box_mode == 1) b = ldexp(sqrt(3.0) * t->side, -(t->bits / 3) * t->level[v]);
            t->bd[v] = b;
        }
    }
    return t;
}

SBHO_API void *sbho_tree_build(const float *pts, const float *w, const float *nrm, int64_t n,
                               int32_t leaf_size, int32_t d)
{
    return sbho_tree_build_ex(pts, w, nrm, n, leaf_size, d, 0, 1, 1);
}

SBHO_API void sbho_tree_free(void *h)
{
    otree *t = (otree *)h;
    if (!t) return;
    free(t->perm); free(t->code); free(t->begin); free(t->end); free(t->first_child);
    free(t->parent); free(t->nchild); free(t->level); free(t->mass); free(t->com); free(t->dip);
    free(t->mass32); free(t->com32); free(t->cdf); free(t->subs); free(t->bd);
    free(t);
}

SBHO_API int64_t sbho_tree_nnodes(const void *h) { return ((const otree *)h)->n_nodes; }

/* Root cube and subdomains: meta = {lo.x, lo.y, lo.z, side, diam0}; ids = {first_sub, n_sub} */
SBHO_API void sbho_tree_meta(const void *h, float meta[5], int64_t ids[2])
{
    const otree *t = (const otree *)h;
    meta[0] = t->lo[0]; meta[1] = t->lo[1]; meta[2] = t->lo[2]; meta[3] = t->side; meta[4] = t->diam0;
    ids[0] = t->first_sub; ids[1] = t->n_sub;
}

/* Copy the tree out (any pointer may be NULL). Arrays are [n] or [n_nodes] (x3 for vectors). */
SBHO_API void sbho_tree_export(const void *h, int64_t *perm, uint64_t *code, int64_t *begin,
                               int64_t *end, int64_t *first_child, int32_t *nchild, int32_t *level,
                               double *mass, double *com, double *dip, float *cdf)
{
    const otree *t = (const otree *)h;
    size_t N = (size_t)t->n_nodes, n = (size_t)t->n;
    if (perm) memcpy(perm, t->perm, n * sizeof(int64_t));
    if (code) memcpy(code, t->code, n * sizeof(uint64_t));
    if (begin) memcpy(begin, t->begin, N * sizeof(int64_t));
    if (end) memcpy(end, t->end, N * sizeof(int64_t));
    if (first_child) memcpy(first_child, t->first_child, N * sizeof(int64_t));
    if (nchild) memcpy(nchild, t->nchild, N * sizeof(int32_t));
    if (level) memcpy(level, t->level, N * sizeof(int32_t));
    if (mass) memcpy(mass, t->mass, N * sizeof(double));
    if (com) memcpy(com, t->com, 3 * N * sizeof(double));
    if (dip) memcpy(dip, t->dip, 3 * N * sizeof(double));
    if (cdf) memcpy(cdf, t->cdf, N * sizeof(float));
}

/* ------------------------------------------------------------------------------------------ */
/* Per-node quantities shared by Barnes-Hut and the estimator                                   */
/* ------------------------------------------------------------------------------------------ */
static double node_term(const otree *t, const sbho_kernel *k, int64_t v, const double q[3])
{
    return term(k, &t->com[3 * v], t->mass[v], &t->dip[3 * v], q);
}

/* |B_a|: the cell diagonal at the node's level, in FP32 (scaling by a power of two is exact) */
static float diam32(const otree *t, int level)
{
    return ldexpf(t->diam0, -(t->bits / 3) * level);
}

/* ||q - p_a|| in FP32 with a fixed operation order: ((dx*dx + dy*dy) + dz*dz), then sqrt */
static float dist32(const float p[3], const float q[3])
{
    float dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
    float s = dx * dx + dy * dy;
    s = s + dz * dz;
    return sqrtf(s);
}

/* far-field ratio beta~ = ||q - p_a|| / |B_a| (Sec. 3.3), FP32 */
static float ffratio32(const otree *t, int64_t v, const float q[3])
{
    if (t->box_mode != 0) return dist32(&t->com32[3 * v], q) / (float)t->bd[v];  /* inf at |B| = 0 */
    return dist32(&t->com32[3 * v], q) / diam32(t, t->level[v]);
}

/* Eq. 5 with |B| from the tight boxes (box modes 1, 2), in FP64: p = min(1, max(1, d_v/B_v) /
 * (d_c/B_c)); d_c = 0 gives 1, and B_c = 0 < d_c gives 0 (beta~_c infinite). */
static double rr_prob_box(const otree *t, int64_t v, int64_t c, double dv, double dc)
{
    if (dc == 0.0) return 1.0;
    if (t->bd[c] == 0.0) return 0.0;
    double bt = dv / t->bd[v];
    double num = bt > 1.0 ? bt : 1.0;
    double r = num / (dc / t->bd[c]);
    return r < 1.0 ? r : 1.0;
}

/* Eq. 5 for the step from node v into its child c with the draw u: the path continues iff u < p,
 * p = min(1, max(1, beta~_v) / beta~_c), beta~ = ||q - p~|| / |B|. The child's cell is exactly
 * 2^(-(bits/3)(l_c - l_v)) times the node's, so p = min(1, X / d_c) with
 * X = max(d_v, |B_v|) 2^(-(bits/3)(l_c - l_v)) (exact in FP32), and u < p is u d_c < X, compared
 * exactly (the product of a 24-bit u and an FP32 d_c is exact in FP64). On a continue *p gets
 * fl32(X / d_c) capped at 1, the factor of p_rr. */
static int rr_continue32(const otree *t, int64_t v, int64_t c, const float q[3], int rr, float u, float *p)
{
    if (rr == RR_OFF) { *p = 1.0f; return 1; }
    if (rr == RR_HALF) { *p = 0.5f; return u < 0.5f; }
    if (t->box_mode != 0) {
        double pb = rr_prob_box(t, v, c, dist32(&t->com32[3 * v], q), dist32(&t->com32[3 * c], q));
        if (!((double)u < pb)) return 0;
        *p = (float)pb;
        return 1;
    }
    float dv = dist32(&t->com32[3 * v], q), dc = dist32(&t->com32[3 * c], q);
    float bv = diam32(t, t->level[v]);
    float X = ldexpf(dv > bv ? dv : bv, -(t->bits / 3) * (t->level[c] - t->level[v]));
    if (!((double)u * (double)dc < (double)X)) return 0;
    *p = dc > X ? X / dc : 1.0f;
    return 1;
}

/* Eq. 5 in exact arithmetic (FP64), used by the enumeration */
static double rr_prob64(const otree *t, int64_t v, int64_t c, const double q[3], int rr)
{
    if (rr == RR_OFF) return 1.0;
    if (rr == RR_HALF) return 0.5;
    double dv = 0, dc = 0;
    for (int a = 0; a < 3; ++a) {
        double x = t->com[3 * v + a] - q[a], y = t->com[3 * c + a] - q[a];
        dv += x * x; dc += y * y;
    }
    if (t->box_mode != 0) return rr_prob_box(t, v, c, sqrt(dv), sqrt(dc));
    double bt = sqrt(dv) / ldexp(sqrt(3.0) * t->side, -(t->bits / 3) * t->level[v]);
    double bc = sqrt(dc) / ldexp(sqrt(3.0) * t->side, -(t->bits / 3) * t->level[c]);
    double num = bt > 1.0 ? bt : 1.0;
    if (bc == 0.0) return 1.0;
    double r = num / bc;
    return r < 1.0 ? r : 1.0;
}

/* Child of v containing the path index (lazy draw). Mass: count the stored prefix fractions
 * cdf_c <= u among all but the last child. Count: the child holding the floor(u * |T|)-th point. */
static int64_t pick_child(const otree *t, int64_t v, uint32_t x, int sampling)
{
    int64_t fc = t->first_child[v];
    int nc = t->nchild[v];
    if (sampling == SAMPLE_COUNT) {
        int64_t cnt = t->end[v] - t->begin[v];
        int64_t target = t->begin[v] + (int64_t)(((uint64_t)(x >> 8) * (uint64_t)cnt) >> 24);
        int64_t c = 0;
        while (c + 1 < nc && t->begin[fc + c + 1] <= target) ++c;
        return fc + c;
    }
    float u = unit24f(x);
    int64_t c = 0;
    for (int j = 0; j < nc - 1; ++j)
        if (t->cdf[fc + j] <= u) ++c;
    return fc + c;
}

/* p(I in T_v) for a path rooted at subdomain a */
static double p_in(const otree *t, int64_t v, int64_t a, int sampling)
{
    if (sampling == SAMPLE_COUNT)
        return (double)(t->end[v] - t->begin[v]) / (double)(t->end[a] - t->begin[a]);
    return t->mass[v] / t->mass[a];
}

/* Contribution swap, Eq. 6: sum over children of m_c f(p_c, q), minus m_v f(p_v, q) */
static double swap_delta(const otree *t, const sbho_kernel *k, int64_t v, const double q[3])
{
    double s = 0;
    for (int c = 0; c < t->nchild[v]; ++c) s += node_term(t, k, t->first_child[v] + c, q);
    return s - node_term(t, k, v, q);
}

/* Scale of one node term in abs_sum. mode 0: |m f(p~, q)|, the scale of rounding the operations
 * of a signed sum of these terms. mode 1, for the winding kernel: the term's first-order change
 * when its record is rounded to FP32 (p~ and N each by a relative eps), divided by eps. With
 * d = p~ - q and r = |d|, the dot product d.N changes by at most eps (|p~| + r)|N| and r^-3 by a
 * factor 3 eps |p~| / r, and |d.N| <= r |N|, so the scale is |N| (r + 4 |p~|) / (4 pi r^3). Near
 * the query d is nearly tangent to the surface and d.N cancels, so this exceeds |term| by far.
 * Other kernels use mode 0 whatever the mode. */
static double node_mag(const otree *t, const sbho_kernel *k, int64_t v, const double q[3], int mode)
{
    if (mode == 0 || k->kind != K_WINDING) return fabs(node_term(t, k, v, q));
    const double *p = &t->com[3 * v], *N = &t->dip[3 * v];
    const double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) return 0.0;
    const double r = sqrt(r2);
    const double pn = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    const double nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    return nn * (r + 4.0 * pn) / (4.0 * M_PI * r2 * r);
}

/* Magnitude of a swap's terms: the children's scales plus the node's own (node_mag). The replay
 * adds these (with the same weights) into abs_sum, the scale against which a computation in lower
 * precision of the same signed sum can be compared. */
static double swap_abs(const otree *t, const sbho_kernel *k, int64_t v, const double q[3], int mode)
{
    double s = 0;
    for (int c = 0; c < t->nchild[v]; ++c) s += node_mag(t, k, t->first_child[v] + c, q, mode);
    return s + node_mag(t, k, v, q, mode);
}

static void node_grad(const otree *t, const sbho_kernel *k, int64_t v, const double q[3], double g[3])
{
    term_grad(k, &t->com[3 * v], t->mass[v], &t->dip[3 * v], q, g);
}

/* gradient of the contribution swap (Eq. 6) at node v with respect to q */
static void swap_grad(const otree *t, const sbho_kernel *k, int64_t v, const double q[3], double g[3])
{
    double gc[3];
    g[0] = g[1] = g[2] = 0.0;
    for (int c = 0; c < t->nchild[v]; ++c) {
        node_grad(t, k, t->first_child[v] + c, q, gc);
        for (int a = 0; a < 3; ++a) g[a] += gc[a];
    }
    node_grad(t, k, v, q, gc);
    for (int a = 0; a < 3; ++a) g[a] -= gc[a];
}

/* ------------------------------------------------------------------------------------------ */
/* Barnes-Hut, Algorithm 1: stop at a leaf or when beta~ >= beta, else recurse into children.   */
/* The far-field test is taken in FP32 (beta~ as above); sums are FP64.                        */
/* ------------------------------------------------------------------------------------------ */
static double bh_rec(const otree *t, const sbho_kernel *k, int64_t v, const double q[3],
                     const float q32[3], float beta)
{
    if (t->nchild[v] == 0 || ffratio32(t, v, q32) >= beta) return node_term(t, k, v, q);
    double F = 0;
    for (int c = 0; c < t->nchild[v]; ++c) F += bh_rec(t, k, t->first_child[v] + c, q, q32, beta);
    return F;
}

/* Algorithm 1's work at one query: the far-field tests of opened nodes plus the accepted terms */
static int64_t bh_work(const otree *t, int64_t v, const float q32[3], float beta)
{
    if (t->nchild[v] == 0 || ffratio32(t, v, q32) >= beta) return 1;
    int64_t w = 1;
    for (int c = 0; c < t->nchild[v]; ++c) w += bh_work(t, t->first_child[v] + c, q32, beta);
    return w;
}

SBHO_API void sbho_bh_work(const void *h, const float *queries, int64_t nq, float beta, int64_t *out)
{
    const otree *t = (const otree *)h;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < nq; ++j) {
        float q32[3] = {queries[3 * j], queries[3 * j + 1], queries[3 * j + 2]};
        out[j] = bh_work(t, 0, q32, beta);
    }
}

SBHO_API void sbho_bh(const void *h, const sbho_kernel *k, const float *queries, int64_t nq,
                      float beta, double *out)
{
    const otree *t = (const otree *)h;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < nq; ++j) {
        float q32[3] = {queries[3 * j], queries[3 * j + 1], queries[3 * j + 2]};
        double q[3] = {q32[0], q32[1], q32[2]};
        out[j] = bh_rec(t, k, 0, q, q32, beta);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Algorithm 2 (stratified path sample estimator), replayed with the Philox stream.             */
/* The counter's query index is qidx[j] when given (queries drawn from a larger set), else j.  */
/* abs_sum[j] (optional) gets the sum of the absolute values of every term the estimate adds.   */
/*   for each subdomain a (children of the root, Sec. 3.3.1):                                  */
/*     CV_a = m_a f(p_a, q);  F_a = 0                                                          */
/*     for s in 1..S: T = a, k = 0, p_rr = 1                                                   */
/*       while T is not a leaf:                                                                */
/*         c   = child of T containing I            (drawn lazily, first word)                 */
/*         p   = Eq. 5 for (T, c); stop unless      (exact test rand < p on FP32 inputs,       */
/*               rand < p                            second word)                               */
/*         Delta = Eq. 6 at T;  p_agg = p(I in T);  p_rr *= p                                  */
/*         F_a += Delta / (p_agg p_rr);  T = c;  k += 1                                        */
/*     F += CV_a + F_a / S                                                                     */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t sampling;   /* SAMPLE_MASS (default) or SAMPLE_COUNT (the paper's uniform index) */
    int32_t rr;         /* RR_PAPER (Eq. 5), RR_OFF, RR_HALF */
    int32_t coherent;   /* 1: every query uses query index 0 in the counter */
    int32_t abs_mode;   /* scale of each term in abs_sum (node_mag): 0 |term|, 1 FP32-record sensitivity */
} sbho_opts;

SBHO_API void sbho_replay(const void *h, const sbho_kernel *k, const float *queries, int64_t nq,
                          int32_t S, uint64_t seed, const sbho_opts *opts, const uint32_t *qidx,
                          double *out, int64_t *nswaps, double *abs_sum, int64_t *nterms)
{
    const otree *t = (const otree *)h;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const int sampling = opts ? opts->sampling : SAMPLE_MASS;
    const int rr = opts ? opts->rr : RR_PAPER;
    const int coherent = opts ? opts->coherent : 0;
    const int abs_mode = opts ? opts->abs_mode : 0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < nq; ++j) {
        float q32[3] = {queries[3 * j], queries[3 * j + 1], queries[3 * j + 2]};
        double q[3] = {q32[0], q32[1], q32[2]};
        double F = 0, A = 0;
        int64_t swaps = 0, terms = t->n_sub;  /* one control variate per subdomain */
        for (int64_t ai = 0; ai < t->n_sub; ++ai) {
            int64_t a = t->subs[ai];
            double CV = node_term(t, k, a, q);
            double Fa = 0, Aa = 0;
            for (int32_t s = 0; s < S; ++s) {
                int64_t T = a;
                uint32_t depth = 0;
                double prr = 1.0;
                while (t->nchild[T] > 0) {
                    uint32_t x[2];
                    decision_words(key, coherent ? 0u : (qidx ? qidx[j] : (uint32_t)j), (uint32_t)ai, (uint32_t)s,
                                   depth, x);
                    int64_t c = pick_child(t, T, x[0], sampling);
                    float p;
                    if (!rr_continue32(t, T, c, q32, rr, unit24f(x[1]), &p)) break;
                    double delta = swap_delta(t, k, T, q);
                    double pagg = p_in(t, T, a, sampling);
                    prr *= (double)p;
                    Fa += delta / (pagg * prr);
                    Aa += swap_abs(t, k, T, q, abs_mode) / (pagg * prr);
                    ++swaps;
                    terms += t->nchild[T] + 1;
                    T = c;
                    ++depth;
                }
            }
            F += CV + Fa / (double)S;
            A += node_mag(t, k, a, q, abs_mode) + Aa / (double)S;
        }
        out[j] = F;
        if (nswaps) nswaps[j] = swaps;
        if (abs_sum) abs_sum[j] = A;
        if (nterms) nterms[j] = terms;
    }
}

/* The same estimator applied to the kernel's query gradient: the paths, drawn exactly as in     */
/* sbho_replay (decisions at the FP32 query q_dec), and their weights 1 / (p_agg p_rr) are held  */
/* fixed, and every term m f is replaced by its gradient at q_val. Because the weights are those */
/* of a valid sampling of the same tree sums, E[grad] = grad F. With q_val = q_dec this is the    */
/* adjoint of the estimate; with q_val = q_dec +- h e_a it gives the frozen-path finite           */
/* difference. val[j] gets the estimate of F at q_val along the same paths, grad[3 j + a] the    */
/* gradient, abs_grad[j] the sum over terms of |gradient term|_1 (the rounding scale).            */
SBHO_API void sbho_replay_grad(const void *h, const sbho_kernel *k, const float *q_dec, const double *q_val,
                               int64_t nq, int32_t S, uint64_t seed, const sbho_opts *opts,
                               const uint32_t *qidx, double *val, double *grad, double *abs_grad)
{
    const otree *t = (const otree *)h;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const int sampling = opts ? opts->sampling : SAMPLE_MASS;
    const int rr = opts ? opts->rr : RR_PAPER;
    const int coherent = opts ? opts->coherent : 0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < nq; ++j) {
        float q32[3] = {q_dec[3 * j], q_dec[3 * j + 1], q_dec[3 * j + 2]};
        double q[3] = {q_val[3 * j], q_val[3 * j + 1], q_val[3 * j + 2]};
        double F = 0, G[3] = {0, 0, 0}, A = 0, g[3];
        for (int64_t ai = 0; ai < t->n_sub; ++ai) {
            int64_t a = t->subs[ai];
            F += node_term(t, k, a, q);
            node_grad(t, k, a, q, g);
            for (int c = 0; c < 3; ++c) { G[c] += g[c]; A += fabs(g[c]); }
            for (int32_t s = 0; s < S; ++s) {
                int64_t T = a;
                uint32_t depth = 0;
                double prr = 1.0;
                while (t->nchild[T] > 0) {
                    uint32_t x[2];
                    decision_words(key, coherent ? 0u : (qidx ? qidx[j] : (uint32_t)j), (uint32_t)ai, (uint32_t)s,
                                   depth, x);
                    int64_t ch = pick_child(t, T, x[0], sampling);
                    float p;
                    if (!rr_continue32(t, T, ch, q32, rr, unit24f(x[1]), &p)) break;
                    double pagg = p_in(t, T, a, sampling);
                    prr *= (double)p;
                    double wgt = 1.0 / (pagg * prr * (double)S);
                    F += wgt * swap_delta(t, k, T, q);
                    swap_grad(t, k, T, q, g);
                    for (int c = 0; c < 3; ++c) G[c] += wgt * g[c];
                    for (int cc = 0; cc <= t->nchild[T]; ++cc) {  /* children, then the node itself */
                        int64_t v = cc < t->nchild[T] ? t->first_child[T] + cc : T;
                        node_grad(t, k, v, q, g);
                        for (int c = 0; c < 3; ++c) A += wgt * fabs(g[c]);
                    }
                    T = ch;
                    ++depth;
                }
            }
        }
        val[j] = F;
        for (int c = 0; c < 3; ++c) grad[3 * j + c] = G[c];
        if (abs_grad) abs_grad[j] = A;
    }
}

/* Exact mean of the one-sample gradient estimator (S = 1) by enumeration, as sbho_enumerate. */
static void enum_grad_rec(const otree *t, const sbho_kernel *k, int64_t a, int64_t T, const double q[3],
                          double P, double prr, int sampling, int rr, double acc[3])
{
    if (t->nchild[T] == 0) return;
    double g[3];
    swap_grad(t, k, T, q, g);
    double pagg = p_in(t, T, a, sampling);
    int64_t fc = t->first_child[T];
    double tot = 0;
    for (int c = 0; c < t->nchild[T]; ++c)
        tot += (sampling == SAMPLE_COUNT) ? (double)(t->end[fc + c] - t->begin[fc + c]) : t->mass[fc + c];
    for (int c = 0; c < t->nchild[T]; ++c) {
        int64_t ch = fc + c;
        double w = (sampling == SAMPLE_COUNT) ? (double)(t->end[ch] - t->begin[ch]) : t->mass[ch];
        double pi = w / tot;
        double p = rr_prob64(t, T, ch, q, rr);
        double prr2 = prr * p;
        if (!(p > 0.0)) continue;
        /* this path continues with probability P pi p and then carries the swap term */
        for (int d = 0; d < 3; ++d) acc[d] += P * pi * p * g[d] / (pagg * prr2);
        enum_grad_rec(t, k, a, ch, q, P * pi * p, prr2, sampling, rr, acc);
    }
}

SBHO_API void sbho_enumerate_grad(const void *h, const sbho_kernel *k, const float *queries, int64_t nq,
                                  const sbho_opts *opts, double *mean)
{
    const otree *t = (const otree *)h;
    const int sampling = opts ? opts->sampling : SAMPLE_MASS;
    const int rr = opts ? opts->rr : RR_PAPER;
    for (int64_t j = 0; j < nq; ++j) {
        double q[3] = {queries[3 * j], queries[3 * j + 1], queries[3 * j + 2]};
        double E[3] = {0, 0, 0}, g[3];
        for (int64_t ai = 0; ai < t->n_sub; ++ai) {
            int64_t a = t->subs[ai];
            node_grad(t, k, a, q, g);
            for (int d = 0; d < 3; ++d) E[d] += g[d];
            enum_grad_rec(t, k, a, a, q, 1.0, 1.0, sampling, rr, E);
        }
        for (int d = 0; d < 3; ++d) mean[3 * j + d] = E[d];
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Subdomains taken per query as the Barnes-Hut contribution nodes at beta_s (Sec. 3.3.1 names  */
/* this cover as an alternative to the root's children): Algorithm 1's walk with parameter      */
/* beta_s gives nodes that partition the sources; each one gets its control variate and one path */
/* of Algorithm 2 started from it (the decisions' words as in sbho_replay, with the node's index */
/* in the walk's order for the subdomain index and sample 0). An oracle-only study of the paper's alternative; the CUDA path does not build it. */
/* work[j] counts the walk's far-field tests, plus a swap's children and node for every swap.    */
/* ------------------------------------------------------------------------------------------ */
static void bh_cut(const otree *t, int64_t v, const float q32[3], float beta, int64_t *out, int64_t *n,
                   int64_t *tests)
{
    ++*tests;
    if (t->nchild[v] == 0 || ffratio32(t, v, q32) >= beta) { out[(*n)++] = v; return; }
    for (int c = 0; c < t->nchild[v]; ++c) bh_cut(t, t->first_child[v] + c, q32, beta, out, n, tests);
}

SBHO_API void sbho_replay_cut(const void *h, const sbho_kernel *k, const float *queries, int64_t nq, float beta_s,
                              uint64_t seed, double *out, int64_t *work)
{
    const otree *t = (const otree *)h;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel
    {
        int64_t *subs = (int64_t *)malloc((size_t)t->n_nodes * sizeof(int64_t));
#pragma omp for schedule(dynamic, 4)
        for (int64_t j = 0; j < nq; ++j) {
            float q32[3] = {queries[3 * j], queries[3 * j + 1], queries[3 * j + 2]};
            double q[3] = {q32[0], q32[1], q32[2]};
            int64_t ns = 0, tests = 0;
            bh_cut(t, 0, q32, beta_s, subs, &ns, &tests);
            double F = 0;
            int64_t W = tests;
            for (int64_t ai = 0; ai < ns; ++ai) {
                int64_t a = subs[ai], T = a;
                uint32_t depth = 0;
                double prr = 1.0;
                F += node_term(t, k, a, q);
                while (t->nchild[T] > 0) {
                    uint32_t x[2];
                    decision_words(key, (uint32_t)j, (uint32_t)ai, 0u, depth, x);
                    int64_t c = pick_child(t, T, x[0], SAMPLE_MASS);
                    float p;
                    if (!rr_continue32(t, T, c, q32, RR_PAPER, unit24f(x[1]), &p)) break;
                    prr *= (double)p;
                    F += swap_delta(t, k, T, q) / (p_in(t, T, a, SAMPLE_MASS) * prr);
                    W += t->nchild[T] + 1;
                    T = c;
                    ++depth;
                }
            }
            out[j] = F;
            if (work) work[j] = W;
        }
        free(subs);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Learned child proposal (a project extension; the paper samples the path index uniformly and  */
/* names importance sampling as future work, Sec. 3.3). A 6-32-32-1 ReLU network scores each    */
/* child c of a node T from query-relative features; the proposal mixes its softmax with the    */
/* mass-proportional one: pi_c = (1 - eps) softmax(s)_c + eps m_c / m_T, every pi_c > 0, so the  */
/* estimator stays unbiased with p_agg the product of the pi's along the path.                   */
/* Parameter layout (1313 values): W1[32][6], b1[32], W2[32][32], b2[32], w3[32], b3.           */
/* ------------------------------------------------------------------------------------------ */
typedef struct { double e1, e2; } moments;  /* sums of P V and P V^2 over outcomes */

enum { MLP_IN = 6, MLP_H = 32, MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1 };

/* features of child c of node T at query q:
 *   ln(d_c / |B_c|), ln(m_c / m_T), ln(|B_c| / |B_T|), ln(d_c / d_T),
 *   |N_c| / m_c and cos(p_c - q, N_c) (dipole kernel only, else 0); distances guarded by 1e-6 |B| */
static void child_features(const otree *t, int64_t T, int64_t c, const double q[3], int use_dipole, double x[6])
{
    double dT = 0, dc = 0, v[3];
    for (int a = 0; a < 3; ++a) {
        double y = t->com[3 * T + a] - q[a];
        v[a] = t->com[3 * c + a] - q[a];
        dT += y * y;
        dc += v[a] * v[a];
    }
    double BT = ldexp(sqrt(3.0) * t->side, -(t->bits / 3) * t->level[T]);
    double Bc = ldexp(sqrt(3.0) * t->side, -(t->bits / 3) * t->level[c]);
    dT = sqrt(dT) + 1e-6 * BT;
    dc = sqrt(dc) + 1e-6 * Bc;
    x[0] = log(dc / Bc);
    x[1] = log(t->mass[c] / t->mass[T]);
    x[2] = log(Bc / BT);
    x[3] = log(dc / dT);
    x[4] = 0.0;
    x[5] = 0.0;
    if (use_dipole) {
        const double *N = &t->dip[3 * c];
        double nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        x[4] = nn / t->mass[c];
        x[5] = nn > 0 ? (v[0] * N[0] + v[1] * N[1] + v[2] * N[2]) / (dc * nn) : 0.0;
    }
}

/* score of one feature row; h1, h2 (optional) receive the hidden activations */
static double mlp_score(const double *w, const double x[6], double *h1o, double *h2o)
{
    const double *W1 = w, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H,
                 *w3 = b2 + MLP_H, *b3 = w3 + MLP_H;
    double h1[MLP_H], h2[MLP_H];
    for (int i = 0; i < MLP_H; ++i) {
        double z = b1[i];
        for (int k = 0; k < MLP_IN; ++k) z += W1[i * MLP_IN + k] * x[k];
        h1[i] = z > 0 ? z : 0;
    }
    double s = b3[0];
    for (int i = 0; i < MLP_H; ++i) {
        double z = b2[i];
        for (int k = 0; k < MLP_H; ++k) z += W2[i * MLP_H + k] * h1[k];
        h2[i] = z > 0 ? z : 0;
        s += w3[i] * h2[i];
    }
    if (h1o) memcpy(h1o, h1, sizeof(h1));
    if (h2o) memcpy(h2o, h2, sizeof(h2));
    return s;
}

SBHO_API int32_t sbho_mlp_nparam(void) { return MLP_NPARAM; }

SBHO_API void sbho_mlp_forward(const double *w, const double *feats, int64_t n, double *scores)
{
    for (int64_t r = 0; r < n; ++r) scores[r] = mlp_score(w, &feats[6 * r], NULL, NULL);
}

/* Loss over decision sets (rows off[s] .. off[s+1]-1): mean over sets of the cross-entropy
 * -sum_c t_c log softmax(s)_c with targets t normalised per set; grad (MLP_NPARAM) of the loss. */
SBHO_API double sbho_mlp_loss_grad(const double *w, const double *feats, const double *targets, const int64_t *off,
                                   int64_t n_sets, double *grad)
{
    memset(grad, 0, sizeof(double) * MLP_NPARAM);
    double *gW1 = grad, *gb1 = gW1 + MLP_H * MLP_IN, *gW2 = gb1 + MLP_H, *gb2 = gW2 + MLP_H * MLP_H,
           *gw3 = gb2 + MLP_H, *gb3 = gw3 + MLP_H;
    const double *W2 = w + MLP_H * MLP_IN + MLP_H, *w3 = W2 + MLP_H * MLP_H + MLP_H;
    double loss = 0;
    for (int64_t st = 0; st < n_sets; ++st) {
        int64_t r0 = off[st], r1 = off[st + 1];
        int64_t nc = r1 - r0;
        double *sc = (double *)malloc(sizeof(double) * (size_t)nc);
        double mx = -1e300, tsum = 0;
        for (int64_t r = r0; r < r1; ++r) {
            sc[r - r0] = mlp_score(w, &feats[6 * r], NULL, NULL);
            if (sc[r - r0] > mx) mx = sc[r - r0];
            tsum += targets[r];
        }
        double z = 0;
        for (int64_t i = 0; i < nc; ++i) z += exp(sc[i] - mx);
        for (int64_t r = r0; r < r1; ++r) {
            double pr = exp(sc[r - r0] - mx) / z;
            double tr = tsum > 0 ? targets[r] / tsum : 1.0 / (double)nc;  /* all-zero targets: no preference */
            loss -= tr * (sc[r - r0] - mx - log(z)) / (double)n_sets;
            double ds = (pr - tr) / (double)n_sets;  /* d loss / d score */
            double h1[MLP_H], h2[MLP_H], dh2[MLP_H], dh1[MLP_H];
            mlp_score(w, &feats[6 * r], h1, h2);
            gb3[0] += ds;
            for (int i = 0; i < MLP_H; ++i) {
                gw3[i] += ds * h2[i];
                dh2[i] = h2[i] > 0 ? ds * w3[i] : 0.0;
                gb2[i] += dh2[i];
            }
            for (int k = 0; k < MLP_H; ++k) {
                double acc = 0;
                for (int i = 0; i < MLP_H; ++i) {
                    gW2[i * MLP_H + k] += dh2[i] * h1[k];
                    acc += W2[i * MLP_H + k] * dh2[i];
                }
                dh1[k] = h1[k] > 0 ? acc : 0.0;
                gb1[k] += dh1[k];
                for (int m = 0; m < MLP_IN; ++m) gW1[k * MLP_IN + m] += dh1[k] * feats[6 * r + m];
            }
        }
        free(sc);
    }
    return loss;
}

/* Proposal probabilities of the children of T. Where the network is used -- at most 64 children
 * and the query nearer than `near` cell diagonals, d_T < near |B_T| (FP32, the same test as the
 * GPU's) -- pi_c = (1 - eps) softmax(s)_c + eps m_c / m_T with the scores clamped to [-40, 40];
 * elsewhere the mass proportion m_c / m_T. Any proposal with every pi_c > 0 keeps the estimator
 * unbiased (Appendix A with p_agg the product of the pi's along the path). */
#define MLP_MAX_CHILDREN 64
#define MLP_SCORE_CLAMP 40.0
static void learned_probs(const otree *t, const double *w, double eps, int use_dipole, float near, int64_t T,
                          const double q[3], const float q32[3], double *pi)
{
    int nc = t->nchild[T];
    int64_t fc = t->first_child[T];
    double z = 0, mt = 0, x[6];
    for (int c = 0; c < nc; ++c) mt += t->mass[fc + c];
    const float reach = near * diam32(t, t->level[T]);
    if (nc > MLP_MAX_CHILDREN || !(dist32(&t->com32[3 * T], q32) < reach)) {
        for (int c = 0; c < nc; ++c) pi[c] = t->mass[fc + c] / mt;
        return;
    }
    for (int c = 0; c < nc; ++c) {
        child_features(t, T, fc + c, q, use_dipole, x);
        double sc = mlp_score(w, x, NULL, NULL);
        sc = sc < -MLP_SCORE_CLAMP ? -MLP_SCORE_CLAMP : (sc > MLP_SCORE_CLAMP ? MLP_SCORE_CLAMP : sc);
        pi[c] = exp(sc);
        z += pi[c];
    }
    for (int c = 0; c < nc; ++c) pi[c] = (1.0 - eps) * pi[c] / z + eps * t->mass[fc + c] / mt;
}

/* features of every child of T at q, rows written to x (6 per child) */
SBHO_API void sbho_child_features(const void *h, int64_t T, const float *q32, int32_t use_dipole, double *x)
{
    const otree *t = (const otree *)h;
    double q[3] = {q32[0], q32[1], q32[2]};
    for (int c = 0; c < t->nchild[T]; ++c) child_features(t, T, t->first_child[T] + c, q, use_dipole, &x[6 * c]);
}

/* exact mean and variance of the one-sample estimator with the learned proposal */
static void enum_learned_rec(const otree *t, const sbho_kernel *k, const double *w, double eps, float near,
                             int64_t T, const double q[3], const float q32[3], double P, double V, double ppath,
                             double prr, moments *acc)
{
    if (t->nchild[T] == 0) { acc->e1 += P * V; acc->e2 += P * V * V; return; }
    double delta = swap_delta(t, k, T, q);
    int nc = t->nchild[T];
    double *pi = (double *)malloc(sizeof(double) * (size_t)nc);
    learned_probs(t, w, eps, k->kind == K_WINDING, near, T, q, q32, pi);
    for (int c = 0; c < nc; ++c) {
        int64_t ch = t->first_child[T] + c;
        double p = rr_prob64(t, T, ch, q, RR_PAPER);
        double Pstop = P * pi[c] * (1.0 - p);
        acc->e1 += Pstop * V;
        acc->e2 += Pstop * V * V;
        double prr2 = prr * p;
        if (p > 0.0) enum_learned_rec(t, k, w, eps, near, ch, q, q32, P * pi[c] * p, V + delta / (ppath * prr2), ppath * pi[c],
                         prr2, acc);
    }
    free(pi);
}

SBHO_API void sbho_enumerate_learned(const void *h, const sbho_kernel *k, const double *w, double eps, float near,
                                     const float *queries, int64_t nq, double *mean, double *var)
{
    const otree *t = (const otree *)h;
    for (int64_t j = 0; j < nq; ++j) {
        double q[3] = {queries[3 * j], queries[3 * j + 1], queries[3 * j + 2]};
        const float *q32 = &queries[3 * j];
        double E = 0, Var = 0;
        for (int64_t ai = 0; ai < t->n_sub; ++ai) {
            int64_t a = t->subs[ai];
            moments m = {0, 0};
            enum_learned_rec(t, k, w, eps, near, a, q, q32, 1.0, 0.0, 1.0, 1.0, &m);
            E += node_term(t, k, a, q) + m.e1;
            Var += m.e2 - m.e1 * m.e1;
        }
        mean[j] = E;
        var[j] = Var;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Exact mean and variance of the one-sample estimator (S = 1) by enumerating every outcome    */
/* of the sampler: at node T reached with probability P and running estimate V, each child c   */
/* is taken with probability pi_c and continued with probability p (Eq. 5); stopping ends the  */
/* path with value V, continuing adds Delta_T / (p_agg p_rr). This is the sum the proof of the */
/* theorem (Appendix A) rearranges. Subdomains are independent, so variances add.             */
/* ------------------------------------------------------------------------------------------ */

static void enum_rec(const otree *t, const sbho_kernel *k, int64_t a, int64_t T, const double q[3],
                     double P, double V, double prr, int sampling, int rr, moments *acc)
{
    if (t->nchild[T] == 0) { acc->e1 += P * V; acc->e2 += P * V * V; return; }
    double delta = swap_delta(t, k, T, q);
    double pagg = p_in(t, T, a, sampling);
    int64_t fc = t->first_child[T];
    double tot = 0;
    for (int c = 0; c < t->nchild[T]; ++c)
        tot += (sampling == SAMPLE_COUNT) ? (double)(t->end[fc + c] - t->begin[fc + c]) : t->mass[fc + c];
    for (int c = 0; c < t->nchild[T]; ++c) {
        int64_t ch = fc + c;
        double w = (sampling == SAMPLE_COUNT) ? (double)(t->end[ch] - t->begin[ch]) : t->mass[ch];
        double pi = w / tot;
        double p = rr_prob64(t, T, ch, q, rr);
        double Pstop = P * pi * (1.0 - p);
        acc->e1 += Pstop * V;
        acc->e2 += Pstop * V * V;
        double prr2 = prr * p;
        if (p > 0.0) enum_rec(t, k, a, ch, q, P * pi * p, V + delta / (pagg * prr2), prr2, sampling, rr, acc);
    }
}

/* mean[j] = E[F_1(q_j)], var[j] = Var[F_1(q_j)] */
SBHO_API void sbho_enumerate(const void *h, const sbho_kernel *k, const float *queries, int64_t nq,
                             const sbho_opts *opts, double *mean, double *var)
{
    const otree *t = (const otree *)h;
    const int sampling = opts ? opts->sampling : SAMPLE_MASS;
    const int rr = opts ? opts->rr : RR_PAPER;
    for (int64_t j = 0; j < nq; ++j) {
        double q[3] = {queries[3 * j], queries[3 * j + 1], queries[3 * j + 2]};
        double E = 0, Var = 0;
        for (int64_t ai = 0; ai < t->n_sub; ++ai) {
            int64_t a = t->subs[ai];
            moments m = {0, 0};
            enum_rec(t, k, a, a, q, 1.0, 0.0, 1.0, sampling, rr, &m);
            E += node_term(t, k, a, q) + m.e1;
            Var += m.e2 - m.e1 * m.e1;
        }
        mean[j] = E;
        var[j] = Var;
    }
}


/* exact mean and variance of the one-sample estimator with the Barnes-Hut-cut subdomains */
SBHO_API void sbho_enumerate_cut(const void *h, const sbho_kernel *k, const float *queries, int64_t nq, float beta_s,
                                 double *mean, double *var)
{
    const otree *t = (const otree *)h;
    int64_t *subs = (int64_t *)malloc((size_t)t->n_nodes * sizeof(int64_t));
    for (int64_t j = 0; j < nq; ++j) {
        const float *q32 = &queries[3 * j];
        double q[3] = {q32[0], q32[1], q32[2]};
        int64_t ns = 0, tests = 0;
        bh_cut(t, 0, q32, beta_s, subs, &ns, &tests);
        double E = 0, Var = 0;
        for (int64_t ai = 0; ai < ns; ++ai) {
            moments m = {0, 0};
            enum_rec(t, k, subs[ai], subs[ai], q, 1.0, 0.0, 1.0, SAMPLE_MASS, RR_PAPER, &m);
            E += node_term(t, k, subs[ai], q) + m.e1;
            Var += m.e2 - m.e1 * m.e1;
        }
        mean[j] = E;
        var[j] = Var;
    }
    free(subs);
}

/* thread control for the timed CPU baseline */
SBHO_API int32_t sbho_max_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

SBHO_API void sbho_set_threads(int32_t n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
