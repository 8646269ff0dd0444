/*
 * bonsai_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for the
 * per-step gravitational tree force of Bonsai (Bedorf et al., SC14,
 * "24.77 Pflops on a Gravitational Tree-Code to Simulate the Milky Way
 * Galaxy with 18600 GPUs").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  The CUDA library never
 * includes, links or calls it, and it shares no code with the CUDA library.
 *
 * What it computes, in the paper's order (Sec. III.A: tree construction,
 * multipole moments, tree walk with force evaluation; Sec. III.B.2 end:
 * leap-frog):
 *
 *   O1  direct summation, the exact target the tree approximates (Sec. I.A:
 *       every particle feels the N-1 others), Eq. 1-2 with Q = 0 and Plummer
 *       softening:  a_i = G sum_{j!=i} m_j r_ij / (r_ij^2+eps^2)^{3/2},
 *       phi_i = -G sum_{j!=i} m_j / (r_ij^2+eps^2)^{1/2},  r_ij = r_j - r_i.
 *   O2  the tree method step by step:
 *       1. bounding cube (Sec. III.B.1: local bounding box -> PH keys),
 *       2. 21-bit quantisation and Peano-Hilbert key (Sec. III.B.1, Fig. 2),
 *       3. sort by key (Table 2 "Sorting SFC"),
 *       4. octree: octants split until a node holds at most 16 particles
 *          (Sec. I.A, "critical value ... 16"), children in key order,
 *       5. walk groups (nodes of <= 64 particles whose parent has more),
 *       6. multipoles: mass, centre of mass, 3x3 symmetric quadrupole
 *          (Sec. VI.A below Eq. 2) by a parallel-axis upward pass,
 *       7. multipole acceptance criterion parameterised by theta (Sec. I.A),
 *       8. p-c and p-p evaluation by Eq. 1-2, softened, times G,
 *       9. counters n_pp, n_pc "recorded during execution" (Sec. VI.A),
 *      10. kick-drift-kick leap-frog (Sec. III.B.2 end) and diagnostics.
 *
 * Readings where the paper is silent (each one also listed in the design
 * notes): 21 bits per axis (63-bit key); Skilling's transpose form of the
 * Hilbert curve with axis 0 most significant in each 3-bit digit; leaf rule
 * count <= 16; group = node with <= 64 particles whose parent has > 64
 * (a max-depth leaf with > 64 particles is cut into runs of 64); MAC
 * "open if d^2 < r_open^2" with r_open = l/theta + |com - centre| and d the
 * distance from the cell's com to the group's box, evaluated in FP32 on
 * FP32-rounded inputs; Plummer softening in every power of |r| in Eq. 1-2;
 * the self pair j == i contributes nothing (it is counted in n_pp).
 *
 * Arithmetic: every floating-point expression is written in the order it is
 * meant to be evaluated, and the file is built with -ffp-contract=off so that
 * no multiply-add is fused.  Key math and multipoles are FP64, the MAC is
 * FP32 on rounded inputs, forces are FP64.
 *
 * Parity pins (closed forms, brute force, invariants) live in the test suite;
 * the adjoint part (frozen-list VJP) is pinned by finite differences.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_KEY_BITS 21
#define ORC_MAX_LEVEL 21

/* ------------------------------------------------------------------------ */
/* 1. Bounding cube (Sec. III.B.1: "each GPU computes its local bounding box",
 *    whose geometry maps coordinates to PH keys).  Reading: the cube is the
 *    box's largest extent widened by 2^-20 relative, centred on the box.    */
/* ------------------------------------------------------------------------ */
void orc_bounding_cube(int64_t n, const double *x, const double *y,
                       const double *z, double lo_out[3], double *L_out) {
    const double *c[3] = {x, y, z};
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = c[d][0];
        hi[d] = c[d][0];
        for (int64_t i = 1; i < n; ++i) {
            if (c[d][i] < lo[d]) lo[d] = c[d][i];
            if (c[d][i] > hi[d]) hi[d] = c[d][i];
        }
    }
    double ext = hi[0] - lo[0];
    if (hi[1] - lo[1] > ext) ext = hi[1] - lo[1];
    if (hi[2] - lo[2] > ext) ext = hi[2] - lo[2];
    double L = ext * (1.0 + 0x1p-20);
    if (ext == 0.0) L = 1.0;
    for (int d = 0; d < 3; ++d) {
        double w = hi[d] - lo[d];
        lo[d] = lo[d] - (L - w) * 0.5;
        lo_out[d] = lo[d];
    }
    *L_out = L;
}

/* Quantise one coordinate to 21 bits: floor((x - lo) * 2^21 / L), clamped. */
static uint32_t orc_quantise(double xv, double lo, double scale) {
    double t = (xv - lo) * scale;
    double f = floor(t);
    if (!(f >= 0.0)) return 0u; /* also catches NaN */
    if (f > (double)((1u << ORC_KEY_BITS) - 1u)) return (1u << ORC_KEY_BITS) - 1u;
    return (uint32_t)f;
}

/* ------------------------------------------------------------------------ */
/* 2. Peano-Hilbert key (Sec. III.B.1, Fig. 2).  The curve is J. Skilling's
 *    "Programming the Hilbert curve" (AIP Conf. Proc. 707, 2004): the axes
 *    are converted to the transposed Hilbert index, then its bits are
 *    interleaved most significant level first, axis 0 first in each digit.
 *    Written here from the published description.                         */
/* ------------------------------------------------------------------------ */
uint64_t orc_hilbert_key(uint32_t q0, uint32_t q1, uint32_t q2, int bits) {
    uint32_t X[3] = {q0, q1, q2};
    const int n = 3;
    uint32_t top = 1u << (bits - 1);
    /* undo excess work: walk the levels from the top down */
    for (uint32_t Q = top; Q > 1; Q >>= 1) {
        uint32_t P = Q - 1;
        for (int i = 0; i < n; ++i) {
            if (X[i] & Q) {
                X[0] ^= P; /* invert low bits of axis 0 */
            } else {
                uint32_t t = (X[0] ^ X[i]) & P; /* exchange low bits */
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    /* Gray encode */
    for (int i = 1; i < n; ++i) X[i] ^= X[i - 1];
    uint32_t t = 0;
    for (uint32_t Q = top; Q > 1; Q >>= 1)
        if (X[n - 1] & Q) t ^= Q - 1;
    for (int i = 0; i < n; ++i) X[i] ^= t;
    /* interleave: level b-1 first, axis 0 most significant in each digit */
    uint64_t key = 0;
    for (int b = bits - 1; b >= 0; --b)
        for (int i = 0; i < n; ++i) key = (key << 1) | ((X[i] >> b) & 1u);
    return key;
}

/* ------------------------------------------------------------------------ */
/* The tree oracle state.  Every array is in sorted (key) order unless the  */
/* name says otherwise; positions are SoA [3][n].                           */
/* ------------------------------------------------------------------------ */
typedef struct orc_tree {
    int64_t n;
    int nleaf, ncrit;
    double lo[3], L, scale;
    uint64_t *key;  /* sorted keys */
    uint32_t *perm; /* sorted slot -> caller index */
    uint32_t *q;    /* quantised coordinates [3][n], sorted */
    double *x;      /* positions [3][n], sorted */
    double *m;      /* masses, sorted */
    /* nodes, breadth-first */
    int64_t nnodes, cap;
    uint32_t *first, *count, *child, *nchild, *level, *parent;
    double *M, *com, *Q, *centre, *side; /* com/centre [3][nn], Q [6][nn] */
    /* groups */
    int64_t ngroups;
    uint32_t *gfirst, *gcount;
    double *gcentre, *ghalf; /* [3][ng] */
} orc_tree;

typedef struct {
    uint64_t key;
    uint32_t idx;
} orc_pair;

static int orc_pair_cmp(const void *a, const void *b) {
    const orc_pair *p = (const orc_pair *)a, *r = (const orc_pair *)b;
    if (p->key < r->key) return -1;
    if (p->key > r->key) return 1;
    return (p->idx < r->idx) ? -1 : (p->idx > r->idx);
}

static int orc_grow_nodes(orc_tree *t) {
    int64_t nc = t->cap ? 2 * t->cap : 1024;
    uint32_t **arrs[6] = {&t->first, &t->count, &t->child, &t->nchild, &t->level, &t->parent};
    for (int k = 0; k < 6; ++k) {
        uint32_t *p = (uint32_t *)realloc(*arrs[k], (size_t)nc * sizeof(uint32_t));
        if (!p) return -1;
        *arrs[k] = p;
    }
    t->cap = nc;
    return 0;
}

static int64_t orc_add_node(orc_tree *t, uint32_t first, uint32_t count, uint32_t level,
                            uint32_t parent) {
    if (t->nnodes == t->cap && orc_grow_nodes(t)) return -1;
    int64_t i = t->nnodes++;
    t->first[i] = first;
    t->count[i] = count;
    t->child[i] = 0;
    t->nchild[i] = 0;
    t->level[i] = level;
    t->parent[i] = parent;
    return i;
}

/* 3-bit digit of a key at tree level l (level 1 is the top digit). */
static uint32_t orc_digit(uint64_t key, uint32_t l) {
    return (uint32_t)((key >> (3 * (ORC_MAX_LEVEL - l))) & 7u);
}

/* 4. Octree (Sec. I.A: octants are split recursively until a node holds no
 *    more than the critical 16 particles).  Breadth-first, children are the
 *    non-empty octants in key order, numbered contiguously.                */
static int orc_build_octree(orc_tree *t) {
    if (orc_add_node(t, 0, (uint32_t)t->n, 0, 0) < 0) return -1;
    for (int64_t i = 0; i < t->nnodes; ++i) {
        uint32_t f = t->first[i], c = t->count[i], l = t->level[i];
        if (c <= (uint32_t)t->nleaf || l >= ORC_MAX_LEVEL) continue; /* leaf */
        t->child[i] = (uint32_t)t->nnodes;
        uint32_t run_start = f;
        for (uint32_t k = f + 1; k <= f + c; ++k) {
            if (k == f + c || orc_digit(t->key[k], l + 1) != orc_digit(t->key[run_start], l + 1)) {
                if (orc_add_node(t, run_start, k - run_start, l + 1, (uint32_t)i) < 0) return -1;
                t->nchild[i] += 1;
                run_start = k;
            }
        }
    }
    return 0;
}

static int orc_group_cmp(const void *a, const void *b) {
    const uint32_t *p = (const uint32_t *)a, *r = (const uint32_t *)b;
    return (p[0] < r[0]) ? -1 : (p[0] > r[0]);
}

/* 5. Groups: a node with <= ncrit particles whose parent has more (the root
 *    if it has <= ncrit); a max-depth leaf with more than ncrit particles is
 *    cut into consecutive runs of ncrit.  Each group's FP64 bounding box
 *    gives its centre and half-size.                                       */
static int orc_make_groups(orc_tree *t) {
    int64_t cap = 1024, ng = 0;
    uint32_t *g = (uint32_t *)malloc((size_t)cap * 2 * sizeof(uint32_t));
    if (!g) return -1;
    uint32_t ncrit = (uint32_t)t->ncrit;
    for (int64_t i = 0; i < t->nnodes; ++i) {
        uint32_t c = t->count[i];
        int is_leaf = (t->nchild[i] == 0);
        int parent_big = (i == 0) || (t->count[t->parent[i]] > ncrit);
        if (!parent_big) continue;
        if (c <= ncrit || is_leaf) {
            for (uint32_t s = 0; s < c; s += ncrit) {
                if (ng == cap) {
                    cap *= 2;
                    uint32_t *p = (uint32_t *)realloc(g, (size_t)cap * 2 * sizeof(uint32_t));
                    if (!p) { free(g); return -1; }
                    g = p;
                }
                g[2 * ng] = t->first[i] + s;
                g[2 * ng + 1] = (c - s < ncrit) ? (c - s) : ncrit;
                ++ng;
            }
        }
    }
    qsort(g, (size_t)ng, 2 * sizeof(uint32_t), orc_group_cmp);
    t->ngroups = ng;
    t->gfirst = (uint32_t *)malloc((size_t)ng * sizeof(uint32_t));
    t->gcount = (uint32_t *)malloc((size_t)ng * sizeof(uint32_t));
    t->gcentre = (double *)malloc((size_t)ng * 3 * sizeof(double));
    t->ghalf = (double *)malloc((size_t)ng * 3 * sizeof(double));
    if (!t->gfirst || !t->gcount || !t->gcentre || !t->ghalf) { free(g); return -1; }
    for (int64_t k = 0; k < ng; ++k) {
        t->gfirst[k] = g[2 * k];
        t->gcount[k] = g[2 * k + 1];
        for (int d = 0; d < 3; ++d) {
            const double *xd = t->x + (size_t)d * t->n;
            double mn = xd[g[2 * k]], mx = xd[g[2 * k]];
            for (uint32_t j = g[2 * k]; j < g[2 * k] + g[2 * k + 1]; ++j) {
                if (xd[j] < mn) mn = xd[j];
                if (xd[j] > mx) mx = xd[j];
            }
            t->gcentre[(size_t)d * ng + k] = (mn + mx) * 0.5;
            t->ghalf[(size_t)d * ng + k] = (mx - mn) * 0.5;
        }
    }
    free(g);
    return 0;
}

/* 6. Multipole moments (Sec. VI.A: mass, position and 3x3 symmetric Q of
 *    each cell).  Q is the non-traceless second moment about the centre of
 *    mass, Q = sum m (x-com)(x-com)^T: expanding -sum m_k/|r - d_k| to
 *    second order about the com gives exactly Eq. 1 in that case.  Leaves
 *    sum their particles; internal cells combine children by the parallel-
 *    axis rule.  Q component order: xx, yy, zz, xy, xz, yz.                 */
static void orc_multipoles(orc_tree *t) {
    int64_t nn = t->nnodes, n = t->n;
    for (int64_t i = nn - 1; i >= 0; --i) {
        double M = 0.0, s[3] = {0.0, 0.0, 0.0}, com[3], Q[6] = {0, 0, 0, 0, 0, 0};
        if (t->nchild[i] == 0) {
            uint32_t f = t->first[i], c = t->count[i];
            for (uint32_t j = f; j < f + c; ++j) {
                M = M + t->m[j];
                for (int d = 0; d < 3; ++d) s[d] = s[d] + t->m[j] * t->x[(size_t)d * n + j];
            }
            for (int d = 0; d < 3; ++d) com[d] = s[d] / M;
            for (uint32_t j = f; j < f + c; ++j) {
                double dx = t->x[j] - com[0];
                double dy = t->x[(size_t)n + j] - com[1];
                double dz = t->x[2 * (size_t)n + j] - com[2];
                double mj = t->m[j];
                Q[0] = Q[0] + (mj * dx) * dx;
                Q[1] = Q[1] + (mj * dy) * dy;
                Q[2] = Q[2] + (mj * dz) * dz;
                Q[3] = Q[3] + (mj * dx) * dy;
                Q[4] = Q[4] + (mj * dx) * dz;
                Q[5] = Q[5] + (mj * dy) * dz;
            }
        } else {
            uint32_t c0 = t->child[i], nc = t->nchild[i];
            for (uint32_t k = c0; k < c0 + nc; ++k) {
                M = M + t->M[k];
                for (int d = 0; d < 3; ++d) s[d] = s[d] + t->M[k] * t->com[(size_t)d * nn + k];
            }
            for (int d = 0; d < 3; ++d) com[d] = s[d] / M;
            for (uint32_t k = c0; k < c0 + nc; ++k) {
                double dx = t->com[k] - com[0];
                double dy = t->com[(size_t)nn + k] - com[1];
                double dz = t->com[2 * (size_t)nn + k] - com[2];
                double Mk = t->M[k];
                Q[0] = Q[0] + (t->Q[k] + (Mk * dx) * dx);
                Q[1] = Q[1] + (t->Q[(size_t)nn + k] + (Mk * dy) * dy);
                Q[2] = Q[2] + (t->Q[2 * (size_t)nn + k] + (Mk * dz) * dz);
                Q[3] = Q[3] + (t->Q[3 * (size_t)nn + k] + (Mk * dx) * dy);
                Q[4] = Q[4] + (t->Q[4 * (size_t)nn + k] + (Mk * dx) * dz);
                Q[5] = Q[5] + (t->Q[5 * (size_t)nn + k] + (Mk * dy) * dz);
            }
        }
        t->M[i] = M;
        for (int d = 0; d < 3; ++d) t->com[(size_t)d * nn + i] = com[d];
        for (int k = 0; k < 6; ++k) t->Q[(size_t)k * nn + i] = Q[k];
        /* geometric cube: the level-l octant holding the node's particles */
        uint32_t l = t->level[i];
        double side = ldexp(t->L, -(int)l);
        t->side[i] = side;
        for (int d = 0; d < 3; ++d) {
            uint32_t kq = t->q[(size_t)d * n + t->first[i]] >> (ORC_KEY_BITS - l);
            t->centre[(size_t)d * nn + i] = t->lo[d] + ((double)kq + 0.5) * side;
        }
    }
}

void orc_tree_free(orc_tree *t) {
    if (!t) return;
    free(t->key); free(t->perm); free(t->q); free(t->x); free(t->m);
    free(t->first); free(t->count); free(t->child); free(t->nchild); free(t->level);
    free(t->parent);
    free(t->M); free(t->com); free(t->Q); free(t->centre); free(t->side);
    free(t->gfirst); free(t->gcount); free(t->gcentre); free(t->ghalf);
    free(t);
}

/* Steps 1-6: bounding cube, keys, sort, octree, groups, multipoles.
 * Positions are caller-order SoA [3][n]; nothing is kept from the caller. */
orc_tree *orc_tree_build(int64_t n, const double *pos, const double *mass, int nleaf,
                         int ncrit) {
    if (n <= 0 || nleaf < 1 || ncrit < 1) return NULL;
    orc_tree *t = (orc_tree *)calloc(1, sizeof(orc_tree));
    if (!t) return NULL;
    t->n = n;
    t->nleaf = nleaf;
    t->ncrit = ncrit;
    orc_bounding_cube(n, pos, pos + n, pos + 2 * n, t->lo, &t->L);
    t->scale = 0x1p21 / t->L;
    orc_pair *pairs = (orc_pair *)malloc((size_t)n * sizeof(orc_pair));
    uint32_t *qc = (uint32_t *)malloc((size_t)n * 3 * sizeof(uint32_t));
    t->key = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    t->perm = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    t->q = (uint32_t *)malloc((size_t)n * 3 * sizeof(uint32_t));
    t->x = (double *)malloc((size_t)n * 3 * sizeof(double));
    t->m = (double *)malloc((size_t)n * sizeof(double));
    if (!pairs || !qc || !t->key || !t->perm || !t->q || !t->x || !t->m) {
        free(pairs); free(qc); orc_tree_free(t);
        return NULL;
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int d = 0; d < 3; ++d)
            qc[(size_t)d * n + i] = orc_quantise(pos[(size_t)d * n + i], t->lo[d], t->scale);
        pairs[i].key = orc_hilbert_key(qc[i], qc[(size_t)n + i], qc[2 * (size_t)n + i], ORC_KEY_BITS);
        pairs[i].idx = (uint32_t)i;
    }
    /* 3. sort ascending by (key, caller index) */
    qsort(pairs, (size_t)n, sizeof(orc_pair), orc_pair_cmp);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t j = pairs[i].idx;
        t->key[i] = pairs[i].key;
        t->perm[i] = j;
        t->m[i] = mass[j];
        for (int d = 0; d < 3; ++d) {
            t->x[(size_t)d * n + i] = pos[(size_t)d * n + j];
            t->q[(size_t)d * n + i] = qc[(size_t)d * n + j];
        }
    }
    free(pairs);
    free(qc);
    if (orc_build_octree(t) || orc_make_groups(t)) { orc_tree_free(t); return NULL; }
    int64_t nn = t->nnodes;
    t->M = (double *)malloc((size_t)nn * sizeof(double));
    t->com = (double *)malloc((size_t)nn * 3 * sizeof(double));
    t->Q = (double *)malloc((size_t)nn * 6 * sizeof(double));
    t->centre = (double *)malloc((size_t)nn * 3 * sizeof(double));
    t->side = (double *)malloc((size_t)nn * sizeof(double));
    if (!t->M || !t->com || !t->Q || !t->centre || !t->side) { orc_tree_free(t); return NULL; }
    orc_multipoles(t);
    return t;
}

/* ---- accessors (copy out) ---------------------------------------------- */
int64_t orc_tree_num_nodes(const orc_tree *t) { return t->nnodes; }
int64_t orc_tree_num_groups(const orc_tree *t) { return t->ngroups; }

void orc_tree_cube(const orc_tree *t, double lo[3], double *L) {
    for (int d = 0; d < 3; ++d) lo[d] = t->lo[d];
    *L = t->L;
}

void orc_tree_keys(const orc_tree *t, uint64_t *key, uint32_t *perm) {
    memcpy(key, t->key, (size_t)t->n * sizeof(uint64_t));
    memcpy(perm, t->perm, (size_t)t->n * sizeof(uint32_t));
}

void orc_tree_nodes(const orc_tree *t, uint32_t *first, uint32_t *count, uint32_t *child,
                    uint32_t *nchild, uint32_t *level) {
    size_t b = (size_t)t->nnodes * sizeof(uint32_t);
    memcpy(first, t->first, b);
    memcpy(count, t->count, b);
    memcpy(child, t->child, b);
    memcpy(nchild, t->nchild, b);
    memcpy(level, t->level, b);
}

void orc_tree_multipoles(const orc_tree *t, double *M, double *com, double *Q, double *centre,
                         double *side) {
    size_t nn = (size_t)t->nnodes;
    memcpy(M, t->M, nn * sizeof(double));
    memcpy(com, t->com, 3 * nn * sizeof(double));
    memcpy(Q, t->Q, 6 * nn * sizeof(double));
    memcpy(centre, t->centre, 3 * nn * sizeof(double));
    memcpy(side, t->side, nn * sizeof(double));
}

void orc_tree_groups(const orc_tree *t, uint32_t *first, uint32_t *count, double *centre,
                     double *half) {
    size_t ng = (size_t)t->ngroups;
    memcpy(first, t->gfirst, ng * sizeof(uint32_t));
    memcpy(count, t->gcount, ng * sizeof(uint32_t));
    memcpy(centre, t->gcentre, 3 * ng * sizeof(double));
    memcpy(half, t->ghalf, 3 * ng * sizeof(double));
}

/* ------------------------------------------------------------------------ */
/* 7. Multipole acceptance criterion (Sec. I.A: an opening angle theta
 *    decides whether a distant octant is used whole).  Reading:
 *      r_open = l / theta + |com - centre|     (FP64, rounded to FP32 once)
 *      d_k    = max(|com_k - c_k| - h_k, 0)    (distance com -> group box)
 *      open  <=>  d_x^2 + d_y^2 + d_z^2 < r_open^2   (FP32, this op order)
 *    com and the group centre are rounded to nearest FP32, the group half-
 *    size is rounded up to FP32.                                           */
/* ------------------------------------------------------------------------ */
static float orc_round_up_f32(double v) {
    float f = (float)v;
    if ((double)f < v) f = nextafterf(f, INFINITY);
    return f;
}

void orc_cell_mac(const orc_tree *t, float theta, float *com_f, float *ropen2_f) {
    int64_t nn = t->nnodes;
    double th = (double)theta;
    for (int64_t i = 0; i < nn; ++i) {
        double dx = t->com[i] - t->centre[i];
        double dy = t->com[(size_t)nn + i] - t->centre[(size_t)nn + i];
        double dz = t->com[2 * (size_t)nn + i] - t->centre[2 * (size_t)nn + i];
        double s = sqrt((dx * dx + dy * dy) + dz * dz);
        double r_open = t->side[i] / th + s;
        ropen2_f[i] = (float)(r_open * r_open);
        for (int d = 0; d < 3; ++d) com_f[(size_t)d * nn + i] = (float)t->com[(size_t)d * nn + i];
    }
}

void orc_group_box_f32(const orc_tree *t, float *centre_f, float *half_f) {
    size_t ng = (size_t)t->ngroups;
    for (size_t k = 0; k < 3 * ng; ++k) {
        centre_f[k] = (float)t->gcentre[k];
        half_f[k] = orc_round_up_f32(t->ghalf[k]);
    }
}

static int orc_mac_open(const float cf[3], float r2, const float gc[3], const float gh[3]) {
    float a[3];
    for (int d = 0; d < 3; ++d) {
        float v = fabsf(cf[d] - gc[d]) - gh[d];
        a[d] = v > 0.0f ? v : 0.0f;
    }
    float d2 = (a[0] * a[0] + a[1] * a[1]) + a[2] * a[2];
    return d2 < r2;
}

/* ------------------------------------------------------------------------ */
/* 8. Eq. 1-2 for one source on one target, Plummer-softened: every |r| is
 *    replaced by s = (|r|^2 + eps^2)^{1/2}.  r = r_j - r_i (source minus
 *    target).  Accumulates phi and a without the factor G.                */
/* ------------------------------------------------------------------------ */
static void orc_eq12(const double r[3], double mj, const double *Qj /* 6 or NULL */, double eps2,
                     double *phi, double a[3]) {
    double s2 = ((r[0] * r[0] + r[1] * r[1]) + r[2] * r[2]) + eps2;
    double s = sqrt(s2);
    double s3 = s2 * s, s5 = s3 * s2, s7 = s5 * s2;
    *phi -= mj / s;
    for (int d = 0; d < 3; ++d) a[d] += mj * r[d] / s3;
    if (Qj) {
        double trQ = (Qj[0] + Qj[1]) + Qj[2];
        double Qr[3];
        Qr[0] = (Qj[0] * r[0] + Qj[3] * r[1]) + Qj[4] * r[2];
        Qr[1] = (Qj[3] * r[0] + Qj[1] * r[1]) + Qj[5] * r[2];
        Qr[2] = (Qj[4] * r[0] + Qj[5] * r[1]) + Qj[2] * r[2];
        double rQr = (r[0] * Qr[0] + r[1] * Qr[1]) + r[2] * Qr[2];
        *phi += 0.5 * trQ / s3;
        *phi -= 1.5 * rQr / s5;
        for (int d = 0; d < 3; ++d) {
            a[d] -= 1.5 * trQ * r[d] / s5;
            a[d] -= 3.0 * Qr[d] / s5;
            a[d] += 7.5 * rQr * r[d] / s7;
        }
    }
}

/* One source of Eq. 1-2 on one target, exported so that the test suite can
 * pin the formula on its own (Q may be NULL for a point mass).  r = source
 * minus target; returns G phi and G a.                                    */
void orc_eval_source(const double r[3], double mj, const double *Qj, double eps, double G,
                     double *phi_out, double a_out[3]) {
    double phi = 0.0, a[3] = {0.0, 0.0, 0.0};
    orc_eq12(r, mj, Qj, eps * eps, &phi, a);
    *phi_out = G * phi;
    for (int d = 0; d < 3; ++d) a_out[d] = G * a[d];
}

/* Interaction lists of one group: a depth-first walk from the root. */
typedef struct {
    uint32_t *pc;
    int64_t npc, cap_pc;
    uint32_t *pp; /* leaf node ids whose particles are p-p sources */
    int64_t npp_leaves, cap_pp, npp;
} orc_lists;

static void orc_push(uint32_t **a, int64_t *n, int64_t *cap, uint32_t v) {
    if (*n == *cap) {
        *cap = *cap ? 2 * *cap : 256;
        *a = (uint32_t *)realloc(*a, (size_t)*cap * sizeof(uint32_t));
    }
    (*a)[(*n)++] = v;
}

static void orc_walk_group(const orc_tree *t, const float *com_f, const float *ropen2_f,
                           const float gc[3], const float gh[3], orc_lists *L) {
    int64_t nn = t->nnodes;
    uint32_t stack[ORC_MAX_LEVEL * 8 + 16];
    int sp = 0;
    L->npc = L->npp_leaves = L->npp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        uint32_t c = stack[--sp];
        float cf[3] = {com_f[c], com_f[(size_t)nn + c], com_f[2 * (size_t)nn + c]};
        if (!orc_mac_open(cf, ropen2_f[c], gc, gh)) {
            orc_push(&L->pc, &L->npc, &L->cap_pc, c);
        } else if (t->nchild[c] == 0) {
            orc_push(&L->pp, &L->npp_leaves, &L->cap_pp, c);
            L->npp += t->count[c];
        } else {
            /* push in reverse so children are visited in key order */
            for (int k = (int)t->nchild[c] - 1; k >= 0; --k) stack[sp++] = t->child[c] + (uint32_t)k;
        }
    }
}

/* The interaction lists of group g (for tests): the accepted cells and the
 * opened leaves, each in walk order.  Returns the list lengths in n_out
 * (n_out[0] cells, n_out[1] leaves); copies at most cap entries of each.  */
int orc_group_lists(const orc_tree *t, float theta, int64_t g, uint32_t *pc, uint32_t *leaves,
                    int64_t cap, int64_t n_out[2]) {
    int64_t nn = t->nnodes, ng = t->ngroups;
    if (g < 0 || g >= ng) return -1;
    float *com_f = (float *)malloc((size_t)nn * 3 * sizeof(float));
    float *ropen2_f = (float *)malloc((size_t)nn * sizeof(float));
    float *gcf = (float *)malloc((size_t)ng * 3 * sizeof(float));
    float *ghf = (float *)malloc((size_t)ng * 3 * sizeof(float));
    if (!com_f || !ropen2_f || !gcf || !ghf) {
        free(com_f); free(ropen2_f); free(gcf); free(ghf);
        return -1;
    }
    orc_cell_mac(t, theta, com_f, ropen2_f);
    orc_group_box_f32(t, gcf, ghf);
    float gc[3] = {gcf[g], gcf[(size_t)ng + g], gcf[2 * (size_t)ng + g]};
    float gh[3] = {ghf[g], ghf[(size_t)ng + g], ghf[2 * (size_t)ng + g]};
    orc_lists L;
    memset(&L, 0, sizeof(L));
    orc_walk_group(t, com_f, ropen2_f, gc, gh, &L);
    for (int64_t k = 0; k < L.npc && k < cap; ++k) pc[k] = L.pc[k];
    for (int64_t k = 0; k < L.npp_leaves && k < cap; ++k) leaves[k] = L.pp[k];
    n_out[0] = L.npc;
    n_out[1] = L.npp_leaves;
    free(L.pc); free(L.pp);
    free(com_f); free(ropen2_f); free(gcf); free(ghf);
    return 0;
}

/* Steps 7-9 for the listed groups: FP64 tree forces in sorted order (acc
 * [3][n], pot [n]; only the groups' particles are written), per-group list
 * lengths, and the counts n_pp = sum |g| |pp|, n_pc = sum |g| |pc|.      */
int orc_tree_forces_list(const orc_tree *t, float theta, double eps, double G, int64_t nlist,
                         const int64_t *glist, double *acc, double *pot, int64_t *g_npp,
                         int64_t *g_npc, uint64_t counts[2]) {
    int64_t n = t->n, nn = t->nnodes, ng = t->ngroups;
    for (int64_t k = 0; k < nlist; ++k)
        if (glist[k] < 0 || glist[k] >= ng) return -1;
    float *com_f = (float *)malloc((size_t)nn * 3 * sizeof(float));
    float *ropen2_f = (float *)malloc((size_t)nn * sizeof(float));
    float *gcf = (float *)malloc((size_t)ng * 3 * sizeof(float));
    float *ghf = (float *)malloc((size_t)ng * 3 * sizeof(float));
    if (!com_f || !ropen2_f || !gcf || !ghf) {
        free(com_f); free(ropen2_f); free(gcf); free(ghf);
        return -1;
    }
    orc_cell_mac(t, theta, com_f, ropen2_f);
    orc_group_box_f32(t, gcf, ghf);
    double eps2 = eps * eps;
    uint64_t npp_tot = 0, npc_tot = 0;
#pragma omp parallel reduction(+ : npp_tot, npc_tot)
    {
        orc_lists L;
        memset(&L, 0, sizeof(L));
#pragma omp for schedule(dynamic, 1)
        for (int64_t k = 0; k < nlist; ++k) {
            int64_t g = glist[k];
            float gc[3] = {gcf[g], gcf[(size_t)ng + g], gcf[2 * (size_t)ng + g]};
            float gh[3] = {ghf[g], ghf[(size_t)ng + g], ghf[2 * (size_t)ng + g]};
            orc_walk_group(t, com_f, ropen2_f, gc, gh, &L);
            uint32_t f = t->gfirst[g], c = t->gcount[g];
            if (g_npp) g_npp[g] = L.npp;
            if (g_npc) g_npc[g] = L.npc;
            npp_tot += (uint64_t)c * (uint64_t)L.npp;
            npc_tot += (uint64_t)c * (uint64_t)L.npc;
            for (uint32_t i = f; i < f + c; ++i) {
                double xi[3] = {t->x[i], t->x[(size_t)n + i], t->x[2 * (size_t)n + i]};
                double phi = 0.0, a[3] = {0.0, 0.0, 0.0};
                for (int64_t k = 0; k < L.npc; ++k) {
                    uint32_t cc = L.pc[k];
                    double r[3], Qc[6];
                    for (int d = 0; d < 3; ++d) r[d] = t->com[(size_t)d * nn + cc] - xi[d];
                    for (int q = 0; q < 6; ++q) Qc[q] = t->Q[(size_t)q * nn + cc];
                    orc_eq12(r, t->M[cc], Qc, eps2, &phi, a);
                }
                for (int64_t k = 0; k < L.npp_leaves; ++k) {
                    uint32_t lf = L.pp[k];
                    for (uint32_t j = t->first[lf]; j < t->first[lf] + t->count[lf]; ++j) {
                        if (j == i) continue; /* self pair: contributes nothing */
                        double r[3];
                        for (int d = 0; d < 3; ++d) r[d] = t->x[(size_t)d * n + j] - xi[d];
                        orc_eq12(r, t->m[j], NULL, eps2, &phi, a);
                    }
                }
                pot[i] = G * phi;
                for (int d = 0; d < 3; ++d) acc[(size_t)d * n + i] = G * a[d];
            }
        }
        free(L.pc);
        free(L.pp);
    }
    if (counts) {
        counts[0] = npp_tot;
        counts[1] = npc_tot;
    }
    free(com_f); free(ropen2_f); free(gcf); free(ghf);
    return 0;
}

/* Steps 7-9 for the contiguous groups [g0, g1). */
int orc_tree_forces(const orc_tree *t, float theta, double eps, double G, int64_t g0, int64_t g1,
                    double *acc, double *pot, int64_t *g_npp, int64_t *g_npc, uint64_t counts[2]) {
    if (g0 < 0) g0 = 0;
    if (g1 > t->ngroups) g1 = t->ngroups;
    if (g1 < g0) g1 = g0;
    int64_t *gl = (int64_t *)malloc((size_t)(g1 - g0 + 1) * sizeof(int64_t));
    if (!gl) return -1;
    for (int64_t g = g0; g < g1; ++g) gl[g - g0] = g;
    int rc = orc_tree_forces_list(t, theta, eps, G, g1 - g0, gl, acc, pot, g_npp, g_npc, counts);
    free(gl);
    return rc;
}

/* Positions and masses in sorted order, and the sorted slot of each caller
 * index is perm^-1; these let a caller map sorted outputs back.           */
void orc_tree_sorted_state(const orc_tree *t, double *pos, double *mass) {
    memcpy(pos, t->x, (size_t)t->n * 3 * sizeof(double));
    memcpy(mass, t->m, (size_t)t->n * sizeof(double));
}

/* ------------------------------------------------------------------------ */
/* O1. Direct summation over all sources for the listed targets (Sec. I.A,
 *     O(N^2); Eq. 1-2 with monopoles only), FP64, sources in index order. */
/* ------------------------------------------------------------------------ */
void orc_direct_forces(int64_t n, const double *pos, const double *mass, double eps, double G,
                       int64_t nt, const int64_t *targets, double *acc, double *pot) {
    double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < nt; ++k) {
        int64_t i = targets ? targets[k] : k;
        double xi[3] = {pos[i], pos[n + i], pos[2 * n + i]};
        double phi = 0.0, a[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r[3] = {pos[j] - xi[0], pos[n + j] - xi[1], pos[2 * n + j] - xi[2]};
            orc_eq12(r, mass[j], NULL, eps2, &phi, a);
        }
        pot[k] = G * phi;
        for (int d = 0; d < 3; ++d) acc[(size_t)d * nt + k] = G * a[d];
    }
}

/* Tree forces in caller order for all particles (convenience for the
 * integrator): builds the tree, evaluates every group, un-permutes.       */
static int orc_forces_caller(int64_t n, const double *pos, const double *mass, int nleaf,
                             int ncrit, float theta, double eps, double G, int direct,
                             double *acc, double *pot, uint64_t counts[2]) {
    if (direct) {
        orc_direct_forces(n, pos, mass, eps, G, n, NULL, acc, pot);
        if (counts) { counts[0] = (uint64_t)n * (uint64_t)n; counts[1] = 0; }
        return 0;
    }
    orc_tree *t = orc_tree_build(n, pos, mass, nleaf, ncrit);
    if (!t) return -1;
    double *as = (double *)malloc((size_t)n * 3 * sizeof(double));
    double *ps = (double *)malloc((size_t)n * sizeof(double));
    if (!as || !ps) { free(as); free(ps); orc_tree_free(t); return -1; }
    int rc = orc_tree_forces(t, theta, eps, G, 0, t->ngroups, as, ps, NULL, NULL, counts);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t j = t->perm[i];
        pot[j] = ps[i];
        for (int d = 0; d < 3; ++d) acc[(size_t)d * n + j] = as[(size_t)d * n + i];
    }
    free(as); free(ps); orc_tree_free(t);
    return rc;
}

int orc_forces(int64_t n, const double *pos, const double *mass, int nleaf, int ncrit,
               float theta, double eps, double G, int direct, double *acc, double *pot,
               uint64_t counts[2]) {
    return orc_forces_caller(n, pos, mass, nleaf, ncrit, theta, eps, G, direct, acc, pot, counts);
}

/* ------------------------------------------------------------------------ */
/* 10. Second-order leap-frog (Sec. III.B.2 end), kick-drift-kick:
 *       v += a dt/2;  x += v dt;  a = forces(x);  v += a dt/2.
 *     acc/pot hold the forces at the current positions on entry (computed
 *     here when *have_acc == 0) and at the final positions on exit.       */
/* ------------------------------------------------------------------------ */
int orc_kdk(int64_t n, double *pos, double *vel, const double *mass, int nsteps, double dt,
            int nleaf, int ncrit, float theta, double eps, double G, int direct, double *acc,
            double *pot, int have_acc) {
    if (!have_acc &&
        orc_forces_caller(n, pos, mass, nleaf, ncrit, theta, eps, G, direct, acc, pot, NULL))
        return -1;
    double h = 0.5 * dt;
    for (int s = 0; s < nsteps; ++s) {
        for (int64_t k = 0; k < 3 * n; ++k) vel[k] = vel[k] + acc[k] * h;
        for (int64_t k = 0; k < 3 * n; ++k) pos[k] = pos[k] + vel[k] * dt;
        if (orc_forces_caller(n, pos, mass, nleaf, ncrit, theta, eps, G, direct, acc, pot, NULL))
            return -1;
        for (int64_t k = 0; k < 3 * n; ++k) vel[k] = vel[k] + acc[k] * h;
    }
    return 0;
}

/* Diagnostics (Sec. VI: "gather and write statistics", excluded from the
 * flop count): out = {E_kin, E_pot, E_tot, Px, Py, Pz, Lx, Ly, Lz, M}
 * with E_kin = sum m v^2 / 2, E_pot = sum m phi / 2, P = sum m v,
 * L = sum m x cross v.                                                    */
void orc_diagnostics(int64_t n, const double *pos, const double *vel, const double *mass,
                     const double *pot, double out[10]) {
    double ek = 0, ep = 0, P[3] = {0, 0, 0}, Lm[3] = {0, 0, 0}, Mt = 0;
    for (int64_t i = 0; i < n; ++i) {
        double m = mass[i];
        double x = pos[i], y = pos[n + i], z = pos[2 * n + i];
        double vx = vel[i], vy = vel[n + i], vz = vel[2 * n + i];
        ek += 0.5 * m * ((vx * vx + vy * vy) + vz * vz);
        ep += 0.5 * m * pot[i];
        P[0] += m * vx;
        P[1] += m * vy;
        P[2] += m * vz;
        Lm[0] += m * (y * vz - z * vy);
        Lm[1] += m * (z * vx - x * vz);
        Lm[2] += m * (x * vy - y * vx);
        Mt += m;
    }
    out[0] = ek;
    out[1] = ep;
    out[2] = ek + ep;
    out[3] = P[0]; out[4] = P[1]; out[5] = P[2];
    out[6] = Lm[0]; out[7] = Lm[1]; out[8] = Lm[2];
    out[9] = Mt;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
