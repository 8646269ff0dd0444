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
 *       5. walk groups (runs of consecutive sibling cells of <= 64
 *          particles each, at most 64 in all, under a cell with more),
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
 * count <= 16; group = a run of consecutive children (each with <= 64
 * particles) of a node with > 64, at most 64 particles in all, formed
 * greedily in key order (a max-depth leaf with > 64 particles is cut into
 * runs of 64; the root is the one group when it has <= 64); MAC
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
    /* frozen interaction lists (adjoint): per group, offsets into the lists */
    int64_t *pc_off, *lf_off;
    uint32_t *pc_list, *lf_list;
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

/* 5. Groups.  Under every node with more than ncrit particles, its children
 *    that hold at most ncrit particles are taken in key order and gathered
 *    into runs: a child joins the current run while the run's total stays
 *    at most ncrit, otherwise it starts the next run; a child with more
 *    than ncrit particles ends the run (its own children form groups one
 *    level down).  Each run is one group: a contiguous range of the sorted
 *    particles.  The root is the single group if it has at most ncrit; a
 *    max-depth leaf with more than ncrit particles is cut into consecutive
 *    runs of ncrit.  Each group's FP64 bounding box gives its centre and
 *    half-size.                                                            */
static int orc_push_group(uint32_t **g, int64_t *cap, int64_t *ng, uint32_t first, uint32_t count) {
    if (*ng == *cap) {
        *cap *= 2;
        uint32_t *p = (uint32_t *)realloc(*g, (size_t)*cap * 2 * sizeof(uint32_t));
        if (!p) return -1;
        *g = p;
    }
    (*g)[2 * *ng] = first;
    (*g)[2 * *ng + 1] = count;
    ++*ng;
    return 0;
}

static int orc_make_groups(orc_tree *t) {
    int64_t cap = 1024, ng = 0;
    uint32_t *g = (uint32_t *)malloc((size_t)cap * 2 * sizeof(uint32_t));
    if (!g) return -1;
    uint32_t ncrit = (uint32_t)t->ncrit;
    int rc = 0;
    if (t->count[0] <= ncrit) rc = orc_push_group(&g, &cap, &ng, t->first[0], t->count[0]);
    for (int64_t i = 0; i < t->nnodes && rc == 0; ++i) {
        uint32_t c = t->count[i];
        if (c <= ncrit) continue;
        if (t->nchild[i] == 0) {  /* a max-depth leaf: runs of ncrit */
            for (uint32_t s = 0; s < c && rc == 0; s += ncrit)
                rc = orc_push_group(&g, &cap, &ng, t->first[i] + s, (c - s < ncrit) ? (c - s) : ncrit);
            continue;
        }
        uint32_t run_first = 0, run_count = 0;
        int open = 0;
        for (uint32_t k = 0; k < t->nchild[i] && rc == 0; ++k) {
            uint32_t j = t->child[i] + k;
            if (t->count[j] > ncrit) {          /* a big child ends the run */
                if (open) rc = orc_push_group(&g, &cap, &ng, run_first, run_count);
                open = 0;
                continue;
            }
            if (open && run_count + t->count[j] <= ncrit) {
                run_count += t->count[j];
            } else {
                if (open) rc = orc_push_group(&g, &cap, &ng, run_first, run_count);
                run_first = t->first[j];
                run_count = t->count[j];
                open = 1;
            }
        }
        if (open && rc == 0) rc = orc_push_group(&g, &cap, &ng, run_first, run_count);
    }
    if (rc) { free(g); return -1; }
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
static void orc_upward(const orc_tree *t, const double *x, const double *m, double *Mo,
                       double *como, double *Qo) {
    int64_t nn = t->nnodes, n = t->n;
    for (int64_t i = nn - 1; i >= 0; --i) {
        double M = 0.0, s[3] = {0.0, 0.0, 0.0}, com[3], Q[6] = {0, 0, 0, 0, 0, 0};
        if (t->nchild[i] == 0) {
            uint32_t f = t->first[i], c = t->count[i];
            for (uint32_t j = f; j < f + c; ++j) {
                M = M + m[j];
                for (int d = 0; d < 3; ++d) s[d] = s[d] + m[j] * x[(size_t)d * n + j];
            }
            for (int d = 0; d < 3; ++d) com[d] = s[d] / M;
            for (uint32_t j = f; j < f + c; ++j) {
                double dx = x[j] - com[0];
                double dy = x[(size_t)n + j] - com[1];
                double dz = x[2 * (size_t)n + j] - com[2];
                double mj = m[j];
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
                M = M + Mo[k];
                for (int d = 0; d < 3; ++d) s[d] = s[d] + Mo[k] * como[(size_t)d * nn + k];
            }
            for (int d = 0; d < 3; ++d) com[d] = s[d] / M;
            for (uint32_t k = c0; k < c0 + nc; ++k) {
                double dx = como[k] - com[0];
                double dy = como[(size_t)nn + k] - com[1];
                double dz = como[2 * (size_t)nn + k] - com[2];
                double Mk = Mo[k];
                Q[0] = Q[0] + (Qo[k] + (Mk * dx) * dx);
                Q[1] = Q[1] + (Qo[(size_t)nn + k] + (Mk * dy) * dy);
                Q[2] = Q[2] + (Qo[2 * (size_t)nn + k] + (Mk * dz) * dz);
                Q[3] = Q[3] + (Qo[3 * (size_t)nn + k] + (Mk * dx) * dy);
                Q[4] = Q[4] + (Qo[4 * (size_t)nn + k] + (Mk * dx) * dz);
                Q[5] = Q[5] + (Qo[5 * (size_t)nn + k] + (Mk * dy) * dz);
            }
        }
        Mo[i] = M;
        for (int d = 0; d < 3; ++d) como[(size_t)d * nn + i] = com[d];
        for (int k = 0; k < 6; ++k) Qo[(size_t)k * nn + i] = Q[k];
    }
}

static void orc_multipoles(orc_tree *t) {
    int64_t nn = t->nnodes, n = t->n;
    orc_upward(t, t->x, t->m, t->M, t->com, t->Q);
    for (int64_t i = 0; i < nn; ++i) {
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
    free(t->pc_off); free(t->lf_off); free(t->pc_list); free(t->lf_list);
    free(t);
}

/* Steps 1-6: bounding cube, keys, sort, octree, groups, multipoles.
 * Positions are caller-order SoA [3][n]; nothing is kept from the caller. */
/* Steps 1-6 with the cube given (lo, L), or the bounding cube if lo is
 * NULL.  A given cube makes the trees of several particle subsets branches
 * of one global octree (Sec. III.B.1: the global bounding box maps every
 * process's coordinates to global PH keys).                               */
static orc_tree *orc_tree_build_in(int64_t n, const double *pos, const double *mass, int nleaf,
                                   int ncrit, const double *lo, double L) {
    if (n <= 0 || nleaf < 1 || ncrit < 1) return NULL;
    orc_tree *t = (orc_tree *)calloc(1, sizeof(orc_tree));
    if (!t) return NULL;
    t->n = n;
    t->nleaf = nleaf;
    t->ncrit = ncrit;
    if (lo) {
        for (int d = 0; d < 3; ++d) t->lo[d] = lo[d];
        t->L = L;
    } else {
        orc_bounding_cube(n, pos, pos + n, pos + 2 * n, t->lo, &t->L);
    }
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

orc_tree *orc_tree_build(int64_t n, const double *pos, const double *mass, int nleaf,
                         int ncrit) {
    return orc_tree_build_in(n, pos, mass, nleaf, ncrit, NULL, 0.0);
}

orc_tree *orc_tree_build_cube(int64_t n, const double *pos, const double *mass, int nleaf,
                              int ncrit, const double lo[3], double L) {
    if (!(L > 0.0)) return NULL;
    return orc_tree_build_in(n, pos, mass, nleaf, ncrit, lo, L);
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

/* ------------------------------------------------------------------------ */
/* Local essential trees (Sec. III.B.2): the part of a process's tree that
 * a remote process needs is what the remote groups' walks visit in it.   */
/* ------------------------------------------------------------------------ */

/* Marks, for every group of dst, the walk of src's tree with that group's
 * box: visited[c] = 1 for every cell the walk reaches, opened[c] = 1 for
 * every cell it opens (an internal cell's children are visited, a leaf's
 * particles become p-p sources).  Visited cells that no group opens are
 * used whole.                                                              */
int orc_let_mark(const orc_tree *src, const orc_tree *dst, float theta, uint8_t *visited,
                 uint8_t *opened) {
    int64_t nn = src->nnodes, ng = dst->ngroups;
    float *com_f = (float *)malloc((size_t)nn * 3 * sizeof(float));
    float *ropen2_f = (float *)malloc((size_t)nn * sizeof(float));
    float *gcf = (float *)malloc((size_t)ng * 3 * sizeof(float));
    float *ghf = (float *)malloc((size_t)ng * 3 * sizeof(float));
    uint32_t *stack = (uint32_t *)malloc(((size_t)ORC_MAX_LEVEL * 8 + 16) * sizeof(uint32_t));
    if (!com_f || !ropen2_f || !gcf || !ghf || !stack) {
        free(com_f); free(ropen2_f); free(gcf); free(ghf); free(stack);
        return -1;
    }
    orc_cell_mac(src, theta, com_f, ropen2_f);
    orc_group_box_f32(dst, gcf, ghf);
    memset(visited, 0, (size_t)nn);
    memset(opened, 0, (size_t)nn);
    for (int64_t g = 0; g < ng; ++g) {
        float gc[3] = {gcf[g], gcf[(size_t)ng + g], gcf[2 * (size_t)ng + g]};
        float gh[3] = {ghf[g], ghf[(size_t)ng + g], ghf[2 * (size_t)ng + g]};
        int sp = 0;
        stack[sp++] = 0;
        while (sp > 0) {
            uint32_t c = stack[--sp];
            visited[c] = 1;
            float cf[3] = {com_f[c], com_f[(size_t)nn + c], com_f[2 * (size_t)nn + c]};
            if (!orc_mac_open(cf, ropen2_f[c], gc, gh)) continue;
            opened[c] = 1;
            for (int k = (int)src->nchild[c] - 1; k >= 0; --k) stack[sp++] = src->child[c] + (uint32_t)k;
        }
    }
    free(com_f); free(ropen2_f); free(gcf); free(ghf); free(stack);
    return 0;
}

/* The force of src's particles on dst's particles through the walks of
 * dst's groups over src's tree (Eq. 1-2, FP64, without self pairs: the two
 * particle sets are disjoint).  acc [3][dst n], pot [dst n] in dst's sorted
 * order (overwritten); per-group list lengths; counts as for the tree.   */
int orc_cross_forces(const orc_tree *src, const orc_tree *dst, float theta, double eps, double G,
                     double *acc, double *pot, int64_t *g_npp, int64_t *g_npc, uint64_t counts[2]) {
    int64_t ns = src->n, nd = dst->n, nn = src->nnodes, ng = dst->ngroups;
    float *com_f = (float *)malloc((size_t)nn * 3 * sizeof(float));
    float *ropen2_f = (float *)malloc((size_t)nn * sizeof(float));
    float *gcf = (float *)malloc((size_t)ng * 3 * sizeof(float));
    float *ghf = (float *)malloc((size_t)ng * 3 * sizeof(float));
    if (!com_f || !ropen2_f || !gcf || !ghf) {
        free(com_f); free(ropen2_f); free(gcf); free(ghf);
        return -1;
    }
    orc_cell_mac(src, theta, com_f, ropen2_f);
    orc_group_box_f32(dst, gcf, ghf);
    double eps2 = eps * eps;
    uint64_t npp_tot = 0, npc_tot = 0;
#pragma omp parallel reduction(+ : npp_tot, npc_tot)
    {
        orc_lists L;
        memset(&L, 0, sizeof(L));
#pragma omp for schedule(dynamic, 1)
        for (int64_t g = 0; g < ng; ++g) {
            float gc[3] = {gcf[g], gcf[(size_t)ng + g], gcf[2 * (size_t)ng + g]};
            float gh[3] = {ghf[g], ghf[(size_t)ng + g], ghf[2 * (size_t)ng + g]};
            orc_walk_group(src, com_f, ropen2_f, gc, gh, &L);
            uint32_t f = dst->gfirst[g], c = dst->gcount[g];
            if (g_npp) g_npp[g] = L.npp;
            if (g_npc) g_npc[g] = L.npc;
            npp_tot += (uint64_t)c * (uint64_t)L.npp;
            npc_tot += (uint64_t)c * (uint64_t)L.npc;
            for (uint32_t i = f; i < f + c; ++i) {
                double xi[3] = {dst->x[i], dst->x[(size_t)nd + i], dst->x[2 * (size_t)nd + i]};
                double phi = 0.0, a[3] = {0.0, 0.0, 0.0};
                for (int64_t k = 0; k < L.npc; ++k) {
                    uint32_t cc = L.pc[k];
                    double r[3], Qc[6];
                    for (int d = 0; d < 3; ++d) r[d] = src->com[(size_t)d * nn + cc] - xi[d];
                    for (int q = 0; q < 6; ++q) Qc[q] = src->Q[(size_t)q * nn + cc];
                    orc_eq12(r, src->M[cc], Qc, eps2, &phi, a);
                }
                for (int64_t k = 0; k < L.npp_leaves; ++k) {
                    uint32_t lf = L.pp[k];
                    for (uint32_t j = src->first[lf]; j < src->first[lf] + src->count[lf]; ++j) {
                        double r[3];
                        for (int d = 0; d < 3; ++d) r[d] = src->x[(size_t)d * ns + j] - xi[d];
                        orc_eq12(r, src->m[j], NULL, eps2, &phi, a);
                    }
                }
                pot[i] = G * phi;
                for (int d = 0; d < 3; ++d) acc[(size_t)d * nd + i] = G * a[d];
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

/* Face-on surface density (Sec. IV, Fig. 4: the disk and bulge seen from
 * above), by cloud-in-cell deposition: particle i in [first, first+count)
 * contributes m_i / (hx hy) times the bilinear weights of the four pixel
 * centres around it, pixel (px, py) having its centre at
 * (xmin + (px + 1/2) hx, ymin + (py + 1/2) hy); parts that fall outside the
 * nx x ny grid are dropped.  window = {xmin, xmax, ymin, ymax};
 * map[py * nx + px], zeroed here; particles in index order.              */
void orc_surface_density(int64_t n, const double *pos, const double *mass, int64_t first,
                         int64_t count, const double window[4], int nx, int ny, double *map) {
    const double hx = (window[1] - window[0]) / nx, hy = (window[3] - window[2]) / ny;
    for (int64_t k = 0; k < (int64_t)nx * ny; ++k) map[k] = 0.0;
    for (int64_t i = first; i < first + count && i < n; ++i) {
        double fx = (pos[i] - window[0]) / hx - 0.5;
        double fy = (pos[n + i] - window[2]) / hy - 0.5;
        if (!(fx > -1.0 && fx < (double)nx && fy > -1.0 && fy < (double)ny)) continue;
        double ix = floor(fx), iy = floor(fy);
        double tx = fx - ix, ty = fy - iy;
        double w = mass[i] / (hx * hy);
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                int px = (int)ix + dx, py = (int)iy + dy;
                if (px < 0 || px >= nx || py < 0 || py >= ny) continue;
                double wx = dx ? tx : 1.0 - tx, wy = dy ? ty : 1.0 - ty;
                map[(int64_t)py * nx + px] += w * wx * wy;
            }
    }
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ======================================================================== */
/* Adjoint (vector-Jacobian products) with the tree and lists frozen.       */
/* The paper has no adjoint; this is the exact derivative of the tree-force */
/* map of Eq. 1-2 for fixed node membership and fixed interaction lists:    */
/* the multipoles (M, com, Q) stay functions of the particles, so gradients */
/* reach particles both as p-p sources and through every cell they are in.  */
/* ======================================================================== */

/* Gradient of  lam . a + mu phi  (Eq. 1-2 for one source, without G) with
 * respect to r = source - target, the source mass m and its quadrupole Q
 * (Q may be NULL).  With s^2 = |r|^2 + eps^2 and u = 1/s:
 *   monopole:  a = m u^3 r,  phi = -m u;
 *   quadrupole: phi_Q = trQ u^3/2 - 3/2 rQr u^5,
 *               a_Q = (-3/2 trQ u^5 + 15/2 rQr u^7) r - 3 u^5 Qr.
 * Adds to g_r[3], *g_m and g_Q[6] (the gradient with respect to the
 * symmetric matrix Q, components xx, yy, zz, xy, xz, yz, not doubled).    */
static void orc_eq12_vjp(const double r[3], double m, const double *Q, double eps2,
                         const double lam[3], double mu, double g_r[3], double *g_m,
                         double *g_Q) {
    double s2 = ((r[0] * r[0] + r[1] * r[1]) + r[2] * r[2]) + eps2;
    double u = 1.0 / sqrt(s2);
    double u2 = u * u, u3 = u2 * u, u5 = u3 * u2, u7 = u5 * u2, u9 = u7 * u2;
    double lr = (lam[0] * r[0] + lam[1] * r[1]) + lam[2] * r[2];
    for (int d = 0; d < 3; ++d)
        g_r[d] += m * (u3 * lam[d] - 3.0 * u5 * lr * r[d]) + mu * m * u3 * r[d];
    *g_m += lr * u3 - mu * u;
    if (!Q) return;
    double trQ = (Q[0] + Q[1]) + Q[2];
    double Qr[3], Ql[3];
    Qr[0] = (Q[0] * r[0] + Q[3] * r[1]) + Q[4] * r[2];
    Qr[1] = (Q[3] * r[0] + Q[1] * r[1]) + Q[5] * r[2];
    Qr[2] = (Q[4] * r[0] + Q[5] * r[1]) + Q[2] * r[2];
    Ql[0] = (Q[0] * lam[0] + Q[3] * lam[1]) + Q[4] * lam[2];
    Ql[1] = (Q[3] * lam[0] + Q[1] * lam[1]) + Q[5] * lam[2];
    Ql[2] = (Q[4] * lam[0] + Q[5] * lam[1]) + Q[2] * lam[2];
    double rQr = (r[0] * Qr[0] + r[1] * Qr[1]) + r[2] * Qr[2];
    double lQr = (lam[0] * Qr[0] + lam[1] * Qr[1]) + lam[2] * Qr[2];
    double fQ = -1.5 * trQ * u5 + 7.5 * rQr * u7;
    double cr = lr * (7.5 * trQ * u7 - 52.5 * rQr * u9) + 15.0 * u7 * lQr;
    for (int d = 0; d < 3; ++d)
        g_r[d] += fQ * lam[d] + cr * r[d] + 15.0 * u7 * lr * Qr[d] - 3.0 * u5 * Ql[d] +
                  mu * (fQ * r[d] - 3.0 * u5 * Qr[d]);
    static const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int k = 0; k < 6; ++k) {
        int a = ia[k], b = ib[k];
        double diag = (a == b) ? (-1.5 * u5 * lr + 0.5 * mu * u3) : 0.0;
        g_Q[k] += diag + r[a] * r[b] * (7.5 * u7 * lr - 1.5 * mu * u5) -
                  1.5 * u5 * (lam[a] * r[b] + r[a] * lam[b]);
    }
}

/* exported for the tests: one source, times G */
void orc_eval_source_vjp(const double r[3], double m, const double *Q, double eps, double G,
                         const double lam[3], double mu, double g_r[3], double *g_m,
                         double g_Q[6]) {
    double gr[3] = {0, 0, 0}, gm = 0.0, gq[6] = {0, 0, 0, 0, 0, 0};
    orc_eq12_vjp(r, m, Q, eps * eps, lam, mu, gr, &gm, Q ? gq : NULL);
    for (int d = 0; d < 3; ++d) g_r[d] = G * gr[d];
    *g_m = G * gm;
    for (int k = 0; k < 6; ++k) g_Q[k] = G * gq[k];
}

/* Record every group's interaction lists for opening angle theta. */
int orc_tree_freeze_lists(orc_tree *t, float theta) {
    int64_t nn = t->nnodes, ng = t->ngroups;
    float *com_f = (float *)malloc((size_t)nn * 3 * sizeof(float));
    float *ropen2_f = (float *)malloc((size_t)nn * sizeof(float));
    float *gcf = (float *)malloc((size_t)ng * 3 * sizeof(float));
    float *ghf = (float *)malloc((size_t)ng * 3 * sizeof(float));
    free(t->pc_off); free(t->lf_off); free(t->pc_list); free(t->lf_list);
    t->pc_off = (int64_t *)calloc((size_t)ng + 1, sizeof(int64_t));
    t->lf_off = (int64_t *)calloc((size_t)ng + 1, sizeof(int64_t));
    t->pc_list = NULL;
    t->lf_list = NULL;
    if (!com_f || !ropen2_f || !gcf || !ghf || !t->pc_off || !t->lf_off) {
        free(com_f); free(ropen2_f); free(gcf); free(ghf);
        return -1;
    }
    orc_cell_mac(t, theta, com_f, ropen2_f);
    orc_group_box_f32(t, gcf, ghf);
    orc_lists L;
    memset(&L, 0, sizeof(L));
    int64_t cap_pc = 0, cap_lf = 0;
    for (int64_t g = 0; g < ng; ++g) {
        float gc[3] = {gcf[g], gcf[(size_t)ng + g], gcf[2 * (size_t)ng + g]};
        float gh[3] = {ghf[g], ghf[(size_t)ng + g], ghf[2 * (size_t)ng + g]};
        orc_walk_group(t, com_f, ropen2_f, gc, gh, &L);
        int64_t p0 = t->pc_off[g], l0 = t->lf_off[g];
        t->pc_off[g + 1] = p0 + L.npc;
        t->lf_off[g + 1] = l0 + L.npp_leaves;
        if (t->pc_off[g + 1] > cap_pc) {
            cap_pc = 2 * t->pc_off[g + 1] + 1024;
            t->pc_list = (uint32_t *)realloc(t->pc_list, (size_t)cap_pc * sizeof(uint32_t));
        }
        if (t->lf_off[g + 1] > cap_lf) {
            cap_lf = 2 * t->lf_off[g + 1] + 1024;
            t->lf_list = (uint32_t *)realloc(t->lf_list, (size_t)cap_lf * sizeof(uint32_t));
        }
        memcpy(t->pc_list + p0, L.pc, (size_t)L.npc * sizeof(uint32_t));
        memcpy(t->lf_list + l0, L.pp, (size_t)L.npp_leaves * sizeof(uint32_t));
    }
    free(L.pc); free(L.pp);
    free(com_f); free(ropen2_f); free(gcf); free(ghf);
    return 0;
}

/* Forces (sorted order) with the frozen lists at positions x and masses m
 * given in the tree's sorted order; the multipoles are recomputed from x, m
 * for the same node membership.                                            */
int orc_tree_frozen_forces(const orc_tree *t, double eps, double G, const double *x,
                           const double *m, double *acc, double *pot) {
    int64_t n = t->n, nn = t->nnodes, ng = t->ngroups;
    if (!t->pc_off) return -1;
    double *M = (double *)malloc((size_t)nn * sizeof(double));
    double *com = (double *)malloc((size_t)nn * 3 * sizeof(double));
    double *Q = (double *)malloc((size_t)nn * 6 * sizeof(double));
    if (!M || !com || !Q) { free(M); free(com); free(Q); return -1; }
    orc_upward(t, x, m, M, com, Q);
    double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t g = 0; g < ng; ++g) {
        for (uint32_t i = t->gfirst[g]; i < t->gfirst[g] + t->gcount[g]; ++i) {
            double xi[3] = {x[i], x[(size_t)n + i], x[2 * (size_t)n + i]};
            double phi = 0.0, a[3] = {0, 0, 0};
            for (int64_t k = t->pc_off[g]; k < t->pc_off[g + 1]; ++k) {
                uint32_t c = t->pc_list[k];
                double r[3], Qc[6];
                for (int d = 0; d < 3; ++d) r[d] = com[(size_t)d * nn + c] - xi[d];
                for (int q = 0; q < 6; ++q) Qc[q] = Q[(size_t)q * nn + c];
                orc_eq12(r, M[c], Qc, eps2, &phi, a);
            }
            for (int64_t k = t->lf_off[g]; k < t->lf_off[g + 1]; ++k) {
                uint32_t lf = t->lf_list[k];
                for (uint32_t j = t->first[lf]; j < t->first[lf] + t->count[lf]; ++j) {
                    if (j == i) continue;
                    double r[3];
                    for (int d = 0; d < 3; ++d) r[d] = x[(size_t)d * n + j] - xi[d];
                    orc_eq12(r, m[j], NULL, eps2, &phi, a);
                }
            }
            pot[i] = G * phi;
            for (int d = 0; d < 3; ++d) acc[(size_t)d * n + i] = G * a[d];
        }
    }
    free(M); free(com); free(Q);
    return 0;
}

/* VJP of the frozen-list forces: given lam (3n) and mu (n, may be NULL) in
 * sorted order, gx (3n) and gm (n) receive d(sum lam.a + mu phi)/dx, dm.
 * Target side, p-p source side and cell side are accumulated in one plain
 * serial loop; the cell adjoints (com, M, Q) are then pushed to every
 * particle of the cell:  x_k gets m_k/M gcom + 2 m_k gQ (x_k - com) and m_k
 * gets gM + gcom.(x_k - com)/M + (x_k - com)^T gQ (x_k - com).            */
int orc_tree_frozen_vjp(const orc_tree *t, double eps, double G, const double *x,
                        const double *m, const double *lam, const double *mu, double *gx,
                        double *gm) {
    int64_t n = t->n, nn = t->nnodes, ng = t->ngroups;
    if (!t->pc_off) return -1;
    double *M = (double *)malloc((size_t)nn * sizeof(double));
    double *com = (double *)malloc((size_t)nn * 3 * sizeof(double));
    double *Q = (double *)malloc((size_t)nn * 6 * sizeof(double));
    double *gcom = (double *)calloc((size_t)nn * 3, sizeof(double));
    double *gM = (double *)calloc((size_t)nn, sizeof(double));
    double *gQ = (double *)calloc((size_t)nn * 6, sizeof(double));
    if (!M || !com || !Q || !gcom || !gM || !gQ) {
        free(M); free(com); free(Q); free(gcom); free(gM); free(gQ);
        return -1;
    }
    orc_upward(t, x, m, M, com, Q);
    memset(gx, 0, (size_t)n * 3 * sizeof(double));
    memset(gm, 0, (size_t)n * sizeof(double));
    double eps2 = eps * eps;
    for (int64_t g = 0; g < ng; ++g) {
        for (uint32_t i = t->gfirst[g]; i < t->gfirst[g] + t->gcount[g]; ++i) {
            double xi[3] = {x[i], x[(size_t)n + i], x[2 * (size_t)n + i]};
            double li[3] = {lam[i], lam[(size_t)n + i], lam[2 * (size_t)n + i]};
            double mi = mu ? mu[i] : 0.0;
            for (int64_t k = t->pc_off[g]; k < t->pc_off[g + 1]; ++k) {
                uint32_t c = t->pc_list[k];
                double r[3], Qc[6], gr[3] = {0, 0, 0}, gmc = 0.0, gq[6] = {0, 0, 0, 0, 0, 0};
                for (int d = 0; d < 3; ++d) r[d] = com[(size_t)d * nn + c] - xi[d];
                for (int q = 0; q < 6; ++q) Qc[q] = Q[(size_t)q * nn + c];
                orc_eq12_vjp(r, M[c], Qc, eps2, li, mi, gr, &gmc, gq);
                for (int d = 0; d < 3; ++d) {
                    gx[(size_t)d * n + i] -= G * gr[d];
                    gcom[(size_t)d * nn + c] += G * gr[d];
                }
                gM[c] += G * gmc;
                for (int q = 0; q < 6; ++q) gQ[(size_t)q * nn + c] += G * gq[q];
            }
            for (int64_t k = t->lf_off[g]; k < t->lf_off[g + 1]; ++k) {
                uint32_t lf = t->lf_list[k];
                for (uint32_t j = t->first[lf]; j < t->first[lf] + t->count[lf]; ++j) {
                    if (j == i) continue;
                    double r[3], gr[3] = {0, 0, 0}, gmj = 0.0;
                    for (int d = 0; d < 3; ++d) r[d] = x[(size_t)d * n + j] - xi[d];
                    orc_eq12_vjp(r, m[j], NULL, eps2, li, mi, gr, &gmj, NULL);
                    for (int d = 0; d < 3; ++d) {
                        gx[(size_t)d * n + i] -= G * gr[d];
                        gx[(size_t)d * n + j] += G * gr[d];
                    }
                    gm[j] += G * gmj;
                }
            }
        }
    }
    /* cell adjoints to the particles of each cell */
    for (int64_t c = 0; c < nn; ++c) {
        double q[3][3] = {{gQ[c], gQ[3 * (size_t)nn + c], gQ[4 * (size_t)nn + c]},
                          {gQ[3 * (size_t)nn + c], gQ[(size_t)nn + c], gQ[5 * (size_t)nn + c]},
                          {gQ[4 * (size_t)nn + c], gQ[5 * (size_t)nn + c], gQ[2 * (size_t)nn + c]}};
        double gc[3] = {gcom[c], gcom[(size_t)nn + c], gcom[2 * (size_t)nn + c]};
        for (uint32_t k = t->first[c]; k < t->first[c] + t->count[c]; ++k) {
            double d[3], qd[3];
            for (int e = 0; e < 3; ++e) d[e] = x[(size_t)e * n + k] - com[(size_t)e * nn + c];
            for (int e = 0; e < 3; ++e) qd[e] = (q[e][0] * d[0] + q[e][1] * d[1]) + q[e][2] * d[2];
            for (int e = 0; e < 3; ++e)
                gx[(size_t)e * n + k] += m[k] / M[c] * gc[e] + 2.0 * m[k] * qd[e];
            gm[k] += gM[c] + ((gc[0] * d[0] + gc[1] * d[1]) + gc[2] * d[2]) / M[c] +
                     ((d[0] * qd[0] + d[1] * qd[1]) + d[2] * qd[2]);
        }
    }
    free(M); free(com); free(Q); free(gcom); free(gM); free(gQ);
    return 0;
}

/* O1 adjoint: VJP of direct summation, all pairs j != i (caller order). */
void orc_direct_vjp(int64_t n, const double *pos, const double *mass, double eps, double G,
                    const double *lam, const double *mu, double *gpos, double *gmass) {
    double eps2 = eps * eps;
    memset(gpos, 0, (size_t)n * 3 * sizeof(double));
    memset(gmass, 0, (size_t)n * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        double li[3] = {lam[i], lam[n + i], lam[2 * n + i]};
        double mi = mu ? mu[i] : 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r[3] = {pos[j] - pos[i], pos[n + j] - pos[n + i], pos[2 * n + j] - pos[2 * n + i]};
            double gr[3] = {0, 0, 0}, gmj = 0.0;
            orc_eq12_vjp(r, mass[j], NULL, eps2, li, mi, gr, &gmj, NULL);
            for (int d = 0; d < 3; ++d) {
                gpos[d * n + i] -= G * gr[d];
                gpos[d * n + j] += G * gr[d];
            }
            gmass[j] += G * gmj;
        }
    }
}

/* ---- K leap-frog steps with frozen per-step trees (adjoint of KDK) ---- */
typedef struct {
    int64_t n;
    int nsteps;
    double dt, eps, G;
    orc_tree **trees; /* tree k built at the nominal x_k, lists frozen */
    double *xs;       /* nominal positions x_0 .. x_K, caller order [K+1][3n] */
} orc_kdk_plan;

void orc_kdk_plan_free(orc_kdk_plan *p) {
    if (!p) return;
    if (p->trees)
        for (int k = 0; k <= p->nsteps; ++k) orc_tree_free(p->trees[k]);
    free(p->trees);
    free(p->xs);
    free(p);
}

/* frozen-list forces at caller-order positions x with tree t's structure */
static int orc_frozen_caller(const orc_tree *t, double eps, double G, const double *x,
                             const double *m, double *acc) {
    int64_t n = t->n;
    double *xs = (double *)malloc((size_t)n * 3 * sizeof(double));
    double *ms = (double *)malloc((size_t)n * sizeof(double));
    double *as = (double *)malloc((size_t)n * 3 * sizeof(double));
    double *ps = (double *)malloc((size_t)n * sizeof(double));
    if (!xs || !ms || !as || !ps) { free(xs); free(ms); free(as); free(ps); return -1; }
    for (int64_t s = 0; s < n; ++s) {
        uint32_t j = t->perm[s];
        ms[s] = m[j];
        for (int d = 0; d < 3; ++d) xs[(size_t)d * n + s] = x[(size_t)d * n + j];
    }
    int rc = orc_tree_frozen_forces(t, eps, G, xs, ms, as, ps);
    for (int64_t s = 0; s < n; ++s)
        for (int d = 0; d < 3; ++d) acc[(size_t)d * n + t->perm[s]] = as[(size_t)d * n + s];
    free(xs); free(ms); free(as); free(ps);
    return rc;
}

/* frozen-list VJP at caller-order x with cotangent lam (caller order, mu = 0);
 * adds into gx (3n) and gm (n), caller order */
static int orc_frozen_vjp_caller(const orc_tree *t, double eps, double G, const double *x,
                                 const double *m, const double *lam, double *gx, double *gm) {
    int64_t n = t->n;
    double *xs = (double *)malloc((size_t)n * 3 * sizeof(double));
    double *ms = (double *)malloc((size_t)n * sizeof(double));
    double *ls = (double *)malloc((size_t)n * 3 * sizeof(double));
    double *gxs = (double *)malloc((size_t)n * 3 * sizeof(double));
    double *gms = (double *)malloc((size_t)n * sizeof(double));
    if (!xs || !ms || !ls || !gxs || !gms) {
        free(xs); free(ms); free(ls); free(gxs); free(gms);
        return -1;
    }
    for (int64_t s = 0; s < n; ++s) {
        uint32_t j = t->perm[s];
        ms[s] = m[j];
        for (int d = 0; d < 3; ++d) {
            xs[(size_t)d * n + s] = x[(size_t)d * n + j];
            ls[(size_t)d * n + s] = lam[(size_t)d * n + j];
        }
    }
    int rc = orc_tree_frozen_vjp(t, eps, G, xs, ms, ls, NULL, gxs, gms);
    for (int64_t s = 0; s < n; ++s) {
        uint32_t j = t->perm[s];
        gm[j] += gms[s];
        for (int d = 0; d < 3; ++d) gx[(size_t)d * n + j] += gxs[(size_t)d * n + s];
    }
    free(xs); free(ms); free(ls); free(gxs); free(gms);
    return rc;
}

/* Nominal trajectory: K kick-drift-kick steps from (pos0, vel0), the tree
 * and lists of step k built and frozen at the nominal x_k.                 */
orc_kdk_plan *orc_kdk_plan_build(int64_t n, const double *pos0, const double *vel0,
                                 const double *mass, int nsteps, double dt, float theta,
                                 double eps, double G, int nleaf, int ncrit) {
    orc_kdk_plan *p = (orc_kdk_plan *)calloc(1, sizeof(orc_kdk_plan));
    if (!p) return NULL;
    p->n = n;
    p->nsteps = nsteps;
    p->dt = dt;
    p->eps = eps;
    p->G = G;
    p->trees = (orc_tree **)calloc((size_t)nsteps + 1, sizeof(orc_tree *));
    p->xs = (double *)malloc((size_t)(nsteps + 1) * 3 * n * sizeof(double));
    double *v = (double *)malloc((size_t)n * 3 * sizeof(double));
    double *a = (double *)malloc((size_t)n * 3 * sizeof(double));
    if (!p->trees || !p->xs || !v || !a) { free(v); free(a); orc_kdk_plan_free(p); return NULL; }
    memcpy(p->xs, pos0, (size_t)n * 3 * sizeof(double));
    memcpy(v, vel0, (size_t)n * 3 * sizeof(double));
    double h = 0.5 * dt;
    for (int k = 0; k <= nsteps; ++k) {
        double *xk = p->xs + (size_t)k * 3 * n;
        if (k > 0) {
            double *xp = p->xs + (size_t)(k - 1) * 3 * n;
            for (int64_t q = 0; q < 3 * n; ++q) v[q] = v[q] + a[q] * h;
            for (int64_t q = 0; q < 3 * n; ++q) xk[q] = xp[q] + v[q] * dt;
        }
        p->trees[k] = orc_tree_build(n, xk, mass, nleaf, ncrit);
        if (!p->trees[k] || orc_tree_freeze_lists(p->trees[k], theta) ||
            orc_frozen_caller(p->trees[k], eps, G, xk, mass, a)) {
            free(v); free(a); orc_kdk_plan_free(p);
            return NULL;
        }
        if (k > 0)
            for (int64_t q = 0; q < 3 * n; ++q) v[q] = v[q] + a[q] * h;
    }
    free(v); free(a);
    return p;
}

/* Run the K steps from (pos0, vel0) with each step's frozen tree. */
int orc_kdk_plan_run(const orc_kdk_plan *p, const double *pos0, const double *vel0,
                     const double *mass, double *pos, double *vel) {
    int64_t n = p->n;
    double *a = (double *)malloc((size_t)n * 3 * sizeof(double));
    if (!a) return -1;
    memcpy(pos, pos0, (size_t)n * 3 * sizeof(double));
    memcpy(vel, vel0, (size_t)n * 3 * sizeof(double));
    double h = 0.5 * p->dt;
    int rc = orc_frozen_caller(p->trees[0], p->eps, p->G, pos, mass, a);
    for (int k = 1; k <= p->nsteps && !rc; ++k) {
        for (int64_t q = 0; q < 3 * n; ++q) vel[q] = vel[q] + a[q] * h;
        for (int64_t q = 0; q < 3 * n; ++q) pos[q] = pos[q] + vel[q] * p->dt;
        rc = orc_frozen_caller(p->trees[k], p->eps, p->G, pos, mass, a);
        for (int64_t q = 0; q < 3 * n; ++q) vel[q] = vel[q] + a[q] * h;
    }
    free(a);
    return rc;
}

/* Reverse of the K steps at the nominal trajectory.  In: xbar, vbar (the
 * cotangents of x_K, v_K) and mbar (direct mass cotangent, may be zero);
 * out: the same arrays hold the cotangents of x_0, v_0, m.
 *   a_K enters only the last half kick: abar_K = h vbar.
 *   for k = K-1 .. 0:  vbar += dt xbar  (drift),
 *                      abar_k = c vbar with c = dt for k > 0 (both half
 *                      kicks use a_k) and c = h for k = 0,
 *                      (xbar, mbar) += VJP_k(abar_k).                      */
int orc_kdk_plan_vjp(const orc_kdk_plan *p, const double *mass, double *xbar, double *vbar,
                     double *mbar) {
    int64_t n = p->n;
    double h = 0.5 * p->dt;
    double *ab = (double *)malloc((size_t)n * 3 * sizeof(double));
    if (!ab) return -1;
    int K = p->nsteps, rc = 0;
    if (K == 0) { free(ab); return 0; }
    for (int64_t q = 0; q < 3 * n; ++q) ab[q] = h * vbar[q];
    rc = orc_frozen_vjp_caller(p->trees[K], p->eps, p->G, p->xs + (size_t)K * 3 * n, mass, ab,
                               xbar, mbar);
    for (int k = K - 1; k >= 0 && !rc; --k) {
        for (int64_t q = 0; q < 3 * n; ++q) vbar[q] = vbar[q] + p->dt * xbar[q];
        double c = (k > 0) ? p->dt : h;
        for (int64_t q = 0; q < 3 * n; ++q) ab[q] = c * vbar[q];
        rc = orc_frozen_vjp_caller(p->trees[k], p->eps, p->G, p->xs + (size_t)k * 3 * n, mass,
                                   ab, xbar, mbar);
    }
    free(ab);
    return rc;
}
