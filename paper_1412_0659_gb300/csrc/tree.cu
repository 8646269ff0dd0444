// tree.cu -- octree construction from the sorted keys, walk groups, the
// FP64 upward pass and the FP32 record packs (Sec. III.A "tree-construction"
// and "computation of multipole moments"; Sec. I.A leaf size 16; Sec. VI.A
// mass, centre of mass and 3x3 symmetric quadrupole per cell).
//
// The octree is built level by level: a node of level l holding more than
// 16 particles is cut into the runs of equal key digit l+1 (8 binary
// searches on its sorted key range); an exclusive scan over the level's
// child counts numbers the children breadth-first, so the numbering is a
// pure function of the sorted keys.  The host reads one count per level to
// size the next launch.
//
// The upward pass computes every leaf in one launch (a leaf needs only its
// particles), then visits the levels bottom-up, where internal nodes
// combine their children by the parallel-axis rule; every FP64 operation is
// an explicit round-to-nearest intrinsic in a fixed order.
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace bgb {


namespace {

__global__ void k_root(uint32_t *first, uint32_t *count, uint32_t *level, uint32_t *parent,
                       uint32_t n) {
    first[0] = 0;
    count[0] = n;
    level[0] = 0;
    parent[0] = 0;
}

// Child boundaries of a node at level l: b[d] = first slot of [f, f + c)
// whose digit l+1 is >= d.  The seven lower bounds share the range, so they
// run in lockstep (branch-free halving; the trip count depends on c only):
// log2(c) rounds of seven independent loads instead of seven chained
// searches.
__device__ inline void child_bounds(const uint64_t *__restrict__ key, uint32_t f, uint32_t c,
                                    int l, uint32_t b[9]) {
    const int shift = 3 * (MAX_LEVEL - 1 - l);
    const uint64_t base = key[f] & ~((8ull << shift) - 1ull);
    uint32_t lo[7];
#pragma unroll
    for (int d = 0; d < 7; ++d) lo[d] = f;
    uint32_t len = c;
    while (len > 1) {
        const uint32_t half = len >> 1;
#pragma unroll
        for (int d = 0; d < 7; ++d)
            lo[d] = key[lo[d] + half] < (base | ((uint64_t)(d + 1) << shift)) ? lo[d] + half : lo[d];
        len -= half;
    }
    b[0] = f;
    b[8] = f + c;
#pragma unroll
    for (int d = 0; d < 7; ++d)
        b[d + 1] = lo[d] + (key[lo[d]] < (base | ((uint64_t)(d + 1) << shift)) ? 1u : 0u);
}

__global__ void __launch_bounds__(256) k_split_count(const uint64_t *__restrict__ key,
                                                     const uint32_t *__restrict__ first,
                                                     const uint32_t *__restrict__ count,
                                                     uint32_t *__restrict__ nchild,
                                                     uint32_t *__restrict__ scan_in, int64_t s,
                                                     int64_t m, int l) {
    int64_t t = blockIdx.x * 256ll + threadIdx.x;
    if (t >= m) return;
    int64_t i = s + t;
    uint32_t f = first[i], c = count[i], nc = 0;
    if (c > (uint32_t)NLEAF && l < MAX_LEVEL) {
        uint32_t b[9];
        child_bounds(key, f, c, l, b);
#pragma unroll
        for (int d = 0; d < 8; ++d) nc += b[d + 1] > b[d];
    }
    nchild[i] = nc;
    scan_in[t] = nc;
}

__global__ void __launch_bounds__(256) k_split_write(
    const uint64_t *__restrict__ key, uint32_t *__restrict__ first, uint32_t *__restrict__ count,
    uint32_t *__restrict__ child, const uint32_t *__restrict__ nchild, uint32_t *__restrict__ level,
    uint32_t *__restrict__ parent, uint2 *__restrict__ topo, const uint32_t *__restrict__ off,
    int64_t s, int64_t m, int64_t e, int l) {
    int64_t t = blockIdx.x * 256ll + threadIdx.x;
    if (t >= m) return;
    int64_t i = s + t;
    uint32_t f = first[i], c = count[i], nc = nchild[i];
    if (nc == 0) {
        child[i] = 0;
        topo[i] = make_uint2(f, c | LEAF_FLAG);
        return;
    }
    uint32_t ch = (uint32_t)(e + off[t]);
    child[i] = ch;
    topo[i] = make_uint2(ch, nc);
    uint32_t b[9];
    child_bounds(key, f, c, l, b);
    uint32_t k = ch;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        if (b[d + 1] > b[d]) {
            first[k] = b[d];
            count[k] = b[d + 1] - b[d];
            level[k] = (uint32_t)(l + 1);
            parent[k] = (uint32_t)i;
            ++k;
        }
    }
}

// Leaves of the deepest level never reach k_split_write: mark them here.
__global__ void k_mark_leaves(const uint32_t *__restrict__ first, const uint32_t *__restrict__ count,
                              uint32_t *__restrict__ child, uint32_t *__restrict__ nchild,
                              uint2 *__restrict__ topo, int64_t s, int64_t m) {
    int64_t t = blockIdx.x * 256ll + threadIdx.x;
    if (t >= m) return;
    int64_t i = s + t;
    child[i] = 0;
    nchild[i] = 0;
    topo[i] = make_uint2(first[i], count[i] | LEAF_FLAG);
}

// ---- upward pass (FP64) ----
// Q order: xx, yy, zz, xy, xz, yz.  LEAVES: one launch over all nodes that
// computes the leaves (they depend on nothing); otherwise one launch per
// level, bottom-up, that combines the children of the level's internal
// nodes.
template <bool LEAVES>
__global__ void __launch_bounds__(128) k_multipoles(
    const double *__restrict__ pos, const double *__restrict__ mass, int64_t n,
    const uint32_t *__restrict__ first, const uint32_t *__restrict__ count,
    const uint32_t *__restrict__ child, const uint32_t *__restrict__ nchild, double *__restrict__ M,
    double *__restrict__ com, double *__restrict__ Q, int64_t nn, int64_t s, int64_t m) {
    int64_t t = blockIdx.x * 128ll + threadIdx.x;
    if (t >= m) return;
    int64_t i = s + t;
    if ((nchild[i] == 0) != LEAVES) return;
    double Ms = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    double q0 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0, q4 = 0.0, q5 = 0.0;
    double cx, cy, cz;
    uint32_t nc = nchild[i];
    if (nc == 0) {
        uint32_t f = first[i], c = count[i];
        for (uint32_t j = f; j < f + c; ++j) {
            double mj = mass[j];
            Ms = __dadd_rn(Ms, mj);
            sx = __dadd_rn(sx, __dmul_rn(mj, pos[j]));
            sy = __dadd_rn(sy, __dmul_rn(mj, pos[n + j]));
            sz = __dadd_rn(sz, __dmul_rn(mj, pos[2 * n + j]));
        }
        cx = __ddiv_rn(sx, Ms);
        cy = __ddiv_rn(sy, Ms);
        cz = __ddiv_rn(sz, Ms);
        for (uint32_t j = f; j < f + c; ++j) {
            double mj = mass[j];
            double dx = __dsub_rn(pos[j], cx), dy = __dsub_rn(pos[n + j], cy),
                   dz = __dsub_rn(pos[2 * n + j], cz);
            double mx = __dmul_rn(mj, dx), my = __dmul_rn(mj, dy);
            q0 = __dadd_rn(q0, __dmul_rn(mx, dx));
            q1 = __dadd_rn(q1, __dmul_rn(my, dy));
            q2 = __dadd_rn(q2, __dmul_rn(__dmul_rn(mj, dz), dz));
            q3 = __dadd_rn(q3, __dmul_rn(mx, dy));
            q4 = __dadd_rn(q4, __dmul_rn(mx, dz));
            q5 = __dadd_rn(q5, __dmul_rn(my, dz));
        }
    } else {
        uint32_t c0 = child[i];
        for (uint32_t k = c0; k < c0 + nc; ++k) {
            double Mk = M[k];
            Ms = __dadd_rn(Ms, Mk);
            sx = __dadd_rn(sx, __dmul_rn(Mk, com[k]));
            sy = __dadd_rn(sy, __dmul_rn(Mk, com[nn + k]));
            sz = __dadd_rn(sz, __dmul_rn(Mk, com[2 * nn + k]));
        }
        cx = __ddiv_rn(sx, Ms);
        cy = __ddiv_rn(sy, Ms);
        cz = __ddiv_rn(sz, Ms);
        for (uint32_t k = c0; k < c0 + nc; ++k) {
            double Mk = M[k];
            double dx = __dsub_rn(com[k], cx), dy = __dsub_rn(com[nn + k], cy),
                   dz = __dsub_rn(com[2 * nn + k], cz);
            double mx = __dmul_rn(Mk, dx), my = __dmul_rn(Mk, dy);
            q0 = __dadd_rn(q0, __dadd_rn(Q[k], __dmul_rn(mx, dx)));
            q1 = __dadd_rn(q1, __dadd_rn(Q[nn + k], __dmul_rn(my, dy)));
            q2 = __dadd_rn(q2, __dadd_rn(Q[2 * nn + k], __dmul_rn(__dmul_rn(Mk, dz), dz)));
            q3 = __dadd_rn(q3, __dadd_rn(Q[3 * nn + k], __dmul_rn(mx, dy)));
            q4 = __dadd_rn(q4, __dadd_rn(Q[4 * nn + k], __dmul_rn(mx, dz)));
            q5 = __dadd_rn(q5, __dadd_rn(Q[5 * nn + k], __dmul_rn(my, dz)));
        }
    }
    M[i] = Ms;
    com[i] = cx;
    com[nn + i] = cy;
    com[2 * nn + i] = cz;
    Q[i] = q0;
    Q[nn + i] = q1;
    Q[2 * nn + i] = q2;
    Q[3 * nn + i] = q3;
    Q[4 * nn + i] = q4;
    Q[5 * nn + i] = q5;
}

// ---- groups: runs of consecutive sibling cells of at most NCRIT particles
// in all.  Each group start is flagged in a per-particle array, a scan
// numbers them in particle order.
// Group starts (flags at the first particle of each group).  A thread per
// node; only nodes with more than NCRIT particles act.  Their children of at
// most NCRIT particles are taken in key order and gathered greedily into runs
// of at most NCRIT particles, a child with more than NCRIT ending the run
// (its own children are grouped by its thread): each run is one group.  The
// root is the one group when it holds at most NCRIT; a max-depth leaf with
// more than NCRIT is cut into runs of NCRIT.
__global__ void __launch_bounds__(256) k_group_flags(const uint32_t *__restrict__ first,
                                                           const uint32_t *__restrict__ count,
                                                           const uint32_t *__restrict__ nchild,
                                                           const uint32_t *__restrict__ child,
                                                           uint32_t *__restrict__ flag, int64_t nn) {
    int64_t i = blockIdx.x * 256ll + threadIdx.x;
    if (i >= nn) return;
    const uint32_t c = count[i];
    if (c <= (uint32_t)NCRIT) {
        if (i == 0) flag[first[0]] = 1u;
        return;
    }
    if (nchild[i] == 0) {
        for (uint32_t s = 0; s < c; s += NCRIT) flag[first[i] + s] = 1u;
        return;
    }
    uint32_t run = 0;
    bool open = false;
    for (uint32_t k = 0; k < nchild[i]; ++k) {
        const uint32_t j = child[i] + k, cj = count[j];
        if (cj > (uint32_t)NCRIT) {
            open = false;
            continue;
        }
        if (!open || run + cj > (uint32_t)NCRIT) {
            flag[first[j]] = 1u;
            run = cj;
            open = true;
        } else {
            run += cj;
        }
    }
}

__global__ void __launch_bounds__(256) k_group_write(const uint32_t *__restrict__ flag,
                                                     const uint32_t *__restrict__ gid, int64_t n,
                                                     uint32_t *__restrict__ gfirst) {
    int64_t i = blockIdx.x * 256ll + threadIdx.x;
    if (i >= n) return;
    if (flag[i]) gfirst[gid[i]] = (uint32_t)i;
}

// Order-preserving integer image of a double: for finite values (the input
// check rejects the others) a < b exactly when key(a) < key(b), with -0 just
// below +0.  Minima and maxima taken on the keys are therefore exact, and
// run on the integer pipes instead of the FP64 one.
__device__ __forceinline__ long long order_key(double v) {
    const long long b = __double_as_longlong(v);
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
__device__ __forceinline__ double from_order_key(long long k) {
    return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffll));
}

// Per group: the FP64 box of the members, its FP32 centre (nearest), the
// centre's FP32 remainder, and the half-size rounded up to FP32.  A warp
// takes 32 consecutive groups: for each, all lanes load its members and
// reduce their minima and maxima; lane k keeps those of group k, and the
// FP64 epilogue then runs once per lane for the 32 groups at a time.
__global__ void __launch_bounds__(256) k_group_box(const double *__restrict__ pos, int64_t n,
                                                   const uint32_t *__restrict__ gfirst,
                                                   uint32_t *__restrict__ gcount, int64_t ng,
                                                   double *__restrict__ gcentre,
                                                   float4 *__restrict__ gbox,
                                                   float4 *__restrict__ ghalf,
                                                   float4 *__restrict__ glo) {
    const int64_t g0 = ((blockIdx.x * 256ll + threadIdx.x) >> 5) * 32;
    const int lane = threadIdx.x & 31;
    if (g0 >= ng) return;
    long long myn[3] = {0, 0, 0}, myx[3] = {0, 0, 0};
    const int kend = (int)min((int64_t)32, ng - g0);
    for (int k = 0; k < kend; ++k) {
        const int64_t g = g0 + k;
        const uint32_t f = gfirst[g];
        const uint32_t e = (g + 1 < ng) ? gfirst[g + 1] : (uint32_t)n;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            long long kn = 0x7fffffffffffffffll, kx = -0x7fffffffffffffffll - 1;
            for (uint32_t j = f + lane; j < e; j += 32) {
                const long long key = order_key(pos[d * n + j]);
                kn = min(kn, key);
                kx = max(kx, key);
            }
            for (int o = 16; o > 0; o >>= 1) {
                kn = min(kn, __shfl_xor_sync(0xffffffffu, kn, o));
                kx = max(kx, __shfl_xor_sync(0xffffffffu, kx, o));
            }
            if (lane == k) {
                myn[d] = kn;
                myx[d] = kx;
            }
        }
    }
    const int64_t g = g0 + lane;
    if (lane >= kend) return;
    const uint32_t f = gfirst[g];
    gcount[g] = ((g + 1 < ng) ? gfirst[g + 1] : (uint32_t)n) - f;
    float cf[3], hf[3], cl[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double mn = from_order_key(myn[d]), mx = from_order_key(myx[d]);
        const double ctr = __dmul_rn(__dadd_rn(mn, mx), 0.5);
        const double half = __dmul_rn(__dsub_rn(mx, mn), 0.5);
        cf[d] = __double2float_rn(ctr);
        cl[d] = __double2float_rn(__dsub_rn(ctr, (double)cf[d]));
        hf[d] = __double2float_ru(half);
        gcentre[d * ng + g] = ctr;
    }
    gbox[g] = make_float4(cf[0], cf[1], cf[2], 0.0f);
    ghalf[g] = make_float4(hf[0], hf[1], hf[2], 0.0f);
    glo[g] = make_float4(cl[0], cl[1], cl[2], 0.0f);
}

// Particle records for the walk: FP32 head and remainder of each coordinate.
__global__ void __launch_bounds__(256) k_body_pack(const double *__restrict__ pos,
                                                   const double *__restrict__ mass, int64_t n,
                                                   float4 *__restrict__ hi, float4 *__restrict__ lo) {
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        double x = pos[i], y = pos[n + i], z = pos[2 * n + i];
        float xh = __double2float_rn(x), yh = __double2float_rn(y), zh = __double2float_rn(z);
        hi[i] = make_float4(xh, yh, zh, __double2float_rn(mass[i]));
        lo[i] = make_float4(__double2float_rn(__dsub_rn(x, (double)xh)),
                            __double2float_rn(__dsub_rn(y, (double)yh)),
                            __double2float_rn(__dsub_rn(z, (double)zh)), 0.0f);
    }
}

__device__ inline uint32_t quantise_q(double x, double lo, double scale) {
    double f = floor(__dmul_rn(__dsub_rn(x, lo), scale));
    if (!(f >= 0.0)) return 0u;
    if (f > (double)((1u << KEY_BITS) - 1u)) return (1u << KEY_BITS) - 1u;
    return (uint32_t)f;
}

// Cell records for a given theta.  The opening radius (Sec. I.A's opening
// angle) is r_open = l/theta + |com - centre|, with l = L/2^level the cube
// side and centre the middle of the level-l cube holding the node (taken
// from its first particle's quantised coordinates); r_open^2 is rounded to
// FP32 once.  com is split into an FP32 head (used by the opening test) and
// remainder.  The force kernel reads Q' = -3 Q and the constants -trQ/2 and
// -3/2 trQ (FP64, rounded to FP32 once), which fold Eq. 1-2 into fewer FP32
// operations.
__global__ void __launch_bounds__(256) k_cell_pack(
    const double *__restrict__ pos, int64_t n, const uint32_t *__restrict__ first,
    const uint32_t *__restrict__ level, const double *__restrict__ M, const double *__restrict__ com,
    const double *__restrict__ Q, int64_t nn, const DevScalars *__restrict__ sc, double theta,
    float4 *__restrict__ mac, float4 *__restrict__ ca, float4 *__restrict__ cb,
    float4 *__restrict__ cc) {
    int64_t i = blockIdx.x * 256ll + threadIdx.x;
    if (i >= nn) return;
    const int l = (int)level[i];
    const double side = ldexp(sc->L, -l);
    const uint32_t f = first[i];
    double s2 = 0.0;
    float ch[3], cl[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        uint32_t k = quantise_q(pos[d * n + f], sc->lo[d], sc->scale) >> (KEY_BITS - l);
        double ctr = __dadd_rn(sc->lo[d], __dmul_rn((double)k + 0.5, side));
        double cd = com[d * nn + i];
        double dd = __dsub_rn(cd, ctr);
        double sq = __dmul_rn(dd, dd);
        s2 = (d == 0) ? sq : __dadd_rn(s2, sq);
        ch[d] = __double2float_rn(cd);
        cl[d] = __double2float_rn(__dsub_rn(cd, (double)ch[d]));
    }
    double r_open = __dadd_rn(__ddiv_rn(side, theta), __dsqrt_rn(s2));
    float r2 = __double2float_rn(__dmul_rn(r_open, r_open));
    mac[i] = make_float4(ch[0], ch[1], ch[2], r2);
    ca[i] = make_float4(cl[0], cl[1], cl[2], __double2float_rn(M[i]));
    double qxx = Q[i], qyy = Q[nn + i], qzz = Q[2 * nn + i];
    double tr = __dadd_rn(__dadd_rn(qxx, qyy), qzz);
    cb[i] = make_float4(__double2float_rn(-3.0 * qxx), __double2float_rn(-3.0 * qyy),
                        __double2float_rn(-3.0 * qzz), __double2float_rn(-3.0 * Q[3 * nn + i]));
    cc[i] = make_float4(__double2float_rn(-3.0 * Q[4 * nn + i]),
                        __double2float_rn(-3.0 * Q[5 * nn + i]), __double2float_rn(-0.5 * tr),
                        __double2float_rn(-1.5 * tr));
}

}  // namespace

// Grow the node arrays to hold at least need nodes, keeping [0, keep).
static int grow_nodes(bonsai_ctx *c, int64_t need, int64_t keep) {
    if ((size_t)need <= c->nd_first.cap) return BONSAI_OK;
    size_t cap = std::max((size_t)need, c->nd_first.cap + c->nd_first.cap / 2);
    DBuf<uint32_t> *u32s[] = {&c->nd_first, &c->nd_count, &c->nd_child, &c->nd_nchild,
                              &c->nd_level, &c->nd_parent};
    for (DBuf<uint32_t> *b : u32s) {
        uint32_t *p = nullptr;
        if (cudaMalloc(&p, cap * sizeof(uint32_t)) != cudaSuccess) return BONSAI_ENOMEM;
        if (keep > 0 && b->p)
            cudaMemcpyAsync(p, b->p, keep * sizeof(uint32_t), cudaMemcpyDeviceToDevice, c->stream);
        BGB_WAIT(c->stream);
        cudaFree(b->p);
        b->p = p;
        b->cap = cap;
    }
    {
        uint2 *p = nullptr;
        if (cudaMalloc(&p, cap * sizeof(uint2)) != cudaSuccess) return BONSAI_ENOMEM;
        if (keep > 0 && c->cell_topo.p)
            cudaMemcpyAsync(p, c->cell_topo.p, keep * sizeof(uint2), cudaMemcpyDeviceToDevice,
                            c->stream);
        BGB_WAIT(c->stream);
        cudaFree(c->cell_topo.p);
        c->cell_topo.p = p;
        c->cell_topo.cap = cap;
    }
    if (ensure(c->nd_scan, cap) || ensure(c->scan_tmp, scan_tmp_elems((int64_t)cap)))
        return BONSAI_ENOMEM;
    return BONSAI_OK;
}

int build_octree(bonsai_ctx *c) {
    const int64_t n = c->n;
    int rc = grow_nodes(c, std::max<int64_t>(1024, n / 2 + 64), 0);
    if (rc) return rc;
    k_root<<<1, 1, 0, c->stream>>>(c->nd_first.p, c->nd_count.p, c->nd_level.p, c->nd_parent.p,
                                   (uint32_t)n);
    c->launches += 1;
    c->level_start[0] = 0;
    c->level_start[1] = 1;
    int depth = 0;
    for (int l = 0; l <= MAX_LEVEL; ++l) {
        const int64_t s = c->level_start[l], e = c->level_start[l + 1], m = e - s;
        if (m == 0) {
            for (int k = l + 1; k <= MAX_LEVEL + 1; ++k) c->level_start[k] = e;
            break;
        }
        depth = l;
        if (l == MAX_LEVEL) {
            k_mark_leaves<<<grid_for(m, 256), 256, 0, c->stream>>>(
                c->nd_first.p, c->nd_count.p, c->nd_child.p, c->nd_nchild.p, c->cell_topo.p, s, m);
            c->launches += 1;
            c->level_start[l + 2 > MAX_LEVEL + 1 ? MAX_LEVEL + 1 : l + 2] = e;
            break;
        }
        k_split_count<<<grid_for(m, 256), 256, 0, c->stream>>>(c->key.p, c->nd_first.p,
                                                                 c->nd_count.p, c->nd_nchild.p,
                                                                 c->nd_scan.p, s, m, l);
        c->launches += 1;
        // scan the child counts in place of a separate buffer: grp_flag is free here
        exclusive_scan_u32(c, c->nd_scan.p, c->grp_flag.p, m, &c->dsc->level_count);
        BGB_CUDA(cudaMemcpyAsync(&c->hsc->level_count, &c->dsc->level_count, sizeof(uint32_t),
                                 cudaMemcpyDeviceToHost, c->stream));
        BGB_WAIT(c->stream);
        const int64_t tot = c->hsc->level_count;
        rc = grow_nodes(c, e + tot, e);
        if (rc) return rc;
        k_split_write<<<grid_for(m, 256), 256, 0, c->stream>>>(
            c->key.p, c->nd_first.p, c->nd_count.p, c->nd_child.p, c->nd_nchild.p, c->nd_level.p,
            c->nd_parent.p, c->cell_topo.p, c->grp_flag.p, s, m, e, l);
        c->launches += 1;
        c->level_start[l + 2] = e + tot;
    }
    c->depth = depth;
    c->n_nodes = c->level_start[depth + 1];
    for (int k = depth + 2; k <= MAX_LEVEL + 1; ++k) c->level_start[k] = c->n_nodes;
    return BONSAI_OK;
}

int build_groups(bonsai_ctx *c) {
    const int64_t n = c->n, nn = c->n_nodes;
    BGB_CUDA(cudaMemsetAsync(c->grp_flag.p, 0, (n + 1) * sizeof(uint32_t), c->stream));
    k_group_flags<<<grid_for(nn, 256), 256, 0, c->stream>>>(c->nd_first.p, c->nd_count.p,
                                                             c->nd_nchild.p, c->nd_child.p,
                                                             c->grp_flag.p, nn);
    c->launches += 1;
    uint32_t *gid = c->grp_flag.p + (n + 1);
    exclusive_scan_u32(c, c->grp_flag.p, gid, n, &c->dsc->n_groups);
    BGB_CUDA(cudaMemcpyAsync(&c->hsc->n_groups, &c->dsc->n_groups, sizeof(uint32_t),
                             cudaMemcpyDeviceToHost, c->stream));
    BGB_WAIT(c->stream);
    const int64_t ng = c->hsc->n_groups;
    c->n_groups = ng;
    if (ensure(c->grp_first, ng) || ensure(c->grp_count, ng) || ensure(c->grp_centre, 3 * ng) ||
        ensure(c->grp_box, ng) || ensure(c->grp_half, ng) || ensure(c->grp_lo, ng) ||
        ensure(c->grp_npp, ng) || ensure(c->grp_npc, ng))
        return BONSAI_ENOMEM;
    k_group_write<<<grid_for(n, 256), 256, 0, c->stream>>>(c->grp_flag.p, gid, n, c->grp_first.p);
    k_group_box<<<grid_for((ng + 31) / 32 * 32, 256), 256, 0, c->stream>>>(
        c->pos.p, n, c->grp_first.p, c->grp_count.p, ng, c->grp_centre.p, c->grp_box.p,
        c->grp_half.p, c->grp_lo.p);
    c->launches += 2;
    return BONSAI_OK;
}

void launch_multipoles(bonsai_ctx *c) {
    const int64_t nn = c->n_nodes;
    k_multipoles<true><<<grid_for(nn, 128), 128, 0, c->stream>>>(
        c->pos.p, c->mass.p, c->n, c->nd_first.p, c->nd_count.p, c->nd_child.p, c->nd_nchild.p,
        c->nd_M.p, c->nd_com.p, c->nd_Q.p, nn, 0, nn);
    c->launches += 1;
    for (int l = c->depth - 1; l >= 0; --l) {  // the deepest level holds leaves only
        const int64_t s = c->level_start[l], m = c->level_start[l + 1] - s;
        if (m <= 0) continue;
        k_multipoles<false><<<grid_for(m, 128), 128, 0, c->stream>>>(
            c->pos.p, c->mass.p, c->n, c->nd_first.p, c->nd_count.p, c->nd_child.p,
            c->nd_nchild.p, c->nd_M.p, c->nd_com.p, c->nd_Q.p, nn, s, m);
        c->launches += 1;
    }
}

void launch_body_pack(bonsai_ctx *c) {
    k_body_pack<<<grid_for(c->n, 256, c->sm_count * 16), 256, 0, c->stream>>>(
        c->pos.p, c->mass.p, c->n, c->body_hi.p, c->body_lo.p);
    c->launches += 1;
}

void launch_cell_pack(bonsai_ctx *c, float theta) {
    const int64_t nn = c->n_nodes;
    k_cell_pack<<<grid_for(nn, 256), 256, 0, c->stream>>>(
        c->pos.p, c->n, c->nd_first.p, c->nd_level.p, c->nd_M.p, c->nd_com.p, c->nd_Q.p, nn,
        c->dsc, (double)theta, c->cell_mac.p, c->cell_a.p, c->cell_b.p, c->cell_c.p);
    c->launches += 1;
}

}  // namespace bgb
