// tree.cu -- octree construction from the sorted keys, walk groups, the
// FP64 upward pass and the FP32 record packs (Sec. III.A "tree-construction"
// and "computation of multipole moments"; Sec. I.A leaf size 16; Sec. VI.A
// mass, centre of mass and 3x3 symmetric quadrupole per cell).
//
// The octree is built level by level in one cooperative launch: a node of
// level l holding more than 16 particles is cut into the runs of equal key
// digit l+1 (8 binary searches on its sorted key range); an exclusive scan
// over the level's child counts numbers the children breadth-first, so the
// numbering is a pure function of the sorted keys.  Grid-wide barriers
// separate the counting and writing phases of each level, and the host
// reads the level table once at the end.
//
// The upward pass computes every leaf in one launch (a leaf needs only its
// particles), then visits the levels bottom-up, where internal nodes
// combine their children by the parallel-axis rule; small trees take it in
// one launch instead (each internal node computed by the thread of its last
// finished child).  Every FP64 operation is an explicit round-to-nearest
// intrinsic in a fixed order, so both give the same moments.
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace bgb {


namespace {

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

// Grid-wide barrier of a cooperative launch (every block resident).  The
// block meets, then one thread fences (cumulatively: the block's writes that
// the meeting ordered before it) and arrives on the counter; the last
// arrival resets it and advances the generation.  The
// wait is bounded: after OCT_SPINS polls (a second or so), or as soon as
// another block has given up, the block records ST_TIMEOUT and reports
// failure, so every block's later barriers end too and the kernel returns.
__device__ bool grid_barrier(DevScalars *sc) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        int good = 1;
        volatile uint32_t *gen = &sc->bar_gen;
        volatile int32_t *status = &sc->status;
        const uint32_t g = *gen;  // read before arriving: it cannot advance before we do
        if (atomicAdd(&sc->bar_count, 1u) == gridDim.x - 1u) {
            atomicExch(&sc->bar_count, 0u);
            __threadfence();
            atomicAdd(&sc->bar_gen, 1u);
        } else {
            uint32_t it = 0;
            while (*gen == g) {
                if (++it > OCT_SPINS || (*status & ST_TIMEOUT)) {
                    atomicOr(&sc->status, ST_TIMEOUT);
                    good = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Block-wide exclusive sum of v over OCT_BLOCK threads; *total gets the sum.
__device__ __forceinline__ uint32_t block_excl_sum(uint32_t v, uint32_t *total) {
    __shared__ uint32_t wsum[OCT_BLOCK / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    __syncthreads();  // wsum is reused from the previous call
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < OCT_BLOCK / 32; ++w) {
        const uint32_t x = wsum[w];
        before += w < warp ? x : 0u;
        all += x;
    }
    *total = all;
    return before + inc - v;
}

// The whole octree in one cooperative launch, level by level.  At level l
// (nodes [s, e)), every block takes a contiguous chunk of the level:
//   A. each node of more than NLEAF particles (and l < MAX_LEVEL) counts
//      its non-empty children from the boundaries of digit l+1; the block
//      sums its counts;
//   -- barrier --
//   B. a block's children start after those of all lower blocks (a sum of
//      the per-block counts) and, within the block, after those of its
//      lower nodes (a block scan in node order), so the numbering is
//      breadth-first and a pure function of the sorted keys.  Each node
//      writes its children (first, count, level, parent) and its topology
//      record, and flags the walk groups it starts: the runs of its
//      children of at most NCRIT particles, gathered greedily in key order
//      up to NCRIT particles, a child of more than NCRIT ending the run
//      (its own children are grouped by its thread); the root when it
//      holds at most NCRIT; NCRIT-particle runs of a max-depth leaf that
//      holds more;
//   -- barrier --
// until a level has no children.  Nodes written by other blocks are read
// through L2 (ld.cg).  If the next level would pass cap nodes, nothing of it
// is written: ST_NODE_OVERFLOW and the node count needed so far are
// reported and the host grows the arrays and launches again.
__global__ void __launch_bounds__(OCT_BLOCK) k_octree(
    const uint64_t *__restrict__ key, uint32_t n, uint32_t *first, uint32_t *count,
    uint32_t *child, uint32_t *nchild, uint32_t *level, uint32_t *parent, uint2 *topo,
    uint32_t *__restrict__ flag, uint32_t cap, uint32_t *bsum, uint32_t *bnd, DevScalars *sc) {
    const uint32_t nb = gridDim.x, blk = blockIdx.x, tid = threadIdx.x;
    if (blk == 0 && tid == 0) {
        first[0] = 0;
        count[0] = n;
        level[0] = 0;
        parent[0] = 0;
        sc->oct_level[0] = 0;
        sc->oct_level[1] = 1;
    }
    __syncthreads();  // block 0 owns the root's chunk of level 0
    uint32_t s = 0, e = 1;
    for (int l = 0; l <= MAX_LEVEL; ++l) {
        const uint32_t m = e - s;
        const uint32_t per = (m + nb - 1u) / nb;
        const uint32_t c0 = min(m, blk * per), c1 = min(m, c0 + per);
        // A: child counts (the boundaries kept for B when the level is small
        // enough for the scratch: the searches' latency is what a small level
        // costs)
        const bool keep = m <= (uint32_t)OCT_KEEP;
        uint32_t mine = 0;
        for (uint32_t t = c0 + tid; t < c1; t += OCT_BLOCK) {
            const uint32_t i = s + t;
            const uint32_t f = __ldcg(first + i), c = __ldcg(count + i);
            uint32_t nc = 0;
            if (c > (uint32_t)NLEAF && l < MAX_LEVEL) {
                uint32_t b[9];
                child_bounds(key, f, c, l, b);
#pragma unroll
                for (int d = 0; d < 8; ++d) nc += b[d + 1] > b[d];
                if (keep) {
#pragma unroll
                    for (int d = 1; d < 8; ++d) bnd[(size_t)(d - 1) * OCT_KEEP + t] = b[d];
                }
            }
            nchild[i] = nc;
            mine += nc;
        }
        uint32_t block_total;
        block_excl_sum(mine, &block_total);
        if (tid == 0) bsum[blk] = block_total;
        if (!grid_barrier(sc)) return;
        // B: this block's offset and the level's total
        uint32_t lower = 0, all = 0;
        for (uint32_t k = tid; k < nb; k += OCT_BLOCK) {
            const uint32_t v = __ldcg(bsum + k);
            all += v;
            lower += k < blk ? v : 0u;
        }
        uint32_t lower_sum, all_sum;
        block_excl_sum(lower, &lower_sum);
        block_excl_sum(all, &all_sum);
        const uint32_t ne = e + all_sum;
        if (ne > cap || ne < e) {  // the next level does not fit: write nothing
            if (blk == 0 && tid == 0) {
                atomicOr(&sc->status, ST_NODE_OVERFLOW);
                sc->oct_need = ne < e ? 0xffffffffu : ne;
            }
            return;
        }
        uint32_t carry = e + lower_sum;
        for (uint32_t base = c0; base < c1; base += OCT_BLOCK) {
            const uint32_t t = base + tid;
            const bool valid = t < c1;
            const uint32_t i = s + t;
            const uint32_t nc = valid ? nchild[i] : 0u;
            uint32_t round;
            const uint32_t off = block_excl_sum(nc, &round);
            if (valid) {
                const uint32_t f = __ldcg(first + i), c = __ldcg(count + i);
                if (i == 0 && c <= (uint32_t)NCRIT) flag[f] = 1u;
                if (nc == 0) {
                    child[i] = 0;
                    topo[i] = make_uint2(f, c | LEAF_FLAG);
                    if (c > (uint32_t)NCRIT)
                        for (uint32_t r = 0; r < c; r += NCRIT) flag[f + r] = 1u;
                } else {
                    const uint32_t ch = carry + off;
                    child[i] = ch;
                    topo[i] = make_uint2(ch, nc);
                    uint32_t b[9];
                    if (keep) {  // written by this thread in A
                        b[0] = f;
                        b[8] = f + c;
#pragma unroll
                        for (int d = 1; d < 8; ++d) b[d] = bnd[(size_t)(d - 1) * OCT_KEEP + t];
                    } else {
                        child_bounds(key, f, c, l, b);
                    }
                    uint32_t k = ch, run = 0;
                    bool open = false;
#pragma unroll
                    for (int d = 0; d < 8; ++d) {
                        if (b[d + 1] > b[d]) {
                            const uint32_t cj = b[d + 1] - b[d];
                            first[k] = b[d];
                            count[k] = cj;
                            level[k] = (uint32_t)(l + 1);
                            parent[k] = i;
                            ++k;
                            if (c > (uint32_t)NCRIT) {
                                if (cj > (uint32_t)NCRIT) {
                                    open = false;
                                } else if (!open || run + cj > (uint32_t)NCRIT) {
                                    flag[b[d]] = 1u;
                                    run = cj;
                                    open = true;
                                } else {
                                    run += cj;
                                }
                            }
                        }
                    }
                }
            }
            carry += round;
        }
        if (blk == 0 && tid == 0 && l + 2 <= MAX_LEVEL + 1) sc->oct_level[l + 2] = ne;
        if (ne == e) {  // no children: level l is the deepest
            if (blk == 0 && tid == 0) {
                sc->oct_depth = (uint32_t)l;
                sc->oct_nodes = e;
            }
            return;
        }
        if (!grid_barrier(sc)) return;
        s = e;
        e = ne;
    }
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

// Small trees: the whole upward pass in one launch, with the same FP64
// operations in the same order as k_multipoles.
__device__ __forceinline__ void store_moments(double *__restrict__ M, double *__restrict__ com,
                                              double *__restrict__ Q, int64_t nn, int64_t i,
                                              double Ms, double cx, double cy, double cz,
                                              const double q[6]) {
    M[i] = Ms;
    com[i] = cx;
    com[nn + i] = cy;
    com[2 * nn + i] = cz;
#pragma unroll
    for (int k = 0; k < 6; ++k) Q[k * nn + i] = q[k];
}

// A leaf from its particles: mass, centre of mass, and the second moment
// about the centre of mass.
__device__ void leaf_moments(const double *__restrict__ pos, const double *__restrict__ mass,
                             int64_t n, uint32_t f, uint32_t c, double *__restrict__ M,
                             double *__restrict__ com, double *__restrict__ Q, int64_t nn,
                             int64_t i) {
    double Ms = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    for (uint32_t j = f; j < f + c; ++j) {
        const double mj = mass[j];
        Ms = __dadd_rn(Ms, mj);
        sx = __dadd_rn(sx, __dmul_rn(mj, pos[j]));
        sy = __dadd_rn(sy, __dmul_rn(mj, pos[n + j]));
        sz = __dadd_rn(sz, __dmul_rn(mj, pos[2 * n + j]));
    }
    const double cx = __ddiv_rn(sx, Ms), cy = __ddiv_rn(sy, Ms), cz = __ddiv_rn(sz, Ms);
    double q[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (uint32_t j = f; j < f + c; ++j) {
        const double mj = mass[j];
        const double dx = __dsub_rn(pos[j], cx), dy = __dsub_rn(pos[n + j], cy),
                     dz = __dsub_rn(pos[2 * n + j], cz);
        const double mx = __dmul_rn(mj, dx), my = __dmul_rn(mj, dy);
        q[0] = __dadd_rn(q[0], __dmul_rn(mx, dx));
        q[1] = __dadd_rn(q[1], __dmul_rn(my, dy));
        q[2] = __dadd_rn(q[2], __dmul_rn(__dmul_rn(mj, dz), dz));
        q[3] = __dadd_rn(q[3], __dmul_rn(mx, dy));
        q[4] = __dadd_rn(q[4], __dmul_rn(mx, dz));
        q[5] = __dadd_rn(q[5], __dmul_rn(my, dz));
    }
    store_moments(M, com, Q, nn, i, Ms, cx, cy, cz, q);
}

// An internal node from its children by the parallel-axis rule.  The
// children were written by other threads of this launch: read through L2.
// The loops run over the eight possible children with the absent ones
// masked, so that the loads of all children can be in flight at once; the
// FP64 operations keep their order.
__device__ void internal_moments(uint32_t c0, uint32_t nc, double *__restrict__ M,
                                 double *__restrict__ com, double *__restrict__ Q, int64_t nn,
                                 int64_t i) {
    double Mk[8], X[8], Y[8], Z[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const bool h = (uint32_t)k < nc;
        const uint32_t j = c0 + (h ? (uint32_t)k : 0u);
        Mk[k] = h ? __ldcg(M + j) : 0.0;
        X[k] = __ldcg(com + j);
        Y[k] = __ldcg(com + nn + j);
        Z[k] = __ldcg(com + 2 * nn + j);
    }
    double Ms = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if ((uint32_t)k < nc) {
            Ms = __dadd_rn(Ms, Mk[k]);
            sx = __dadd_rn(sx, __dmul_rn(Mk[k], X[k]));
            sy = __dadd_rn(sy, __dmul_rn(Mk[k], Y[k]));
            sz = __dadd_rn(sz, __dmul_rn(Mk[k], Z[k]));
        }
    }
    const double cx = __ddiv_rn(sx, Ms), cy = __ddiv_rn(sy, Ms), cz = __ddiv_rn(sz, Ms);
    double q[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if ((uint32_t)k < nc) {
            const uint32_t j = c0 + (uint32_t)k;
            const double dx = __dsub_rn(X[k], cx), dy = __dsub_rn(Y[k], cy),
                         dz = __dsub_rn(Z[k], cz);
            const double mx = __dmul_rn(Mk[k], dx), my = __dmul_rn(Mk[k], dy);
            q[0] = __dadd_rn(q[0], __dadd_rn(__ldcg(Q + j), __dmul_rn(mx, dx)));
            q[1] = __dadd_rn(q[1], __dadd_rn(__ldcg(Q + nn + j), __dmul_rn(my, dy)));
            q[2] = __dadd_rn(q[2], __dadd_rn(__ldcg(Q + 2 * nn + j), __dmul_rn(__dmul_rn(Mk[k], dz), dz)));
            q[3] = __dadd_rn(q[3], __dadd_rn(__ldcg(Q + 3 * nn + j), __dmul_rn(mx, dy)));
            q[4] = __dadd_rn(q[4], __dadd_rn(__ldcg(Q + 4 * nn + j), __dmul_rn(mx, dz)));
            q[5] = __dadd_rn(q[5], __dadd_rn(__ldcg(Q + 5 * nn + j), __dmul_rn(my, dz)));
        }
    }
    store_moments(M, com, Q, nn, i, Ms, cx, cy, cz, q);
}

// A thread per node: a leaf's thread computes the leaf, then climbs.  At
// each parent it counts itself in (arrive, zeroed by the caller); the child
// that arrives last, which finds every sibling finished, computes the parent
// and climbs on; the others stop.  Nothing waits, and each node is computed
// once, after all its children.
__global__ void __launch_bounds__(128) k_upward(
    const double *__restrict__ pos, const double *__restrict__ mass, int64_t n,
    const uint32_t *__restrict__ first, const uint32_t *__restrict__ count,
    const uint32_t *__restrict__ child, const uint32_t *__restrict__ nchild,
    const uint32_t *__restrict__ parent, double *__restrict__ M, double *__restrict__ com,
    double *__restrict__ Q, int64_t nn, uint32_t *__restrict__ arrive) {
    const int64_t i = blockIdx.x * 128ll + threadIdx.x;
    if (i >= nn || nchild[i] != 0) return;
    leaf_moments(pos, mass, n, first[i], count[i], M, com, Q, nn, i);
    uint32_t node = (uint32_t)i;
    while (node != 0u) {
        const uint32_t p = parent[node];
        // one acquire-release arrival: this node's moments are released
        // with it, and the last arrival acquires every sibling's
        uint32_t before;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
                     : "=r"(before)
                     : "l"(arrive + p)
                     : "memory");
        if (before != nchild[p] - 1u) break;
        internal_moments(child[p], nchild[p], M, com, Q, nn, p);
        node = p;
    }
}

// ---- groups: runs of consecutive sibling cells of at most NCRIT particles
// in all, flagged at their first particle by k_octree; a scan numbers them
// in particle order.
__global__ void __launch_bounds__(256) k_group_write(const uint32_t *__restrict__ flag,
                                                     const uint32_t *__restrict__ gid, int64_t n,
                                                     uint32_t *__restrict__ gfirst) {
    int64_t i = blockIdx.x * 256ll + threadIdx.x;
    if (i >= n) return;
    if (flag[i]) gfirst[gid[i]] = (uint32_t)i;
}

// Per group: the FP64 box of the members, its FP32 centre (nearest), the
// centre's FP32 remainder, and the half-size rounded up to FP32.  A warp
// takes GPW consecutive groups: for each, all lanes load its members and
// reduce their minima and maxima; lane k keeps those of group k, and the
// FP64 epilogue then runs once per lane for the GPW groups at a time.
template <int GPW>  // groups per warp: 32, 4 or 1, fewer when the groups are few
__global__ void __launch_bounds__(256) k_group_box(const double *__restrict__ pos, int64_t n,
                                                   const uint32_t *__restrict__ gfirst,
                                                   uint32_t *__restrict__ gcount, int64_t ng,
                                                   double *__restrict__ gcentre,
                                                   float4 *__restrict__ gbox,
                                                   float4 *__restrict__ ghalf,
                                                   float4 *__restrict__ glo) {
    const int64_t g0 = ((blockIdx.x * 256ll + threadIdx.x) >> 5) * GPW;
    const int lane = threadIdx.x & 31;
    if (g0 >= ng) return;
    long long myn[3] = {0, 0, 0}, myx[3] = {0, 0, 0};
    const int kend = (int)min((int64_t)GPW, ng - g0);
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

// Grow the node arrays to hold at least need nodes (contents not kept).
static int grow_nodes(bonsai_ctx *c, int64_t need) {
    if ((size_t)need <= c->nd_first.cap) return BONSAI_OK;
    const size_t cap = std::max((size_t)need, c->nd_first.cap + c->nd_first.cap / 2);
    BGB_WAIT(c->stream);  // earlier work may still read the old arrays
    DBuf<uint32_t> *u32s[] = {&c->nd_first, &c->nd_count, &c->nd_child, &c->nd_nchild,
                              &c->nd_level, &c->nd_parent};
    for (DBuf<uint32_t> *b : u32s) {
        cudaFree(b->p);
        b->p = nullptr;
        b->cap = 0;
        if (cudaMalloc(&b->p, cap * sizeof(uint32_t)) != cudaSuccess) {
            b->p = nullptr;
            return BONSAI_ENOMEM;
        }
        b->cap = cap;
    }
    cudaFree(c->cell_topo.p);
    c->cell_topo.p = nullptr;
    c->cell_topo.cap = 0;
    if (cudaMalloc(&c->cell_topo.p, cap * sizeof(uint2)) != cudaSuccess) {
        c->cell_topo.p = nullptr;
        return BONSAI_ENOMEM;
    }
    c->cell_topo.cap = cap;
    return BONSAI_OK;
}

// The octree and the walk-group starts (k_octree, one cooperative launch),
// then the group numbering (a scan of the flags); one readback gives the
// level table, the node count and the group count.  A launch that runs out
// of node storage writes nothing past it and is repeated with larger
// arrays.
int build_octree(bonsai_ctx *c) {
    const int64_t n = c->n;
    int rc = grow_nodes(c, std::max<int64_t>(1024, n / 2 + 64));
    if (rc) return rc;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_octree, OCT_BLOCK, 0) !=
            cudaSuccess ||
        per_sm < 1)
        return BONSAI_ECUDA;
    // enough blocks for the widest possible level (8 children per node of
    // more than NLEAF particles), at most all resident ones
    const int64_t widest = 8 * (n / (NLEAF + 1)) + 1;
    const int64_t blocks =
        std::min<int64_t>((int64_t)per_sm * c->sm_count, (widest + OCT_BLOCK - 1) / OCT_BLOCK);
    if (ensure(c->nd_scan, (size_t)blocks) || ensure(c->nd_bounds, (size_t)7 * OCT_KEEP))
        return BONSAI_ENOMEM;
    for (int attempt = 0;; ++attempt) {
        BGB_CUDA(cudaMemsetAsync(c->grp_flag.p, 0, (n + 1) * sizeof(uint32_t), c->stream));
        // the status word may carry the input check's bit: cleared only
        // for a repeat, when it is known to be clean but for the overflow
        if (attempt > 0) BGB_CUDA(cudaMemsetAsync(&c->dsc->status, 0, sizeof(int32_t), c->stream));
        BGB_CUDA(cudaMemsetAsync(&c->dsc->bar_count, 0, 2 * sizeof(uint32_t), c->stream));
        BGB_CUDA(cudaMemsetAsync(&c->dsc->oct_nodes, 0, 3 * sizeof(uint32_t), c->stream));
        const uint64_t *key = c->key.p;
        uint32_t nn32 = (uint32_t)n, cap = (uint32_t)std::min<size_t>(c->nd_first.cap, 0xffffffffu);
        uint32_t *first = c->nd_first.p, *count = c->nd_count.p, *child = c->nd_child.p;
        uint32_t *nchild = c->nd_nchild.p, *level = c->nd_level.p, *parent = c->nd_parent.p;
        uint2 *topo = c->cell_topo.p;
        uint32_t *flag = c->grp_flag.p, *bsum = c->nd_scan.p, *bnd = c->nd_bounds.p;
        DevScalars *sc = c->dsc;
        void *args[] = {&key, &nn32, &first, &count, &child, &nchild, &level, &parent,
                        &topo, &flag, &cap, &bsum, &bnd, &sc};
        BGB_CUDA(cudaLaunchCooperativeKernel((const void *)k_octree, dim3((unsigned)blocks),
                                             dim3(OCT_BLOCK), args, 0, c->stream));
        c->launches += 1;
        uint32_t *gid = c->grp_flag.p + (n + 1);
        exclusive_scan_u32(c, c->grp_flag.p, gid, n, &c->dsc->n_groups);
        BGB_CUDA(cudaMemcpyAsync(c->hsc, c->dsc, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                                 c->stream));
        BGB_WAIT(c->stream);
        const int32_t st = c->hsc->status;
        if (st & ST_BAD_INPUT) return BONSAI_EINVAL;
        if (st & ST_TIMEOUT) return BONSAI_ETIMEOUT;
        if (st & ST_LONG_TIES) return BUILD_RETRY_EXACT;  // the order is not final
        if (!(st & ST_NODE_OVERFLOW)) break;
        const uint64_t need = c->hsc->oct_need;
        if (need >= 0xffffffffull || attempt > 8) return BONSAI_ENOMEM;
        rc = grow_nodes(c, (int64_t)std::max<uint64_t>(need + need / 2, 2 * c->nd_first.cap));
        if (rc) return rc;
    }
    const DevScalars &h = *c->hsc;
    c->depth = (int)h.oct_depth;
    c->n_nodes = h.oct_nodes;
    for (int k = 0; k <= c->depth + 1; ++k) c->level_start[k] = h.oct_level[k];
    for (int k = c->depth + 2; k <= MAX_LEVEL + 1; ++k) c->level_start[k] = c->n_nodes;
    c->n_groups = h.n_groups;
    return BONSAI_OK;
}

int build_groups(bonsai_ctx *c) {
    const int64_t n = c->n, ng = c->n_groups;
    if (ensure(c->grp_first, ng) || ensure(c->grp_count, ng) || ensure(c->grp_centre, 3 * ng) ||
        ensure(c->grp_box, ng) || ensure(c->grp_half, ng) || ensure(c->grp_lo, ng) ||
        ensure(c->grp_npp, ng) || ensure(c->grp_npc, ng))
        return BONSAI_ENOMEM;
    const uint32_t *gid = c->grp_flag.p + (n + 1);
    k_group_write<<<grid_for(n, 256), 256, 0, c->stream>>>(c->grp_flag.p, gid, n, c->grp_first.p);
    // groups per warp: as many as still leave four warps per scheduler
    const int64_t warps = 16 * (int64_t)c->sm_count;
    if (ng / 32 >= warps)
        k_group_box<32><<<grid_for((ng + 31) / 32 * 32, 256), 256, 0, c->stream>>>(
            c->pos.p, n, c->grp_first.p, c->grp_count.p, ng, c->grp_centre.p, c->grp_box.p,
            c->grp_half.p, c->grp_lo.p);
    else if (ng / 4 >= warps)
        k_group_box<4><<<grid_for((ng + 3) / 4 * 32, 256), 256, 0, c->stream>>>(
            c->pos.p, n, c->grp_first.p, c->grp_count.p, ng, c->grp_centre.p, c->grp_box.p,
            c->grp_half.p, c->grp_lo.p);
    else
        k_group_box<1><<<grid_for(ng * 32, 256), 256, 0, c->stream>>>(
            c->pos.p, n, c->grp_first.p, c->grp_count.p, ng, c->grp_centre.p, c->grp_box.p,
            c->grp_half.p, c->grp_lo.p);
    c->launches += 2;
    return BONSAI_OK;
}

// Below UPWARD_ONE_LAUNCH nodes the one-launch pass (k_upward) is used:
// there launch latency dominates.  Above, its climbing threads would run
// alone in their warps on the scarce FP64 pipe, and a launch per level,
// with every lane of a warp on its own node, is faster.
constexpr int64_t UPWARD_ONE_LAUNCH = 1 << 16;

int launch_multipoles(bonsai_ctx *c) {
    const int64_t nn = c->n_nodes;
    if (nn <= UPWARD_ONE_LAUNCH) {
        if (ensure(c->nd_arrive, (size_t)nn)) return BONSAI_ENOMEM;
        BGB_CUDA(cudaMemsetAsync(c->nd_arrive.p, 0, nn * sizeof(uint32_t), c->stream));
        k_upward<<<grid_for(nn, 128), 128, 0, c->stream>>>(
            c->pos.p, c->mass.p, c->n, c->nd_first.p, c->nd_count.p, c->nd_child.p,
            c->nd_nchild.p, c->nd_parent.p, c->nd_M.p, c->nd_com.p, c->nd_Q.p, nn,
            c->nd_arrive.p);
        c->launches += 1;
        return BONSAI_OK;
    }
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
    return BONSAI_OK;
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
