// let.cu -- domains and local essential trees (Sec. III.B), emulated with
// one context per domain on one GPU.
//
// Domains are equal pieces of the global Peano-Hilbert order; a domain's
// tree is built in the global cube, so that it is a branch of the global
// octree (Sec. III.B.1).  A local essential tree (LET) is the part of a
// domain's tree that a remote domain needs (Sec. III.B.2).  It is found by
// walking the tree with every group box of the remote domain and marking
// each cell reached (and each cell opened).  The marked cells, in the
// tree's breadth-first order, form a tree of their own: an opened cell keeps
// all its children, an opened leaf its particles, a cell no group opens
// becomes a childless, particle-less leaf.  Every cell the remote groups'
// walks reach is in it, and every cell they use whole or open is used whole
// or opened in it, so walking the LET gives exactly the lists of walking the
// whole remote tree.  The LET owns its arrays: they are the data a process
// would send.
#include <new>

#include "internal.cuh"

struct bonsai_let {
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    float theta = 0.0f;
    int64_t nn = 0, np = 0, src_nodes = 0;
    bgb::DBuf<float4> mac, ca, cb, cc, hi, lo;
    bgb::DBuf<uint2> topo;
    bgb::DBuf<uint32_t> src_node, kind;  // per LET cell: source cell, 0 used whole / 1 opened cell / 2 opened leaf
    bgb::DBuf<uint32_t> vis, opn, vscan, pcount, pscan, tmp, front;
    bgb::DBuf<int32_t> status;  // [0]: frontier overflow
    bool has_sources = false;   // src_node / kind describe the current cells
    uint32_t *dtot = nullptr;   // device: {cells, particles}
    uint32_t *htot = nullptr;   // pinned host mirror
};

namespace bgb {

namespace {

constexpr int MARK_WARPS = 4;        // warps per block of the marking walk
constexpr int MARK_FCAP = 16384;     // frontier entries per buffer per warp

__global__ void k_set_cube(DevScalars *sc, double lo0, double lo1, double lo2, double L) {
    sc->lo[0] = lo0;
    sc->lo[1] = lo1;
    sc->lo[2] = lo2;
    sc->L = L;
    sc->scale = __ddiv_rn(0x1p21, L);
}

__global__ void __launch_bounds__(256) k_domain_state(const double *__restrict__ pos,
                                                     const double *__restrict__ vel,
                                                     const double *__restrict__ mass,
                                                     const uint32_t *__restrict__ id, int64_t n,
                                                     int64_t first, int64_t count,
                                                     double *__restrict__ pos_o,
                                                     double *__restrict__ vel_o,
                                                     double *__restrict__ mass_o,
                                                     uint32_t *__restrict__ id_o) {
    for (int64_t k = blockIdx.x * 256ll + threadIdx.x; k < count; k += (int64_t)gridDim.x * 256) {
        const int64_t i = first + k;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (pos_o) pos_o[d * count + k] = pos[d * n + i];
            if (vel_o) vel_o[d * count + k] = vel[d * n + i];
        }
        if (mass_o) mass_o[k] = mass[i];
        if (id_o) id_o[k] = id[i];
    }
}

// One warp per group of the remote domain (grid-stride): a breadth-first
// walk of the source tree with the group's box, marking every cell reached
// (vis) and every cell opened (opn).  The frontier lives in per-warp
// global scratch; an overflow stops adding cells and sets status[0].
__global__ void __launch_bounds__(MARK_WARPS * 32) k_let_mark(
    const float4 *__restrict__ mac, const uint2 *__restrict__ topo,
    const float4 *__restrict__ gbox, const float4 *__restrict__ ghalf, int64_t ngroups,
    uint32_t *__restrict__ vis, uint32_t *__restrict__ opn, uint32_t *__restrict__ front,
    int32_t *__restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * MARK_WARPS + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * MARK_WARPS;
    uint32_t *fa = front + gw * 2 * MARK_FCAP;
    uint32_t *fb = fa + MARK_FCAP;
    for (int64_t g = gw; g < ngroups; g += nw) {
        const float4 box = gbox[g], half = ghalf[g];
        uint32_t *cur = fa, *nxt = fb;
        if (lane == 0) cur[0] = 0u;
        uint32_t ncur = 1;
        bool overflow = false;
        __syncwarp();
        while (ncur > 0) {
            uint32_t nnext = 0;
            for (uint32_t base = 0; base < ncur; base += 32) {
                const uint32_t idx = base + lane;
                const bool valid = idx < ncur;
                const uint32_t node = valid ? cur[idx] : 0u;
                const float4 m = mac[node];
                const uint2 tp = topo[node];
                const bool open = valid && mac_open(m, box, half);
                if (valid) vis[node] = 1u;
                if (open) opn[node] = 1u;
                const uint32_t nch = (open && (tp.y & LEAF_FLAG) == 0u) ? tp.y : 0u;
                // warp scan of the children counts
                uint32_t inc = nch;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += t;
                }
                const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
                const uint32_t off = inc - nch;
                if (nnext + tot > (uint32_t)MARK_FCAP) {
                    overflow = true;
                } else {
                    for (uint32_t k = 0; k < nch; ++k) nxt[nnext + off + k] = tp.x + k;
                    nnext += tot;
                }
            }
            __threadfence_block();
            __syncwarp();
            uint32_t *t = cur;
            cur = nxt;
            nxt = t;
            ncur = nnext;
        }
        if (overflow && lane == 0) atomicOr(&status[0], 1);
        __syncwarp();
    }
}

// Particle count of each marked, opened leaf (the particles the LET carries).
__global__ void __launch_bounds__(256) k_let_counts(const uint2 *__restrict__ topo,
                                                   const uint32_t *__restrict__ vis,
                                                   const uint32_t *__restrict__ opn, int64_t nn,
                                                   uint32_t *__restrict__ pcount) {
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < nn; i += (int64_t)gridDim.x * 256) {
        const uint2 t = topo[i];
        const bool leaf = (t.y & LEAF_FLAG) != 0u;
        pcount[i] = (vis[i] && opn[i] && leaf) ? (t.y & ~LEAF_FLAG) : 0u;
    }
}

// The marked cells, in breadth-first order, as a tree of their own.
__global__ void __launch_bounds__(256) k_let_compact(
    const float4 *__restrict__ mac, const uint2 *__restrict__ topo, const float4 *__restrict__ ca,
    const float4 *__restrict__ cb, const float4 *__restrict__ cc, const float4 *__restrict__ bhi,
    const float4 *__restrict__ blo, int64_t nn, const uint32_t *__restrict__ vis,
    const uint32_t *__restrict__ opn, const uint32_t *__restrict__ vscan,
    const uint32_t *__restrict__ pscan, float4 *__restrict__ lmac, uint2 *__restrict__ ltopo,
    float4 *__restrict__ lca, float4 *__restrict__ lcb, float4 *__restrict__ lcc,
    float4 *__restrict__ lhi, float4 *__restrict__ llo, uint32_t *__restrict__ src_node,
    uint32_t *__restrict__ kind) {
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < nn; i += (int64_t)gridDim.x * 256) {
        if (!vis[i]) continue;
        const uint32_t li = vscan[i];
        lmac[li] = mac[i];
        lca[li] = ca[i];
        lcb[li] = cb[i];
        lcc[li] = cc[i];
        src_node[li] = (uint32_t)i;
        const uint2 t = topo[i];
        const bool leaf = (t.y & LEAF_FLAG) != 0u;
        if (!opn[i]) {
            ltopo[li] = make_uint2(0u, LEAF_FLAG);  // used whole by every remote group
            kind[li] = 0u;
        } else if (!leaf) {
            ltopo[li] = make_uint2(vscan[t.x], t.y);  // all children are marked: contiguous
            kind[li] = 1u;
        } else {
            const uint32_t c = t.y & ~LEAF_FLAG, p = pscan[i];
            ltopo[li] = make_uint2(p, t.y);
            kind[li] = 2u;
            for (uint32_t k = 0; k < c; ++k) {
                lhi[p + k] = bhi[t.x + k];
                llo[p + k] = blo[t.x + k];
            }
        }
    }
}

// A received LET's topology must describe a tree that the walk can follow
// safely: an internal cell's 1-8 children come after it (so no path
// returns to a cell) and inside the cell array, a leaf's particles inside
// the particle array.  Any other entry sets status[0].
__global__ void __launch_bounds__(256) k_let_validate(const uint2 *__restrict__ topo, int64_t nn,
                                                     int64_t np, int32_t *__restrict__ status) {
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < nn; i += (int64_t)gridDim.x * 256) {
        const uint2 t = topo[i];
        const uint64_t cnt = t.y & ~LEAF_FLAG;
        const bool ok = (t.y & LEAF_FLAG) ? (uint64_t)t.x + cnt <= (uint64_t)np
                                          : (cnt >= 1 && cnt <= 8 && (int64_t)t.x > i &&
                                             (uint64_t)t.x + cnt <= (uint64_t)nn);
        if (!ok) atomicOr(&status[0], 1);
    }
}

}  // namespace

void launch_set_cube(bonsai_ctx *c) {
    k_set_cube<<<1, 1, 0, c->stream>>>(c->dsc, c->cube[0], c->cube[1], c->cube[2], c->cube[3]);
    c->launches += 1;
}

}  // namespace bgb

using namespace bgb;

extern "C" int tree_domain_state(bonsai_ctx *c, int64_t first, int64_t count, double *pos,
                                 double *vel, double *mass, uint32_t *caller_id) {
    if (!c || first < 0 || count < 1) return BONSAI_EINVAL;
    if (!c->have_tree) return BONSAI_ESTATE;
    if (first > c->n || count > c->n - first) return BONSAI_EINVAL;
    k_domain_state<<<grid_for(count, 256, c->sm_count * 16), 256, 0, c->stream>>>(
        c->pos.p, c->vel.p, c->mass.p, c->id.p, c->n, first, count, pos, vel, mass, caller_id);
    c->launches += 1;
    BGB_CUDA(cudaPeekAtLastError());
    BGB_WAIT(c->stream);
    return BONSAI_OK;
}

extern "C" int let_create(bonsai_let **out, void *stream) {
    if (!out) return BONSAI_EINVAL;
    *out = nullptr;
    bonsai_let *l = new (std::nothrow) bonsai_let();
    if (!l) return BONSAI_ENOMEM;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&l->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaMalloc(&l->dtot, 4 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost(&l->htot, 4 * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        if (l->dtot) cudaFree(l->dtot);
        delete l;
        return BONSAI_ECUDA;
    }
    l->stream = static_cast<cudaStream_t>(stream);
    *out = l;
    return BONSAI_OK;
}

extern "C" void let_destroy(bonsai_let *l) {
    if (!l) return;
    wait_stream(l->stream);  // bounded; cudaFree below waits for the device in any case
    release(l->mac); release(l->ca); release(l->cb); release(l->cc); release(l->hi); release(l->lo);
    release(l->topo); release(l->src_node); release(l->kind); release(l->vis); release(l->opn);
    release(l->vscan); release(l->pcount); release(l->pscan); release(l->tmp); release(l->front);
    release(l->status);
    if (l->dtot) cudaFree(l->dtot);
    if (l->htot) cudaFreeHost(l->htot);
    delete l;
}

namespace bgb {

// The LET of src's tree for the group boxes (box, half: device float4 [ng],
// {c.xyz, 0} and {h.xyz, 0} as the walk stores them).
static int let_build_impl(bonsai_let *l, bonsai_ctx *src, const float4 *box, const float4 *half,
                          int64_t ng, float theta) {
    cudaStream_t s = l->stream;
    if (src->packed_theta != theta) {  // the source's cell records at this theta
        launch_cell_pack(src, theta);
        src->packed_theta = theta;
    }
    BGB_WAIT(src->stream);  // the boxes and records come from finished work
    const int64_t nn = src->n_nodes;
    int blocks = src->sm_count * 2;
    const int64_t need_blocks = (ng + MARK_WARPS - 1) / MARK_WARPS;
    if (blocks > need_blocks) blocks = (int)need_blocks;
    if (blocks < 1) blocks = 1;
    if (ensure(l->vis, nn) || ensure(l->opn, nn) || ensure(l->vscan, nn) || ensure(l->pcount, nn) ||
        ensure(l->pscan, nn) || ensure(l->tmp, scan_tmp_elems(nn)) ||
        ensure(l->front, (size_t)blocks * MARK_WARPS * 2 * MARK_FCAP) || ensure(l->status, 4))
        return BONSAI_ENOMEM;
    BGB_CUDA(cudaMemsetAsync(l->vis.p, 0, nn * sizeof(uint32_t), s));
    BGB_CUDA(cudaMemsetAsync(l->opn.p, 0, nn * sizeof(uint32_t), s));
    BGB_CUDA(cudaMemsetAsync(l->status.p, 0, 4 * sizeof(int32_t), s));
    k_let_mark<<<blocks, MARK_WARPS * 32, 0, s>>>(src->cell_mac.p, src->cell_topo.p, box, half, ng,
                                                 l->vis.p, l->opn.p, l->front.p, l->status.p);
    k_let_counts<<<grid_for(nn, 256, l->sm_count * 16), 256, 0, s>>>(src->cell_topo.p, l->vis.p,
                                                                     l->opn.p, nn, l->pcount.p);
    exclusive_scan_into(s, l->vis.p, l->vscan.p, nn, l->tmp.p, l->dtot);
    exclusive_scan_into(s, l->pcount.p, l->pscan.p, nn, l->tmp.p, l->dtot + 1);
    BGB_CUDA(cudaMemcpyAsync(l->htot, l->dtot, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BGB_CUDA(cudaMemcpyAsync(&l->htot[2], l->status.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BGB_WAIT(s);
    if ((int32_t)l->htot[2]) return BONSAI_EOVERFLOW;
    const int64_t lnn = l->htot[0], lnp = l->htot[1];
    if (ensure(l->mac, lnn) || ensure(l->topo, lnn) || ensure(l->ca, lnn) || ensure(l->cb, lnn) ||
        ensure(l->cc, lnn) || ensure(l->src_node, lnn) || ensure(l->kind, lnn) ||
        ensure(l->hi, lnp) || ensure(l->lo, lnp))
        return BONSAI_ENOMEM;
    k_let_compact<<<grid_for(nn, 256, l->sm_count * 16), 256, 0, s>>>(
        src->cell_mac.p, src->cell_topo.p, src->cell_a.p, src->cell_b.p, src->cell_c.p,
        src->body_hi.p, src->body_lo.p, nn, l->vis.p, l->opn.p, l->vscan.p, l->pscan.p, l->mac.p,
        l->topo.p, l->ca.p, l->cb.p, l->cc.p, l->hi.p, l->lo.p, l->src_node.p, l->kind.p);
    BGB_CUDA(cudaPeekAtLastError());
    BGB_WAIT(s);
    l->nn = lnn;
    l->np = lnp;
    l->src_nodes = nn;
    l->theta = theta;
    l->has_sources = true;
    return BONSAI_OK;
}

}  // namespace bgb

extern "C" int let_build(bonsai_let *l, bonsai_ctx *src, const bonsai_ctx *dst, float theta) {
    if (!l || !src || !dst || !(theta > 0.0f) || !isfinite(theta)) return BONSAI_EINVAL;
    if (!src->have_tree || !dst->have_tree) return BONSAI_ESTATE;
    if (src->cube[3] != dst->cube[3] || src->cube[3] <= 0.0 || src->cube[0] != dst->cube[0] ||
        src->cube[1] != dst->cube[1] || src->cube[2] != dst->cube[2])
        return BONSAI_EINVAL;  // both must be branches of one global octree
    BGB_WAIT(dst->stream);  // dst's group boxes come from a finished build
    return let_build_impl(l, src, dst->grp_box.p, dst->grp_half.p, dst->n_groups, theta);
}

extern "C" int let_build_boxes(bonsai_let *l, bonsai_ctx *src, const float *box, const float *half,
                               int64_t ngroups, float theta) {
    if (!l || !src || !box || !half || ngroups < 0 || !(theta > 0.0f) || !isfinite(theta))
        return BONSAI_EINVAL;
    if (!src->have_tree) return BONSAI_ESTATE;
    if (ngroups == 0) {  // nothing to walk: an empty LET
        l->nn = l->np = 0;
        l->src_nodes = src->n_nodes;
        l->has_sources = false;
        return BONSAI_OK;
    }
    return let_build_impl(l, src, reinterpret_cast<const float4 *>(box),
                          reinterpret_cast<const float4 *>(half), ngroups, theta);
}

extern "C" int tree_get_group_boxes(bonsai_ctx *c, float *box, float *half, int64_t *ngroups) {
    if (!c) return BONSAI_EINVAL;
    if (!c->have_tree) return BONSAI_ESTATE;
    if (ngroups) *ngroups = c->n_groups;
    const size_t bytes = (size_t)c->n_groups * sizeof(float4);
    if (box) BGB_CUDA(cudaMemcpyAsync(box, c->grp_box.p, bytes, cudaMemcpyDeviceToDevice, c->stream));
    if (half) BGB_CUDA(cudaMemcpyAsync(half, c->grp_half.p, bytes, cudaMemcpyDeviceToDevice, c->stream));
    BGB_WAIT(c->stream);
    return BONSAI_OK;
}

namespace {

// Packed LET: a 64-byte header, then the cell records (mac, ca, cb, cc as
// float4 [nn], topo as uint2 [nn] padded to 16 bytes) and the particle
// records (hi, lo as float4 [np]).
struct LetHeader {
    uint64_t magic;   // "BGBLET01"
    int64_t nn, np;
    int64_t bytes;    // total packed size
    float theta;
    uint32_t pad[7];
};
static_assert(sizeof(LetHeader) == 64, "LET header");
constexpr uint64_t LET_MAGIC = 0x31305445'4C424742ull;  // "BGBLET01" little-endian

int64_t pad16(int64_t b) { return (b + 15) & ~(int64_t)15; }
int64_t packed_bytes(int64_t nn, int64_t np) {
    return (int64_t)sizeof(LetHeader) + 4 * 16 * nn + pad16(8 * nn) + 2 * 16 * np;
}

}  // namespace

extern "C" int let_pack(const bonsai_let *l, void *buf, int64_t cap, int64_t *bytes) {
    if (!l || !bytes) return BONSAI_EINVAL;
    const int64_t b = packed_bytes(l->nn, l->np);
    *bytes = b;
    if (!buf) return BONSAI_OK;
    if (cap < b || (reinterpret_cast<uintptr_t>(buf) & 15u)) return BONSAI_EINVAL;
    LetHeader h{};
    h.magic = LET_MAGIC;
    h.nn = l->nn;
    h.np = l->np;
    h.bytes = b;
    h.theta = l->theta;
    cudaStream_t s = l->stream;
    char *p = static_cast<char *>(buf);
    BGB_CUDA(cudaMemcpyAsync(p, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    p += sizeof(h);
    const size_t c16 = 16 * (size_t)l->nn, p16 = 16 * (size_t)l->np;
    if (l->nn) {
        BGB_CUDA(cudaMemcpyAsync(p, l->mac.p, c16, cudaMemcpyDeviceToDevice, s));
        BGB_CUDA(cudaMemcpyAsync(p + c16, l->ca.p, c16, cudaMemcpyDeviceToDevice, s));
        BGB_CUDA(cudaMemcpyAsync(p + 2 * c16, l->cb.p, c16, cudaMemcpyDeviceToDevice, s));
        BGB_CUDA(cudaMemcpyAsync(p + 3 * c16, l->cc.p, c16, cudaMemcpyDeviceToDevice, s));
        BGB_CUDA(cudaMemcpyAsync(p + 4 * c16, l->topo.p, 8 * (size_t)l->nn, cudaMemcpyDeviceToDevice, s));
    }
    p += 4 * c16 + pad16(8 * l->nn);
    if (l->np) {
        BGB_CUDA(cudaMemcpyAsync(p, l->hi.p, p16, cudaMemcpyDeviceToDevice, s));
        BGB_CUDA(cudaMemcpyAsync(p + p16, l->lo.p, p16, cudaMemcpyDeviceToDevice, s));
    }
    BGB_WAIT(s);  // h lives on this stack frame
    return BONSAI_OK;
}

extern "C" int let_unpack(bonsai_let *l, const void *buf, int64_t bytes) {
    if (!l || !buf || bytes < (int64_t)sizeof(LetHeader) || (reinterpret_cast<uintptr_t>(buf) & 15u))
        return BONSAI_EINVAL;
    cudaStream_t s = l->stream;
    LetHeader h{};
    BGB_CUDA(cudaMemcpyAsync(&h, buf, sizeof(h), cudaMemcpyDeviceToHost, s));
    BGB_WAIT(s);
    if (h.magic != LET_MAGIC || h.nn < 0 || h.np < 0 || h.nn > 0xffffffffll || h.np > 0xffffffffll ||
        h.bytes != bytes || packed_bytes(h.nn, h.np) != bytes || !(h.theta > 0.0f))
        return BONSAI_EINVAL;
    if (ensure(l->mac, h.nn) || ensure(l->topo, h.nn) || ensure(l->ca, h.nn) || ensure(l->cb, h.nn) ||
        ensure(l->cc, h.nn) || ensure(l->hi, h.np) || ensure(l->lo, h.np))
        return BONSAI_ENOMEM;
    const char *p = static_cast<const char *>(buf) + sizeof(LetHeader);
    const size_t c16 = 16 * (size_t)h.nn, p16 = 16 * (size_t)h.np;
    if (ensure(l->status, 4)) return BONSAI_ENOMEM;
    if (h.nn) {
        BGB_CUDA(cudaMemcpyAsync(l->mac.p, p, c16, cudaMemcpyDeviceToDevice, s));
        BGB_CUDA(cudaMemcpyAsync(l->ca.p, p + c16, c16, cudaMemcpyDeviceToDevice, s));
        BGB_CUDA(cudaMemcpyAsync(l->cb.p, p + 2 * c16, c16, cudaMemcpyDeviceToDevice, s));
        BGB_CUDA(cudaMemcpyAsync(l->cc.p, p + 3 * c16, c16, cudaMemcpyDeviceToDevice, s));
        BGB_CUDA(cudaMemcpyAsync(l->topo.p, p + 4 * c16, 8 * (size_t)h.nn, cudaMemcpyDeviceToDevice, s));
    }
    p += 4 * c16 + pad16(8 * h.nn);
    if (h.np) {
        BGB_CUDA(cudaMemcpyAsync(l->hi.p, p, p16, cudaMemcpyDeviceToDevice, s));
        BGB_CUDA(cudaMemcpyAsync(l->lo.p, p + p16, p16, cudaMemcpyDeviceToDevice, s));
    }
    BGB_CUDA(cudaMemsetAsync(l->status.p, 0, 4 * sizeof(int32_t), s));
    if (h.nn) {
        k_let_validate<<<grid_for(h.nn, 256, l->sm_count * 16), 256, 0, s>>>(l->topo.p, h.nn, h.np,
                                                                            l->status.p);
        BGB_CUDA(cudaPeekAtLastError());
    }
    int32_t bad = 0;
    BGB_CUDA(cudaMemcpyAsync(&bad, l->status.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BGB_WAIT(s);
    if (bad) {
        l->nn = l->np = 0;
        l->has_sources = false;
        return BONSAI_EINVAL;
    }
    l->nn = h.nn;
    l->np = h.np;
    l->theta = h.theta;
    l->src_nodes = 0;
    l->has_sources = false;  // the source-cell map stays with the sender
    return BONSAI_OK;
}

extern "C" int let_get_info(const bonsai_let *l, int64_t out[4]) {
    if (!l || !out) return BONSAI_EINVAL;
    out[0] = l->nn;
    out[1] = l->np;
    out[2] = l->nn * (int64_t)(sizeof(float4) * 4 + sizeof(uint2)) + l->np * (int64_t)(2 * sizeof(float4));
    out[3] = l->src_nodes;
    return BONSAI_OK;
}

extern "C" int let_debug_cells(const bonsai_let *l, uint32_t *src_node, uint32_t *kind) {
    if (!l) return BONSAI_EINVAL;
    if (l->nn == 0 || !l->has_sources) return BONSAI_ESTATE;
    if (src_node) BGB_CUDA(cudaMemcpyAsync(src_node, l->src_node.p, l->nn * sizeof(uint32_t),
                                           cudaMemcpyDeviceToDevice, l->stream));
    if (kind) BGB_CUDA(cudaMemcpyAsync(kind, l->kind.p, l->nn * sizeof(uint32_t),
                                       cudaMemcpyDeviceToDevice, l->stream));
    BGB_WAIT(l->stream);
    return BONSAI_OK;
}

extern "C" int let_forces(bonsai_ctx *dst, const bonsai_let *l, float eps) {
    if (!dst || !l || !(eps >= 0.0f) || !isfinite(eps)) return BONSAI_EINVAL;
    if (!dst->have_forces || l->nn == 0) return BONSAI_ESTATE;
    BGB_CUDA(cudaMemsetAsync(&dst->dsc->n_pp, 0, 2 * sizeof(uint64_t), dst->stream));
    BGB_CUDA(cudaMemsetAsync(&dst->dsc->status, 0, 3 * sizeof(int32_t), dst->stream));
    const LetTree t{l->mac.p, l->topo.p, l->ca.p, l->cb.p, l->cc.p, l->hi.p, l->lo.p, l->nn};
    int rc = walk_let(dst, t, eps);
    if (rc) return rc;
    BGB_CUDA(cudaMemcpyAsync(dst->hsc, dst->dsc, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                             dst->stream));
    BGB_WAIT(dst->stream);
    cudaEventElapsedTime(&dst->stats.ms_walk, dst->ev[8], dst->ev[9]);
    dst->stats.n_pp = dst->hsc->n_pp;
    dst->stats.n_pc = dst->hsc->n_pc;
    dst->stats.flops = 23.0 * (double)dst->hsc->n_pp + 65.0 * (double)dst->hsc->n_pc;
    if (dst->hsc->status & ST_OVERFLOW) {
        dst->have_forces = false;
        return BONSAI_EOVERFLOW;
    }
    return BONSAI_OK;
}
