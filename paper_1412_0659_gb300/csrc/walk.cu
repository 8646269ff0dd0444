// walk.cu -- the fused group walk and force evaluation (Sec. III.A: the
// walk and the force computation in one kernel, interaction lists kept on
// chip and evaluated on the fly; Eq. 1-2 of Sec. VI.A).
//
// One warp owns one group of <= 64 targets (two per lane when the group has
// more than 32).  Warps fetch groups from a global counter, so the grid is
// persistent: one wave of resident warps.  The walk is breadth-first: each
// lane tests one cell of the current frontier against the group's box
// (ballot + popc compaction replaces Bonsai's shared-memory stacks):
//   accepted          -> its multipole record is converted to group-relative
//                        FP32 and appended to the warp's p-c ring in smem;
//   opened leaf       -> its particles are appended to the p-p ring (a warp
//                        scan of the leaf sizes spreads them over lanes);
//   opened internal   -> its children go to the next frontier (global
//                        scratch, one region per resident warp, L2-resident).
// Whenever a ring holds 32 entries the warp evaluates them: every lane reads
// the same entry (shared-memory broadcast) and applies it to its targets.
// The list never reaches DRAM.  All force arithmetic is FP32 on coordinates
// relative to the group centre; the opening test is evaluated exactly as
// specified (round-to-nearest FP32, fixed order) so that the interaction
// lists are a pure function of the FP32-rounded cell and group data.
#include "internal.cuh"

namespace bgb {

namespace {

constexpr int WALK_WARPS = 4;  // warps per block
constexpr int RING = 64;       // entries per ring (power of two)
constexpr int FCAP = 16384;    // frontier entries per buffer per warp

struct __align__(16) WarpLists {
    float4 ca[RING];  // {dx, dy, dz, M}: cell com relative to the group centre
    float4 cb[RING];  // -3 x {Qxx, Qyy, Qzz, Qxy}
    float4 cc[RING];  // {-3 Qxz, -3 Qyz, -trQ/2, -3/2 trQ}
    float4 pp[RING];  // {dx, dy, dz, m}: particle relative to the group centre
    int pid[RING];    // sorted index of the particle (self-pair mask)
};

struct WalkArgs {
    const float4 *mac;
    const uint2 *topo;
    const float4 *ca, *cb, *cc;
    const float4 *body_hi, *body_lo;
    const uint32_t *gfirst, *gcount;
    const float4 *gbox, *ghalf, *glo;
    int64_t ngroups;
    int64_t n;
    float eps2;
    float G;
    float *acc;  // sorted [3][n]
    float *pot;  // sorted [n]
    float *acc_c;  // caller order [3][n] or null
    float *pot_c;  // caller order [n] or null
    const uint32_t *id;
    int32_t *gnpp, *gnpc;
    uint32_t *frontier;
    DevScalars *sc;
};

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, uint32_t &total) {
    const int lane = threadIdx.x & 31;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    total = __shfl_sync(0xffffffffu, inc, 31);
    return inc - v;
}

// Eq. 1-2 for one cell on one target, Plummer-softened in every power of s:
//   r = com - x_i, s^2 = r^2 + eps^2, u = 1/s, w = u^2,
//   phi += -u (M + w (-trQ/2 + 3/2 rQr w))
//   a   += u w (M + w (-3/2 trQ + 15/2 rQr w)) r - 3 u^5 Q r.
// The cell record holds Q' = -3Q, so with q = r.Q'r w = -3 rQr w the two
// brackets are M + w (c.z - q/2) and M + w (c.w - 5q/2), with c.z = -trQ/2
// and c.w = -3/2 trQ; the last term is u w w (Q'r).  35 FP32 instructions.
__device__ __forceinline__ void pc_one(const float4 a, const float4 b, const float4 c, float tx,
                                       float ty, float tz, float eps2, float &ax, float &ay,
                                       float &az, float &ph) {
    const float rx = a.x - tx, ry = a.y - ty, rz = a.z - tz;
    float s2 = fmaf(rx, rx, eps2);
    s2 = fmaf(ry, ry, s2);
    s2 = fmaf(rz, rz, s2);
    const float u = rsqrtf(s2);
    const float w = u * u;
    const float qx = fmaf(b.x, rx, fmaf(b.w, ry, c.x * rz));  // Q'r
    const float qy = fmaf(b.w, rx, fmaf(b.y, ry, c.y * rz));
    const float qz = fmaf(c.x, rx, fmaf(c.y, ry, b.z * rz));
    const float q = fmaf(rx, qx, fmaf(ry, qy, rz * qz)) * w;  // r.Q'r / s^2
    const float tp = fmaf(w, fmaf(-0.5f, q, c.z), a.w);
    ph = fmaf(-u, tp, ph);
    const float uw = u * w;
    const float A = uw * fmaf(w, fmaf(-2.5f, q, c.w), a.w);
    const float B = uw * w;
    ax = fmaf(A, rx, ax);
    ay = fmaf(A, ry, ay);
    az = fmaf(A, rz, az);
    ax = fmaf(B, qx, ax);
    ay = fmaf(B, qy, ay);
    az = fmaf(B, qz, az);
}

// Monopole p-p term.  With MASK the self pair (same sorted index) is skipped
// here; without it the self pair adds exactly -m_i rsqrt(eps^2) to phi and
// nothing to a (r = 0), which the caller removes once per target.
template <bool MASK>
__device__ __forceinline__ void pp_one(const float4 s, int sid, int tid, float tx, float ty,
                                       float tz, float eps2, float &ax, float &ay, float &az,
                                       float &ph) {
    const float dx = s.x - tx, dy = s.y - ty, dz = s.z - tz;
    float r2 = fmaf(dx, dx, eps2);
    r2 = fmaf(dy, dy, r2);
    r2 = fmaf(dz, dz, r2);
    float rinv = rsqrtf(r2);
    if (MASK) rinv = (sid == tid) ? 0.0f : rinv;
    const float mr = s.w * rinv;
    const float mr3 = mr * rinv * rinv;
    ph = ph - mr;
    ax = fmaf(mr3, dx, ax);
    ay = fmaf(mr3, dy, ay);
    az = fmaf(mr3, dz, az);
}

// Targets of one lane: two slots.  A group of c targets is spread over
// T2 = ceil(c/2) lanes (slot k of lane tl holds target tl + k*T2), and the
// S = floor(32/T2) copies of that layout each take every S-th list entry;
// the S partial sums of a target are added with shuffles at the end.  This
// keeps most lanes busy for the small groups that dominate real trees.
struct Targets {
    float x[2], y[2], z[2];
    float ax[2], ay[2], az[2], ph[2];
    int id[2];
};

__device__ __forceinline__ void eval_pc(const WarpLists &L, int j0, int cnt, int S, Targets &t,
                                        float eps2) {
#pragma unroll 2
    for (int j = j0; j < cnt; j += S) {
        const float4 a = L.ca[j], b = L.cb[j], c = L.cc[j];
#pragma unroll
        for (int k = 0; k < 2; ++k)
            pc_one(a, b, c, t.x[k], t.y[k], t.z[k], eps2, t.ax[k], t.ay[k], t.az[k], t.ph[k]);
    }
}

template <bool MASK>
__device__ __forceinline__ void eval_pp(const WarpLists &L, int j0, int cnt, int S, Targets &t,
                                        float eps2) {
#pragma unroll 2
    for (int j = j0; j < cnt; j += S) {
        const float4 p = L.pp[j];
        const int sid = L.pid[j];
#pragma unroll
        for (int k = 0; k < 2; ++k)
            pp_one<MASK>(p, sid, t.id[k], t.x[k], t.y[k], t.z[k], eps2, t.ax[k], t.ay[k], t.az[k],
                         t.ph[k]);
    }
}

// Sum the S partial results of a target into the lanes of the first copy.
__device__ __forceinline__ float sum_copies(float v, int lane, int T2, int S) {
    float r = v;
    for (int m = 1; m < S; ++m) r += __shfl_sync(0xffffffffu, v, min(lane + m * T2, 31));
    return r;
}

// MASK: skip the self pair inside the p-p loop (needed when eps = 0, or when
// theta >= 1/sqrt(3) so that a target's own leaf may be accepted as a cell).
// Otherwise every target meets itself exactly once in its p-p list: for
// theta < 1/sqrt(3) a cell containing the group is always opened (the
// distance from its com to the group box is at most sqrt(3) l < l/theta),
// and the self term is removed after the loop.
template <bool MASK>
__global__ void __launch_bounds__(WALK_WARPS * 32) k_walk(const WalkArgs A) {
    __shared__ WarpLists lists[WALK_WARPS];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    WarpLists &L = lists[wib];
    const uint32_t lt = lanemask_lt();
    const int64_t gw = (int64_t)blockIdx.x * WALK_WARPS + wib;
    uint32_t *fa = A.frontier + gw * 2 * FCAP;
    uint32_t *fb = fa + FCAP;
    const float eps2 = A.eps2;

    while (true) {
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(&A.sc->group_counter, 1u);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= A.ngroups) break;

        const uint32_t gf = A.gfirst[g], gc = A.gcount[g];
        const float4 box = A.gbox[g], half = A.ghalf[g], clo = A.glo[g];
        // lane layout: T2 lanes hold the targets, S copies split the sources
        const int T2 = (int)((gc + 1u) >> 1);
        const int S = 32 / T2;
        const int cp = lane / T2;            // this lane's copy
        const int tl = lane - cp * T2;       // this lane's target column
        const bool active = cp < S;
        Targets t;
        float self[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const uint32_t li = (uint32_t)(tl + k * T2);
            const bool v = active && li < gc;
            const int64_t i = gf + (v ? li : 0u);
            const float4 h = A.body_hi[i], l = A.body_lo[i];
            t.x[k] = (h.x - box.x) + (l.x - clo.x);
            t.y[k] = (h.y - box.y) + (l.y - clo.y);
            t.z[k] = (h.z - box.z) + (l.z - clo.z);
            t.id[k] = v ? (int)i : -1;
            t.ax[k] = t.ay[k] = t.az[k] = t.ph[k] = 0.0f;
            self[k] = h.w;
        }
        const int j0 = active ? cp : 1 << 30;  // first ring entry of this lane

        uint32_t pc_head = 0, pc_tail = 0, pp_head = 0, pp_tail = 0;
        uint32_t npc = 0, npp = 0;
        uint32_t *cur = fa, *nxt = fb;
        if (lane == 0) cur[0] = 0u;  // the root
        uint32_t ncur = 1;
        uint32_t maxf = 1;
        bool overflow = false;
        __syncwarp();

        while (ncur > 0) {
            uint32_t nnext = 0;
            for (uint32_t base = 0; base < ncur; base += 32) {
                const uint32_t idx = base + lane;
                const bool valid = idx < ncur;
                const uint32_t node = valid ? cur[idx] : 0u;
                const float4 m = A.mac[node];
                const uint2 tp = A.topo[node];
                // opening test: squared distance from com to the group box
                float dx = fmaxf(__fsub_rn(fabsf(__fsub_rn(m.x, box.x)), half.x), 0.0f);
                float dy = fmaxf(__fsub_rn(fabsf(__fsub_rn(m.y, box.y)), half.y), 0.0f);
                float dz = fmaxf(__fsub_rn(fabsf(__fsub_rn(m.z, box.z)), half.z), 0.0f);
                const float d2 =
                    __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                const bool open = d2 < m.w;
                const bool leaf = (tp.y & LEAF_FLAG) != 0u;
                const bool accept = valid && !open;

                // accepted cells -> p-c ring
                const uint32_t am = __ballot_sync(0xffffffffu, accept);
                if (accept) {
                    const uint32_t s = (pc_tail + __popc(am & lt)) & (RING - 1);
                    const float4 a = A.ca[node];
                    const float4 rel = make_float4((m.x - box.x) + (a.x - clo.x),
                                                   (m.y - box.y) + (a.y - clo.y),
                                                   (m.z - box.z) + (a.z - clo.z), a.w);
                    L.ca[s] = rel;
                    L.cb[s] = A.cb[node];
                    L.cc[s] = A.cc[node];
                }
                pc_tail += __popc(am);
                npc += __popc(am);

                // one warp scan for both the children of opened internal cells
                // (low 9 bits: at most 8 per lane) and the particles of opened
                // leaves (high bits); two scans when a leaf is very large
                const uint32_t nch = (valid && open && !leaf) ? tp.y : 0u;
                const uint32_t lc = (valid && open && leaf) ? (tp.y & ~LEAF_FLAG) : 0u;
                uint32_t noff, ntot, loff, ltot;
                if (__any_sync(0xffffffffu, lc > 4096u)) {
                    noff = warp_excl_scan(nch, ntot);
                    loff = warp_excl_scan(lc, ltot);
                } else {
                    uint32_t tot;
                    const uint32_t off = warp_excl_scan(nch | (lc << 9), tot);
                    noff = off & 511u;
                    ntot = tot & 511u;
                    loff = off >> 9;
                    ltot = tot >> 9;
                }
                // opened internal cells -> next frontier
                if (nnext + ntot > (uint32_t)FCAP) {
                    overflow = true;
                } else {
                    for (uint32_t k = 0; k < nch; ++k) nxt[nnext + noff + k] = tp.x + k;
                    nnext += ntot;
                }

                // opened leaves -> p-p ring, 32 particles per round
                npp += ltot;
                for (uint32_t r = 0; r < ltot; r += 32) {
                    const uint32_t k = r + lane;
                    // owner lane: the last lane whose offset is <= k
                    int src = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const uint32_t o = __shfl_sync(0xffffffffu, loff, src + step);
                        if (o <= k) src += step;
                    }
                    const uint32_t sfirst = __shfl_sync(0xffffffffu, tp.x, src);
                    const uint32_t soff = __shfl_sync(0xffffffffu, loff, src);
                    if (k < ltot) {
                        const uint32_t j = sfirst + (k - soff);
                        const float4 h = A.body_hi[j], l = A.body_lo[j];
                        const uint32_t s = (pp_tail + lane) & (RING - 1);
                        L.pp[s] = make_float4((h.x - box.x) + (l.x - clo.x),
                                              (h.y - box.y) + (l.y - clo.y),
                                              (h.z - box.z) + (l.z - clo.z), h.w);
                        L.pid[s] = (int)j;
                    }
                    pp_tail += min(32u, ltot - r);
                    __syncwarp();
                    if (pp_tail - pp_head >= 32u) {
                        // the head is a multiple of 32: the 32 entries do not wrap
                        const int hb = (int)(pp_head & (RING - 1));
                        eval_pp<MASK>(L, hb + j0, hb + 32, S, t, eps2);
                        pp_head += 32;
                        __syncwarp();
                    }
                }
                __syncwarp();
                while (pc_tail - pc_head >= 32u) {
                    const int hb = (int)(pc_head & (RING - 1));
                    eval_pc(L, hb + j0, hb + 32, S, t, eps2);
                    pc_head += 32;
                }
                __syncwarp();
            }
            __threadfence_block();
            __syncwarp();
            uint32_t *tmp = cur;
            cur = nxt;
            nxt = tmp;
            ncur = nnext;
            maxf = max(maxf, ncur);
        }
        // drain the rings: fewer than 32 entries each, starting at a multiple of 32
        {
            const int hb = (int)(pc_head & (RING - 1));
            eval_pc(L, hb + j0, hb + (int)(pc_tail - pc_head), S, t, eps2);
            const int hp = (int)(pp_head & (RING - 1));
            eval_pp<MASK>(L, hp + j0, hp + (int)(pp_tail - pp_head), S, t, eps2);
        }
        __syncwarp();

#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float ax = A.G * sum_copies(t.ax[k], lane, T2, S);
            const float ay = A.G * sum_copies(t.ay[k], lane, T2, S);
            const float az = A.G * sum_copies(t.az[k], lane, T2, S);
            float phs = sum_copies(t.ph[k], lane, T2, S);
            if (!MASK) phs = phs + self[k] * rsqrtf(eps2);  // remove the self pair
            const float ph = A.G * phs;
            const uint32_t li = (uint32_t)(tl + k * T2);
            if (cp == 0 && li < gc) {
                const int64_t i = gf + li;
                A.acc[i] = ax;
                A.acc[A.n + i] = ay;
                A.acc[2 * A.n + i] = az;
                A.pot[i] = ph;
                if (A.acc_c) {
                    const uint32_t o = A.id[i];
                    A.acc_c[o] = ax;
                    A.acc_c[A.n + o] = ay;
                    A.acc_c[2 * A.n + o] = az;
                }
                if (A.pot_c) A.pot_c[A.id[i]] = ph;
            }
        }
        if (lane == 0) {
            A.gnpp[g] = (int32_t)npp;
            A.gnpc[g] = (int32_t)npc;
            atomicAdd((unsigned long long *)&A.sc->n_pp, (unsigned long long)gc * npp);
            atomicAdd((unsigned long long *)&A.sc->n_pc, (unsigned long long)gc * npc);
            atomicMax(&A.sc->max_frontier, (int)maxf);
            if (overflow) atomicOr(&A.sc->status, ST_OVERFLOW);
        }
        __syncwarp();
    }
}

}  // namespace

int walk_resident_warps(bonsai_ctx *c) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk<true>, WALK_WARPS * 32, 0) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return per_sm * c->sm_count * WALK_WARPS;
}

size_t walk_frontier_elems(int warps) { return (size_t)warps * 2 * FCAP; }

int walk_force(bonsai_ctx *c, float theta, float eps, float *acc_c, float *pot_c) {
    const bool mask_self = !(eps > 0.0f) || !(theta < 0.57f);
    WalkArgs a;
    a.mac = c->cell_mac.p;
    a.topo = c->cell_topo.p;
    a.ca = c->cell_a.p;
    a.cb = c->cell_b.p;
    a.cc = c->cell_c.p;
    a.body_hi = c->body_hi.p;
    a.body_lo = c->body_lo.p;
    a.gfirst = c->grp_first.p;
    a.gcount = c->grp_count.p;
    a.gbox = c->grp_box.p;
    a.ghalf = c->grp_half.p;
    a.glo = c->grp_lo.p;
    a.ngroups = c->n_groups;
    a.n = c->n;
    a.eps2 = eps * eps;
    a.G = (float)c->prm.G;
    a.acc = c->acc.p;
    a.pot = c->pot.p;
    a.acc_c = acc_c;
    a.pot_c = pot_c;
    a.id = c->id.p;
    a.gnpp = c->grp_npp.p;
    a.gnpc = c->grp_npc.p;
    a.frontier = c->frontier.p;
    a.sc = c->dsc;
    const int blocks = c->walk_warps / WALK_WARPS;
    cudaEventRecord(c->ev[8], c->stream);
    if (mask_self)
        k_walk<true><<<blocks, WALK_WARPS * 32, 0, c->stream>>>(a);
    else
        k_walk<false><<<blocks, WALK_WARPS * 32, 0, c->stream>>>(a);
    cudaEventRecord(c->ev[9], c->stream);
    c->launches += 1;
    return cudaPeekAtLastError() == cudaSuccess ? BONSAI_OK : BONSAI_ECUDA;
}

}  // namespace bgb
