// walk.cu -- the fused group walk and force evaluation (Sec. III.A: the
// walk and the force computation in one kernel, interaction lists kept on
// chip and evaluated on the fly; Eq. 1-2 of Sec. VI.A), and its adjoint.
//
// One warp owns one group of <= 64 targets (or, at small N, one piece of a
// group's targets).  Warps fetch groups from a global counter, so the grid
// is persistent: one wave of resident warps.
// The walk is breadth-first: each lane tests one cell of the current
// frontier against the group's box (ballot + popc compaction replaces
// Bonsai's shared-memory stacks):
//   accepted          -> its multipole record is converted to group-relative
//                        FP32 and appended to the warp's p-c ring in smem;
//   opened leaf       -> its particles are appended to the p-p ring (a warp
//                        scan of the leaf sizes spreads them over lanes);
//   opened internal   -> its children go to the next frontier (global
//                        scratch, one region per resident warp, L2-resident).
// Whenever a ring holds 32 entries the warp evaluates them.  The list never
// reaches DRAM.  All force arithmetic is FP32 on coordinates relative to the
// group centre; the opening test is evaluated exactly as specified
// (round-to-nearest FP32, fixed order) so that the interaction lists are a
// pure function of the FP32-rounded cell and group data.
//
// The traversal is one template (walk_group) shared by two evaluation
// policies: the forward one (targets in lanes, list entries broadcast from
// shared memory; a lane's first two targets evaluated as one packed FP32
// pair, bit-identical to the scalar arithmetic) and the adjoint one (list
// entries in lanes, targets broadcast), which recomputes exactly the same
// lists.
#include "internal.cuh"
#include "packed.cuh"

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
    int pid[RING];    // sorted index of the particle
    int cid[RING];    // node index of the cell
    float4 gbox, ghalf, glo;  // the group's box, read from here rather than kept in registers
    uint2 tsel;               // first target and target count of the walk
};

// Targets of one group for the adjoint policy, two per record (targets 2p
// and 2p+1 in record p), so that one 16-byte shared load yields two packed
// operands.  Slots beyond the group copy target 0 with zero cotangents.
struct __align__(16) WarpTargets {
    float4 nxy[NCRIT / 2];  // {-x, -x', -y, -y'}: minus the group-relative position
    float4 nzi[NCRIT / 2];  // {-z, -z', sorted index (bits), sorted index' (bits)}
    float4 lxy[NCRIT / 2];  // {lambda_x, lambda_x', lambda_y, lambda_y'}
    float4 lzm[NCRIT / 2];  // {lambda_z, lambda_z', mu, mu'}
    float2 nmu[NCRIT / 2];  // {-mu, -mu'}
};

struct WalkArgs {
    const float4 *mac;
    const uint2 *topo;
    const float4 *ca, *cb, *cc;
    const float4 *body_hi, *body_lo;  // targets (the groups' particles)
    const float4 *src_hi, *src_lo;    // p-p sources (the tree's particles)
    const uint32_t *gfirst, *gcount;
    const uint32_t *gorder;  // forward and adjoint walks: the order of fetching groups (null: index order)
    const float4 *gbox, *ghalf, *glo;
    int64_t ngroups;
    int64_t n;
    float eps2;
    float G;
    // forward outputs
    float *acc;    // sorted [3][n]
    float *pot;    // sorted [n]
    float *acc_c;  // caller order [3][n] or null
    float *pot_c;  // caller order [n] or null
    int accumulate;  // add to acc/pot instead of writing them
    int parts;       // forward and adjoint walks: pieces each group's targets are split into (1-8)
    const uint32_t *id;
    int32_t *gnpp, *gnpc;
    // adjoint inputs / outputs (sorted order)
    const float *lam;  // [3][n]
    const float *mu;   // [n] or null
    float4 *cell_adj;  // [3][nn]: {gcom.xyz, gM}, {gQxx, gQyy, gQzz, gQxy}, {gQxz, gQyz, 0, 0}
    float4 *part_adj;  // [n]: {gx, gy, gz, gm}
    int64_t nn;
    uint32_t *frontier;
    uint32_t fcap;  // usable entries of each frontier buffer (<= FCAP)
    DevScalars *sc;
    // all-FP64 evaluation
    const double *pos64, *mass64;  // sorted [3][n], [n]
    const double *gcentre;         // [3][ngroups]
    const double *ndM, *ndcom, *ndQ;  // [nn], [3][nn], [6][nn]
    double *acc64, *pot64;         // caller order [3][n], [n] or null
    double G64, eps2_64;
    // list recording (parity tests): per-group offsets [ngroups + 1] and outputs
    const int64_t *lpc_off, *lpp_off;
    uint32_t *lpc_out, *lpp_out;
};

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// A shared-memory float4 read that the compiler may not hoist into registers.
__device__ __forceinline__ float4 lds_f4(const float4 *p) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
}

__device__ __forceinline__ uint2 lds_u2(const uint2 *p) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];"
                 : "=r"(v.x), "=r"(v.y)
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
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

// ---------------------------------------------------------------------------
// Forward evaluation
// ---------------------------------------------------------------------------

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

// pc_one and pp_one on the two targets of a packed pair: every packed
// operation is the scalar one on each half, in the same order, so the two
// targets get bit-identical results to the scalar code.  The potential is
// accumulated negated (phn = -phi): phn + u tp and phn + m/r round exactly as
// phi - u tp and phi - m/r do.
__device__ __forceinline__ void pc_two(const float4 a, const float4 b, const float4 c, f32x2 tx,
                                       f32x2 ty, f32x2 tz, f32x2 e2, f32x2 &ax, f32x2 &ay,
                                       f32x2 &az, f32x2 &phn) {
    const f32x2 rx = sub2(dup2(a.x), tx), ry = sub2(dup2(a.y), ty), rz = sub2(dup2(a.z), tz);
    f32x2 s2 = fma2(rx, rx, e2);
    s2 = fma2(ry, ry, s2);
    s2 = fma2(rz, rz, s2);
    float s0, s1;
    u2(s2, s0, s1);
    const f32x2 u = p2(rsqrtf(s0), rsqrtf(s1));
    const f32x2 w = mul2(u, u);
    const f32x2 bx = dup2(b.x), by = dup2(b.y), bz = dup2(b.z), bw = dup2(b.w);
    const f32x2 cx = dup2(c.x), cy = dup2(c.y);
    const f32x2 qx = fma2(bx, rx, fma2(bw, ry, mul2(cx, rz)));
    const f32x2 qy = fma2(bw, rx, fma2(by, ry, mul2(cy, rz)));
    const f32x2 qz = fma2(cx, rx, fma2(cy, ry, mul2(bz, rz)));
    const f32x2 q = mul2(fma2(rx, qx, fma2(ry, qy, mul2(rz, qz))), w);
    const f32x2 M = dup2(a.w);
    const f32x2 tp = fma2(w, fma2(dup2(-0.5f), q, dup2(c.z)), M);
    phn = fma2(u, tp, phn);
    const f32x2 uw = mul2(u, w);
    const f32x2 A = mul2(uw, fma2(w, fma2(dup2(-2.5f), q, dup2(c.w)), M));
    const f32x2 B = mul2(uw, w);
    ax = fma2(A, rx, ax);
    ay = fma2(A, ry, ay);
    az = fma2(A, rz, az);
    ax = fma2(B, qx, ax);
    ay = fma2(B, qy, ay);
    az = fma2(B, qz, az);
}

template <bool MASK>
__device__ __forceinline__ void pp_two(const float4 s, int sid, int id0, int id1, f32x2 tx,
                                       f32x2 ty, f32x2 tz, f32x2 e2, f32x2 &ax, f32x2 &ay,
                                       f32x2 &az, f32x2 &phn) {
    const f32x2 dx = sub2(dup2(s.x), tx), dy = sub2(dup2(s.y), ty), dz = sub2(dup2(s.z), tz);
    f32x2 r2 = fma2(dx, dx, e2);
    r2 = fma2(dy, dy, r2);
    r2 = fma2(dz, dz, r2);
    float r0, r1;
    u2(r2, r0, r1);
    float i0 = rsqrtf(r0), i1 = rsqrtf(r1);
    if (MASK) {
        i0 = (sid == id0) ? 0.0f : i0;
        i1 = (sid == id1) ? 0.0f : i1;
    }
    const f32x2 rinv = p2(i0, i1);
    const f32x2 mr = mul2(dup2(s.w), rinv);
    const f32x2 mr3 = mul2(mul2(mr, rinv), rinv);
    phn = add2(phn, mr);
    ax = fma2(mr3, dx, ax);
    ay = fma2(mr3, dy, ay);
    az = fma2(mr3, dz, az);
}

// Targets of one lane: K = 2 or 3 slots, chosen per group.  A group of c
// targets is spread over T = ceil(c/K) lanes (slot k of lane tl holds
// target tl + k*T), and the S = floor(32/T) copies of that layout each
// take every S-th list entry; the S partial sums of a target are added with
// shuffles at the end.  K is the one of 2 and 3 that keeps more of the
// warp's target slots busy (c S / (32 K)): groups of 33-48 targets use 48 of
// 64 slots or fewer with two slots per lane, and up to 96 of 96 with three.
constexpr int KMAX = 3;
struct Targets {
    float x[KMAX], y[KMAX], z[KMAX];
    float ax[KMAX], ay[KMAX], az[KMAX], ph[KMAX];
    int id[KMAX];
};

// Sum the S partial results of a target into the lanes of the first copy.
__device__ __forceinline__ float sum_copies(float v, int lane, int T, int S) {
    float r = v;
    for (int m = 1; m < S; ++m) r += __shfl_sync(0xffffffffu, v, min(lane + m * T, 31));
    return r;
}

// Slots per lane for a group of c targets: 3 when that fills more slots.
__device__ __forceinline__ int slots_for(uint32_t c) {
    const uint32_t t2 = (c + 1u) >> 1, t3 = (c + 2u) / 3u;
    const uint32_t s2 = 32u / t2, s3 = 32u / t3;
    return (2u * s3 > 3u * s2) ? 3 : 2;  // c s3 / 96 > c s2 / 64
}

// Self pairs.  SELF_MASK: skip the self pair inside the p-p loop (needed when
// eps = 0, or when theta >= 1/sqrt(3) so that a target's own leaf may be
// accepted as a cell).  SELF_SUB: every target meets itself exactly once in
// its p-p list: for theta < 1/sqrt(3) a cell containing the group is always
// opened (the distance from its com to the group box is at most
// sqrt(3) l < l/theta), and the self term is removed after the loop.
// SELF_NONE: targets and sources are disjoint sets (a remote domain's
// local essential tree).
constexpr int SELF_SUB = 0, SELF_MASK = 1, SELF_NONE = 2;
// Ring appends of the FP32 policies: a cell's com relative to the group
// centre is (com_hi - c_hi) + (com_lo - c_lo), each difference rounded once,
// so the FP32 record is accurate relative to the separation.
struct Fp32Rings {
    __device__ __forceinline__ void append_cell(const WalkArgs &A, WarpLists &L, uint32_t s,
                                                uint32_t node, float4 m, float4 box, float4 clo,
                                                uint32_t) {
        const float4 a = A.ca[node];
        L.ca[s] = make_float4((m.x - box.x) + (a.x - clo.x), (m.y - box.y) + (a.y - clo.y),
                              (m.z - box.z) + (a.z - clo.z), a.w);
        L.cb[s] = A.cb[node];
        L.cc[s] = A.cc[node];
        L.cid[s] = (int)node;
    }
    __device__ __forceinline__ void append_particle(const WalkArgs &A, WarpLists &L, uint32_t s,
                                                    uint32_t j, float4 box, float4 clo, uint32_t) {
        const float4 h = A.src_hi[j], l = A.src_lo[j];
        L.pp[s] = make_float4((h.x - box.x) + (l.x - clo.x), (h.y - box.y) + (l.y - clo.y),
                              (h.z - box.z) + (l.z - clo.z), h.w);
        L.pid[s] = (int)j;
    }
};

template <int SELF>
struct ForwardPolicy : Fp32Rings {
    int K, T, S, cp, tl, j0;
    Targets t;  // slots 0 and 1 live packed in the pair below during the walk
    f32x2 x01, y01, z01, ax01, ay01, az01, phn01, e2;
    float self[KMAX];
    float eps2;

    __device__ __forceinline__ void begin(const WalkArgs &A, WarpTargets *, uint32_t, uint32_t gf,
                                          uint32_t gc, float4 box, float4 clo, int lane) {
        eps2 = A.eps2;
        K = slots_for(gc);
        T = (int)((gc + (uint32_t)K - 1u) / (uint32_t)K);
        S = 32 / T;
        cp = lane / T;
        tl = lane - cp * T;
        const bool active = cp < S;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const uint32_t li = (uint32_t)(tl + k * T);
            const bool v = active && k < K && li < gc;
            const int64_t i = gf + (v ? li : 0u);
            const float4 h = A.body_hi[i], l = A.body_lo[i];
            t.x[k] = (h.x - box.x) + (l.x - clo.x);
            t.y[k] = (h.y - box.y) + (l.y - clo.y);
            t.z[k] = (h.z - box.z) + (l.z - clo.z);
            t.id[k] = v ? (int)i : -1;
            t.ax[k] = t.ay[k] = t.az[k] = t.ph[k] = 0.0f;
            self[k] = h.w;
        }
        j0 = active ? cp : 1 << 30;  // first ring entry of this lane
        x01 = p2(t.x[0], t.x[1]);
        y01 = p2(t.y[0], t.y[1]);
        z01 = p2(t.z[0], t.z[1]);
        ax01 = ay01 = az01 = phn01 = 0ull;
        e2 = dup2(eps2);
    }

    // entries [hb, hb + cnt) of the p-c ring (hb a multiple of 32, cnt <= 32)
    __device__ __forceinline__ void flush_pc(const WarpLists &L, int hb, int cnt) {
        const int end = hb + cnt;
        if (K == 2) {
#pragma unroll 1
            for (int j = hb + j0; j < end; j += S) {
                const float4 a = L.ca[j], b = L.cb[j], c = L.cc[j];
                pc_two(a, b, c, x01, y01, z01, e2, ax01, ay01, az01, phn01);
            }
        } else {
#pragma unroll 1
            for (int j = hb + j0; j < end; j += S) {
                const float4 a = L.ca[j], b = L.cb[j], c = L.cc[j];
                pc_two(a, b, c, x01, y01, z01, e2, ax01, ay01, az01, phn01);
                pc_one(a, b, c, t.x[2], t.y[2], t.z[2], eps2, t.ax[2], t.ay[2], t.az[2], t.ph[2]);
            }
        }
    }

    __device__ __forceinline__ void flush_pp(const WarpLists &L, int hb, int cnt) {
        const int end = hb + cnt;
        if (K == 2) {
#pragma unroll 1
            for (int j = hb + j0; j < end; j += S) {
                const float4 p = L.pp[j];
                const int sid = L.pid[j];
                pp_two<SELF == SELF_MASK>(p, sid, t.id[0], t.id[1], x01, y01, z01, e2, ax01, ay01,
                                          az01, phn01);
            }
        } else {
#pragma unroll 1
            for (int j = hb + j0; j < end; j += S) {
                const float4 p = L.pp[j];
                const int sid = L.pid[j];
                pp_two<SELF == SELF_MASK>(p, sid, t.id[0], t.id[1], x01, y01, z01, e2, ax01, ay01,
                                          az01, phn01);
                pp_one<SELF == SELF_MASK>(p, sid, t.id[2], t.x[2], t.y[2], t.z[2], eps2, t.ax[2],
                                          t.ay[2], t.az[2], t.ph[2]);
            }
        }
    }

    __device__ __forceinline__ void finish(const WalkArgs &A, uint32_t gf, uint32_t gc, int lane) {
        u2(ax01, t.ax[0], t.ax[1]);
        u2(ay01, t.ay[0], t.ay[1]);
        u2(az01, t.az[0], t.az[1]);
        u2(phn01, t.ph[0], t.ph[1]);
        t.ph[0] = -t.ph[0];
        t.ph[1] = -t.ph[1];
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (k >= K) break;
            const float ax = A.G * sum_copies(t.ax[k], lane, T, S);
            const float ay = A.G * sum_copies(t.ay[k], lane, T, S);
            const float az = A.G * sum_copies(t.az[k], lane, T, S);
            float phs = sum_copies(t.ph[k], lane, T, S);
            if (SELF == SELF_SUB) phs = phs + self[k] * rsqrtf(eps2);  // remove the self pair
            const float ph = A.G * phs;
            const uint32_t li = (uint32_t)(tl + k * T);
            if (cp == 0 && li < gc) {
                const int64_t i = gf + li;
                if (A.accumulate) {
                    A.acc[i] += ax;
                    A.acc[A.n + i] += ay;
                    A.acc[2 * A.n + i] += az;
                    A.pot[i] += ph;
                    continue;
                }
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
    }
};

// ---------------------------------------------------------------------------
// Adjoint evaluation
// ---------------------------------------------------------------------------

// The adjoint evaluates two targets per packed FP32 operation (packed.cuh).
__device__ __forceinline__ ulonglong2 lds2(const float4 &v) {
    return *reinterpret_cast<const ulonglong2 *>(&v);
}

// One list entry (in both halves) and two targets.
struct TargetPair {
    f32x2 nx, ny, nz;  // minus the target positions
    f32x2 lx, ly, lz, mu, nmu;  // lambda, mu, -mu
    int2 id;           // sorted indices
};

// Gradient of lambda.a + mu phi for one cell on two targets (without G),
// with respect to r = com - x_i (g_r), the cell mass (gM) and the symmetric
// quadrupole Q.  With u = 1/s, w = u^2, Q' = -3Q (as stored), rq = r.Q'r,
// lq = lambda.Q'r, lr = lambda.r, z = w rq:
//   alpha = u^3 (M + w (c.w - 5/2 z))            (c.w = -3/2 trQ)
//   K     = u^5 (-3M + w (-5 c.w + 35/2 z))
//   gam   = mu u^5 - 5 u^7 lr
//   beta  = lr K + mu alpha - 5 u^7 lq
//   g_r   = alpha lambda + beta r + gam Q'r + u^5 Q'lambda
//   gM    = lr u^3 - mu u
//   gQ    = P0 I + (r v2^T + v2 r^T) / 2,  P0 = mu u^3 / 2 - 3/2 u^5 lr,
//           v2 = (15/2 u^7 lr - 3/2 mu u^5) r - 3 u^5 lambda = -3/2 vq,
//           vq = gam r + 2 u^5 lambda.
// The caller accumulates mu u^3 and u^5 lr (for P0) and r vq^T (for gQ)
// and applies the constant factors once per cell.  The cell record (both
// halves equal): a = {com, M}, b, c as stored, M3 = -3M, cw5 = -5 c.w.
struct CellDup {
    f32x2 x, y, z, M, bx, by, bz, bw, cx, cy, cw, M3, cw5;
};

// u = 1/s of one cell and two targets (the first, latency-bound part of the
// p-c VJP, taken for a whole chunk before the rest).
__device__ __forceinline__ f32x2 pc_inv_s(const CellDup &C, f32x2 nx, f32x2 ny, f32x2 nz,
                                          f32x2 eps2, f32x2 &rx, f32x2 &ry, f32x2 &rz) {
    rx = add2(C.x, nx);
    ry = add2(C.y, ny);
    rz = add2(C.z, nz);
    f32x2 s2 = fma2(rx, rx, eps2);
    s2 = fma2(ry, ry, s2);
    s2 = fma2(rz, rz, s2);
    float s0, s1;
    u2(s2, s0, s1);
    return p2(rsqrtf(s0), rsqrtf(s1));
}

template <bool GIVEN_U>
__device__ __forceinline__ void pc_vjp2(const CellDup &C, const TargetPair &T, f32x2 eps2,
                                        f32x2 ug, f32x2 &gx, f32x2 &gy, f32x2 &gz, f32x2 &gM,
                                        f32x2 &u3, f32x2 &u5, f32x2 &lr, f32x2 &vx, f32x2 &vy,
                                        f32x2 &vz, f32x2 &rx, f32x2 &ry, f32x2 &rz) {
    const f32x2 k_m25 = dup2(-2.5f), k_175 = dup2(17.5f), k_m5 = dup2(-5.0f);
    // with GIVEN_U the caller passes u and r = com - x (rx, ry, rz) of the
    // first phase; otherwise both are computed here
    const f32x2 u = GIVEN_U ? ug : pc_inv_s(C, T.nx, T.ny, T.nz, eps2, rx, ry, rz);
    const f32x2 w = mul2(u, u);
    u3 = mul2(u, w);
    u5 = mul2(u3, w);
    const f32x2 qx = fma2(C.bx, rx, fma2(C.bw, ry, mul2(C.cx, rz)));  // Q'r
    const f32x2 qy = fma2(C.bw, rx, fma2(C.by, ry, mul2(C.cy, rz)));
    const f32x2 qz = fma2(C.cx, rx, fma2(C.cy, ry, mul2(C.bz, rz)));
    const f32x2 px = fma2(C.bx, T.lx, fma2(C.bw, T.ly, mul2(C.cx, T.lz)));  // Q'lambda
    const f32x2 py = fma2(C.bw, T.lx, fma2(C.by, T.ly, mul2(C.cy, T.lz)));
    const f32x2 pz = fma2(C.cx, T.lx, fma2(C.cy, T.ly, mul2(C.bz, T.lz)));
    const f32x2 rq = fma2(rx, qx, fma2(ry, qy, mul2(rz, qz)));
    const f32x2 lq = fma2(T.lx, qx, fma2(T.ly, qy, mul2(T.lz, qz)));
    lr = fma2(T.lx, rx, fma2(T.ly, ry, mul2(T.lz, rz)));
    const f32x2 z = mul2(w, rq);
    const f32x2 alpha = mul2(u3, fma2(w, fma2(k_m25, z, C.cw), C.M));
    const f32x2 K = mul2(u5, fma2(w, fma2(k_175, z, C.cw5), C.M3));
    const f32x2 c5 = mul2(mul2(k_m5, w), u5);  // -5 u^7
    const f32x2 beta = fma2(lr, K, fma2(T.mu, alpha, mul2(c5, lq)));
    const f32x2 gam = fma2(T.mu, u5, mul2(c5, lr));
    gx = fma2(alpha, T.lx, fma2(beta, rx, fma2(gam, qx, mul2(u5, px))));
    gy = fma2(alpha, T.ly, fma2(beta, ry, fma2(gam, qy, mul2(u5, py))));
    gz = fma2(alpha, T.lz, fma2(beta, rz, fma2(gam, qz, mul2(u5, pz))));
    gM = fma2(lr, u3, mul2(T.nmu, u));
    const f32x2 u5x2 = add2(u5, u5);
    vx = fma2(gam, rx, mul2(u5x2, T.lx));
    vy = fma2(gam, ry, mul2(u5x2, T.ly));
    vz = fma2(gam, rz, mul2(u5x2, T.lz));
}

// Gradient of lambda.a + mu phi for one p-p source on two targets (without G):
//   g_r = m u^3 (lambda + (mu - 3 w lr) r),  gm = lr u^3 - mu u;
// zero for the self pair (u is set to 0, which also avoids r = 0 at eps = 0).
__device__ __forceinline__ f32x2 pp_inv_s(f32x2 sx, f32x2 sy, f32x2 sz, int sid, f32x2 nx,
                                          f32x2 ny, f32x2 nz, int2 id, f32x2 eps2, f32x2 &rx,
                                          f32x2 &ry, f32x2 &rz) {
    rx = add2(sx, nx);
    ry = add2(sy, ny);
    rz = add2(sz, nz);
    f32x2 s2 = fma2(rx, rx, eps2);
    s2 = fma2(ry, ry, s2);
    s2 = fma2(rz, rz, s2);
    float s0, s1;
    u2(s2, s0, s1);
    return p2(sid == id.x ? 0.0f : rsqrtf(s0), sid == id.y ? 0.0f : rsqrtf(s1));
}

template <bool GIVEN_U>
__device__ __forceinline__ void pp_vjp2(f32x2 sx, f32x2 sy, f32x2 sz, f32x2 sm, int sid,
                                        const TargetPair &T, f32x2 eps2, f32x2 ug, f32x2 rx,
                                        f32x2 ry, f32x2 rz, f32x2 &gx, f32x2 &gy, f32x2 &gz,
                                        f32x2 &gm) {
    // with GIVEN_U the caller passes u and r of the first phase
    const f32x2 u = GIVEN_U ? ug : pp_inv_s(sx, sy, sz, sid, T.nx, T.ny, T.nz, T.id, eps2, rx, ry, rz);
    const f32x2 w = mul2(u, u);
    const f32x2 u3 = mul2(u, w);
    const f32x2 lr = fma2(T.lx, rx, fma2(T.ly, ry, mul2(T.lz, rz)));
    const f32x2 co = fma2(mul2(dup2(-3.0f), w), lr, T.mu);
    const f32x2 k = mul2(sm, u3);
    gx = mul2(k, fma2(co, rx, T.lx));
    gy = mul2(k, fma2(co, ry, T.ly));
    gz = mul2(k, fma2(co, rz, T.lz));
    gm = fma2(lr, u3, mul2(T.nmu, u));
}

__device__ __forceinline__ TargetPair load_targets(const WarpTargets *T, int p) {
    const ulonglong2 a = lds2(T->nxy[p]), b = lds2(T->nzi[p]), c = lds2(T->lxy[p]);
    const ulonglong2 d = lds2(T->lzm[p]);
    const f32x2 e = *reinterpret_cast<const f32x2 *>(&T->nmu[p]);
    float i0, i1;
    u2(b.y, i0, i1);
    return TargetPair{a.x, a.y, b.x, c.x, c.y, d.x, d.y, e,
                      make_int2(__float_as_int(i0), __float_as_int(i1))};
}

// Per-warp scratch of the adjoint: a 32 x 24 transpose buffer for the target
// gradients of a chunk of 8 targets, and the running target gradients.  A
// lane's row holds, per target pair tp, {gx, gy, gz} as packed pairs
// (x0 x1 y0 y1 z0 z1 at 6 tp); 26-float rows make the 8-byte row stores of a
// half-warp and the column reads conflict-free.
constexpr int ADJ_CHUNK = 8;
constexpr int ADJ_ROW = 3 * ADJ_CHUNK + 2;
struct __align__(16) WarpAdjoint {
    float red[32 * ADJ_ROW];
    float tacc[NCRIT * 3];
};

// The adjoint evaluates each ring flush with one list entry per lane and a
// loop over the group's targets (broadcast from shared memory), two targets
// per packed FP32 operation.  The cell or source adjoint stays in the lane's
// registers (packed: one half per target parity, added at the end).  The 3-vector target
// gradients of 8 targets at a time are transposed through shared memory and
// each column summed by one lane (24 lanes, 32 rows), which costs far fewer
// instructions than a shuffle reduction per target.  Every lane is busy
// whatever the group size.  Source and cell adjoints go to global memory with
// one vector atomic per 4 values per flush; target gradients once per group.
struct AdjointPolicy : Fp32Rings {
    WarpTargets *T;
    WarpAdjoint *W;
    int gc;
    float eps2, G;
    float4 *cell_adj;
    float4 *part_adj;
    int64_t nn;

    __device__ __forceinline__ void begin(const WalkArgs &A, WarpTargets *tgt, uint32_t,
                                          uint32_t gf, uint32_t gcount, float4 box, float4 clo,
                                          int lane) {
        T = tgt;
        gc = (int)gcount;
        eps2 = A.eps2;
        G = A.G;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            // slots beyond the group: target 0's position and index, zero
            // cotangents, so that every term they produce is exactly zero
            const int li = lane + 32 * k;
            const bool v = li < gc;
            const int64_t i = gf + (v ? li : 0);
            const float4 h = A.body_hi[i], l = A.body_lo[i];
            const float lx = v ? A.lam[i] : 0.0f, ly = v ? A.lam[A.n + i] : 0.0f;
            const float lz = v ? A.lam[2 * A.n + i] : 0.0f;
            const float mu = (v && A.mu) ? A.mu[i] : 0.0f;
            float *rec = reinterpret_cast<float *>(T) + (li >> 1) * 4 + (li & 1);
            constexpr int K = 4 * (NCRIT / 2);  // floats per array
            rec[0] = -((h.x - box.x) + (l.x - clo.x));
            rec[2] = -((h.y - box.y) + (l.y - clo.y));
            rec[K] = -((h.z - box.z) + (l.z - clo.z));
            rec[K + 2] = __int_as_float((int)i);
            rec[2 * K] = lx;
            rec[2 * K + 2] = ly;
            rec[3 * K] = lz;
            rec[3 * K + 2] = mu;
            reinterpret_cast<float *>(T->nmu)[(li >> 1) * 2 + (li & 1)] = -mu;
        }
        for (int k = lane; k < NCRIT * 3; k += 32) W->tacc[k] = 0.0f;
        __syncwarp();
    }

    // this lane's gradients of target pair tp of the chunk into its row
    __device__ __forceinline__ void put_pair(int tp, f32x2 gx, f32x2 gy, f32x2 gz, int lane) {
        f32x2 *row = reinterpret_cast<f32x2 *>(&W->red[lane * ADJ_ROW + 6 * tp]);
        row[0] = gx;
        row[1] = gy;
        row[2] = gz;
    }

    // add the chunk's target gradients (all rows) to tacc.  A row holds, as
    // packed pairs, column c = 3 tp + component for target pair tp (its two
    // halves are targets t0 + 2 tp and t0 + 2 tp + 1); a chunk of NP pairs
    // fills the first 3 NP columns.  Lane c of each half-warp sums column c
    // over 16 rows with packed adds (half h takes rows 16 h .. 16 h + 15, so
    // each half-warp reads 12 consecutive pairs of one row: no bank
    // conflict), and one 64-bit shuffle adds the two halves.
    template <int NP>
    __device__ __forceinline__ void reduce_chunk(int t0, int lane) {
        __syncwarp();
        const int h = lane >> 4, c = lane & 15;
        f32x2 s = 0ull;
        if (c < 3 * NP) {
            const f32x2 *col = reinterpret_cast<const f32x2 *>(W->red) + (16 * h) * (ADJ_ROW / 2) + c;
            f32x2 a[4];  // four short chains
#pragma unroll
            for (int k = 0; k < 4; ++k) a[k] = col[k * (ADJ_ROW / 2)];
#pragma unroll
            for (int r = 4; r < 16; r += 4)
#pragma unroll
                for (int k = 0; k < 4; ++k) a[k] = add2(a[k], col[(r + k) * (ADJ_ROW / 2)]);
            s = add2(add2(a[0], a[1]), add2(a[2], a[3]));
        }
        s = add2(s, __shfl_down_sync(0xffffffffu, s, 16));
        if (h == 0 && c < 3 * NP) {
            float lo, hi;
            u2(s, lo, hi);
            const int tp = c / 3, comp = c - 3 * tp;
            const int t = t0 + 2 * tp;
            if (t < gc) W->tacc[3 * t + comp] += lo;
            if (t + 1 < gc) W->tacc[3 * (t + 1) + comp] += hi;
        }
        __syncwarp();
    }

    // Running cell adjoint of one lane (packed: one half per target parity):
    // g_com, gM, sum mu u^3, sum u^5 lr, and sum r vq^T (diagonal, symmetric
    // off-diagonal pairs).
    struct PcAcc {
        f32x2 ax = 0ull, ay = 0ull, az = 0ull, aM = 0ull, aP1 = 0ull, aP2 = 0ull;
        f32x2 dxx = 0ull, dyy = 0ull, dzz = 0ull, oxy = 0ull, oxz = 0ull, oyz = 0ull;
    };

    // Target pair tp of the chunk at t0 into the cell adjoint and the row.
    template <bool GIVEN_U>
    __device__ __forceinline__ void pc_pair(const CellDup &C, f32x2 e2, int t0, int tp, int lane,
                                            PcAcc &S, f32x2 ug = 0ull, f32x2 rx = 0ull,
                                            f32x2 ry = 0ull, f32x2 rz = 0ull) {
        const TargetPair T2 = load_targets(T, (t0 >> 1) + tp);
        f32x2 gx, gy, gz, gM, u3, u5, lr, vx, vy, vz;
        pc_vjp2<GIVEN_U>(C, T2, e2, ug, gx, gy, gz, gM, u3, u5, lr, vx, vy, vz, rx, ry, rz);
        S.ax = add2(S.ax, gx);
        S.ay = add2(S.ay, gy);
        S.az = add2(S.az, gz);
        S.aM = add2(S.aM, gM);
        S.aP1 = fma2(T2.mu, u3, S.aP1);
        S.aP2 = fma2(u5, lr, S.aP2);
        S.dxx = fma2(rx, vx, S.dxx);
        S.dyy = fma2(ry, vy, S.dyy);
        S.dzz = fma2(rz, vz, S.dzz);
        S.oxy = fma2(rx, vy, fma2(ry, vx, S.oxy));
        S.oxz = fma2(rx, vz, fma2(rz, vx, S.oxz));
        S.oyz = fma2(ry, vz, fma2(rz, vy, S.oyz));
        put_pair(tp, gx, gy, gz, lane);
    }

    // Full chunks of 8 targets, then a last chunk of as many target pairs as
    // the group has left (slots past the group hold zero cotangents; columns
    // of the transpose rows past it belong to targets >= gc and are skipped).
    template <bool FULL>
    __device__ __forceinline__ void flush_pc(const WarpLists &L, int hb, int cnt, int lane) {
        const bool v = FULL || lane < cnt;
        const int j = hb + (v ? lane : 0);
        const float4 a = L.ca[j];
        float4 b = L.cb[j], c = L.cc[j];
        float M = a.w;
        if (!FULL && !v) {  // an empty lane: a massless, quadrupole-free cell
            M = 0.0f;
            b = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            c = b;
        }
        const CellDup C{dup2(a.x), dup2(a.y), dup2(a.z), dup2(M), dup2(b.x), dup2(b.y),
                        dup2(b.z), dup2(b.w), dup2(c.x), dup2(c.y), dup2(c.w),
                        dup2(-3.0f * M), dup2(-5.0f * c.w)};
        const f32x2 e2 = dup2(eps2);
        PcAcc S;
        int t0 = 0;
        for (; t0 + ADJ_CHUNK <= gc; t0 += ADJ_CHUNK) {
            // the chunk's four reciprocal distances first: their MUFU
            // latencies overlap instead of heading four dependent chains
            f32x2 uu[ADJ_CHUNK / 2], rr[ADJ_CHUNK / 2][3];
#pragma unroll
            for (int tp = 0; tp < ADJ_CHUNK / 2; ++tp) {
                const int p = (t0 >> 1) + tp;
                const ulonglong2 a = lds2(T->nxy[p]), b = lds2(T->nzi[p]);
                uu[tp] = pc_inv_s(C, a.x, a.y, b.x, e2, rr[tp][0], rr[tp][1], rr[tp][2]);
            }
#pragma unroll
            for (int tp = 0; tp < ADJ_CHUNK / 2; ++tp)
                pc_pair<true>(C, e2, t0, tp, lane, S, uu[tp], rr[tp][0], rr[tp][1], rr[tp][2]);
            reduce_chunk<ADJ_CHUNK / 2>(t0, lane);
        }
        const int np = (gc - t0 + 1) >> 1;  // one code copy for the ragged tail
        if (np > 0) {
#pragma unroll 1
            for (int tp = 0; tp < np; ++tp) pc_pair<false>(C, e2, t0, tp, lane, S);
            reduce_chunk<ADJ_CHUNK / 2>(t0, lane);
        }
        if (v) {
            // gQ = P0 I + (r v2^T + v2 r^T) / 2 with v2 = -3/2 vq: diagonal
            // P0 - 3/2 r_a vq_a, off-diagonal -3/4 (r_a vq_b + r_b vq_a)
            const float P = 0.5f * fold(S.aP1) - 1.5f * fold(S.aP2);
            const float aQ[6] = {P - 1.5f * fold(S.dxx), P - 1.5f * fold(S.dyy),
                                 P - 1.5f * fold(S.dzz), -0.75f * fold(S.oxy),
                                 -0.75f * fold(S.oxz), -0.75f * fold(S.oyz)};
            cell_add(L.cid[j], fold(S.ax), fold(S.ay), fold(S.az), fold(S.aM), aQ);
        }
    }

    // the sum of the two halves
    __device__ __forceinline__ static float fold(f32x2 v) {
        float a, b;
        u2(v, a, b);
        return a + b;
    }

    __device__ __forceinline__ void cell_add(int node, float ax, float ay, float az, float aM,
                                             const float aQ[6]) {
        atomicAdd(&cell_adj[node], make_float4(G * ax, G * ay, G * az, G * aM));
        atomicAdd(&cell_adj[nn + node], make_float4(G * aQ[0], G * aQ[1], G * aQ[2], G * aQ[3]));
        atomicAdd(&cell_adj[2 * nn + node], make_float4(G * aQ[4], G * aQ[5], 0.0f, 0.0f));
    }

    template <bool GIVEN_U>
    __device__ __forceinline__ void pp_pair(f32x2 sx, f32x2 sy, f32x2 sz, f32x2 sm, int sid,
                                            f32x2 e2, int t0, int tp, int lane, f32x2 &ax,
                                            f32x2 &ay, f32x2 &az, f32x2 &am, f32x2 ug = 0ull,
                                            f32x2 rx = 0ull, f32x2 ry = 0ull, f32x2 rz = 0ull) {
        const TargetPair T2 = load_targets(T, (t0 >> 1) + tp);
        f32x2 gx, gy, gz, gm;
        pp_vjp2<GIVEN_U>(sx, sy, sz, sm, sid, T2, e2, ug, rx, ry, rz, gx, gy, gz, gm);
        ax = add2(ax, gx);
        ay = add2(ay, gy);
        az = add2(az, gz);
        am = add2(am, gm);
        put_pair(tp, gx, gy, gz, lane);
    }

    template <bool FULL>
    __device__ __forceinline__ void flush_pp(const WarpLists &L, int hb, int cnt, int lane) {
        const bool v = FULL || lane < cnt;
        const int j = hb + (v ? lane : 0);
        float4 s = L.pp[j];
        if (!FULL && !v) s.w = 0.0f;  // an empty lane: a massless source
        const int sid = L.pid[j];
        const f32x2 sx = dup2(s.x), sy = dup2(s.y), sz = dup2(s.z), sm = dup2(s.w);
        const f32x2 e2 = dup2(eps2);
        f32x2 ax = 0ull, ay = 0ull, az = 0ull, am = 0ull;
        int t0 = 0;
        for (; t0 + ADJ_CHUNK <= gc; t0 += ADJ_CHUNK) {
            f32x2 uu[ADJ_CHUNK / 2], rr[ADJ_CHUNK / 2][3];  // reciprocal distances first, as for p-c
#pragma unroll
            for (int tp = 0; tp < ADJ_CHUNK / 2; ++tp) {
                const int p = (t0 >> 1) + tp;
                const ulonglong2 a = lds2(T->nxy[p]), b = lds2(T->nzi[p]);
                float i0, i1;
                u2(b.y, i0, i1);
                uu[tp] = pp_inv_s(sx, sy, sz, sid, a.x, a.y, b.x,
                                  make_int2(__float_as_int(i0), __float_as_int(i1)), e2, rr[tp][0],
                                  rr[tp][1], rr[tp][2]);
            }
#pragma unroll
            for (int tp = 0; tp < ADJ_CHUNK / 2; ++tp)
                pp_pair<true>(sx, sy, sz, sm, sid, e2, t0, tp, lane, ax, ay, az, am, uu[tp], rr[tp][0],
                              rr[tp][1], rr[tp][2]);
            reduce_chunk<ADJ_CHUNK / 2>(t0, lane);
        }
        const int np = (gc - t0 + 1) >> 1;
        if (np > 0) {
#pragma unroll 1
            for (int tp = 0; tp < np; ++tp)
                pp_pair<false>(sx, sy, sz, sm, sid, e2, t0, tp, lane, ax, ay, az, am);
            reduce_chunk<ADJ_CHUNK / 2>(t0, lane);
        }
        if (v) atomicAdd(&part_adj[sid], make_float4(G * fold(ax), G * fold(ay), G * fold(az),
                                                     G * fold(am)));
    }

    __device__ __forceinline__ void finish(const WalkArgs &A, uint32_t gf, uint32_t gcount, int lane) {
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int li = lane + 32 * k;
            if (li < gc)
                atomicAdd(&part_adj[gf + li],
                          make_float4(-G * W->tacc[3 * li], -G * W->tacc[3 * li + 1],
                                      -G * W->tacc[3 * li + 2], 0.0f));
        }
        __syncwarp();
    }
};

// Forward and adjoint policies take the lane for their flushes differently.
template <class P>
__device__ __forceinline__ void do_flush_pc(P &pol, const WarpLists &L, int hb, int cnt, int lane);
template <int SELF>
__device__ __forceinline__ void do_flush_pc(ForwardPolicy<SELF> &pol, const WarpLists &L, int hb,
                                            int cnt, int) {
    pol.flush_pc(L, hb, cnt);
}
__device__ __forceinline__ void do_flush_pc(AdjointPolicy &pol, const WarpLists &L, int hb, int cnt,
                                            int lane) {
    if (cnt >= 32) pol.flush_pc<true>(L, hb, 32, lane);
    else if (cnt > 0) pol.flush_pc<false>(L, hb, cnt, lane);
}
template <int SELF>
__device__ __forceinline__ void do_flush_pp(ForwardPolicy<SELF> &pol, const WarpLists &L, int hb,
                                            int cnt, int) {
    pol.flush_pp(L, hb, cnt);
}
__device__ __forceinline__ void do_flush_pp(AdjointPolicy &pol, const WarpLists &L, int hb, int cnt,
                                            int lane) {
    if (cnt >= 32) pol.flush_pp<true>(L, hb, 32, lane);
    else if (cnt > 0) pol.flush_pp<false>(L, hb, cnt, lane);
}

// ---------------------------------------------------------------------------
// All-FP64 evaluation: the same walk and lists (the opening test is the same
// FP32 test), with the p-p and p-c terms of Eq. 1-2 evaluated in FP64 on the
// FP64 multipoles and positions, relative to the FP64 group centre.  The
// paper runs FP32 only; this variant is the reference of the precision
// study and is slow on purpose (FP64 pipe).
// ---------------------------------------------------------------------------

struct __align__(16) WarpLists64 {
    double cx[RING], cy[RING], cz[RING], cm[RING];
    double q[6][RING];  // xx yy zz xy xz yz
    double px[RING], py[RING], pz[RING], pm[RING];
    int pid[RING];
    float4 gbox, ghalf, glo;
    uint2 tsel;
};

__device__ __forceinline__ void pc_one64(double rx, double ry, double rz, double M, double qxx,
                                         double qyy, double qzz, double qxy, double qxz,
                                         double qyz, double eps2, double &ax, double &ay,
                                         double &az, double &ph) {
    const double s2 = fma(rz, rz, fma(ry, ry, fma(rx, rx, eps2)));
    const double u = 1.0 / sqrt(s2);
    const double w = u * u, u3 = u * w, u5 = u3 * w, u7 = u5 * w;
    const double tr = qxx + qyy + qzz;
    const double qx = qxx * rx + qxy * ry + qxz * rz;
    const double qy = qxy * rx + qyy * ry + qyz * rz;
    const double qz = qxz * rx + qyz * ry + qzz * rz;
    const double rQr = rx * qx + ry * qy + rz * qz;
    ph += -M * u + 0.5 * tr * u3 - 1.5 * rQr * u5;
    const double A = M * u3 - 1.5 * tr * u5 + 7.5 * rQr * u7;
    const double B = -3.0 * u5;
    ax += A * rx + B * qx;
    ay += A * ry + B * qy;
    az += A * rz + B * qz;
}

struct Fp64Policy {
    int gc;
    bool two;
    double eps2, cx, cy, cz;
    double tx[2], ty[2], tz[2], ax[2], ay[2], az[2], ph[2];
    int id[2];

    __device__ __forceinline__ void begin(const WalkArgs &A, WarpTargets *, uint32_t g,
                                          uint32_t gf, uint32_t gcount, float4, float4, int lane) {
        gc = (int)gcount;
        two = gc > 32;
        eps2 = A.eps2_64;
        cx = A.gcentre[g];
        cy = A.gcentre[A.ngroups + g];
        cz = A.gcentre[2 * A.ngroups + g];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int li = lane + 32 * k;
            const bool v = li < gc;
            const int64_t i = gf + (v ? li : 0);
            tx[k] = A.pos64[i] - cx;
            ty[k] = A.pos64[A.n + i] - cy;
            tz[k] = A.pos64[2 * A.n + i] - cz;
            id[k] = v ? (int)i : -1;
            ax[k] = ay[k] = az[k] = ph[k] = 0.0;
        }
    }
    __device__ __forceinline__ void append_cell(const WalkArgs &A, WarpLists64 &L, uint32_t s,
                                                uint32_t node, float4, float4, float4, uint32_t) {
        const int64_t nn = A.nn;
        L.cx[s] = A.ndcom[node] - cx;
        L.cy[s] = A.ndcom[nn + node] - cy;
        L.cz[s] = A.ndcom[2 * nn + node] - cz;
        L.cm[s] = A.ndM[node];
#pragma unroll
        for (int k = 0; k < 6; ++k) L.q[k][s] = A.ndQ[k * nn + node];
    }
    __device__ __forceinline__ void append_particle(const WalkArgs &A, WarpLists64 &L, uint32_t s,
                                                    uint32_t j, float4, float4, uint32_t) {
        L.px[s] = A.pos64[j] - cx;
        L.py[s] = A.pos64[A.n + j] - cy;
        L.pz[s] = A.pos64[2 * A.n + j] - cz;
        L.pm[s] = A.mass64[j];
        L.pid[s] = (int)j;
    }
    __device__ __forceinline__ void flush_pc(const WarpLists64 &L, int hb, int cnt) {
        for (int j = hb; j < hb + cnt; ++j) {
            const int nk = two ? 2 : 1;
            for (int k = 0; k < nk; ++k)
                pc_one64(L.cx[j] - tx[k], L.cy[j] - ty[k], L.cz[j] - tz[k], L.cm[j], L.q[0][j],
                         L.q[1][j], L.q[2][j], L.q[3][j], L.q[4][j], L.q[5][j], eps2, ax[k], ay[k],
                         az[k], ph[k]);
        }
    }
    __device__ __forceinline__ void flush_pp(const WarpLists64 &L, int hb, int cnt) {
        for (int j = hb; j < hb + cnt; ++j) {
            const int nk = two ? 2 : 1;
            for (int k = 0; k < nk; ++k) {
                if (L.pid[j] == id[k]) continue;  // the self pair
                const double rx = L.px[j] - tx[k], ry = L.py[j] - ty[k], rz = L.pz[j] - tz[k];
                const double s2 = fma(rz, rz, fma(ry, ry, fma(rx, rx, eps2)));
                const double u = 1.0 / sqrt(s2);
                const double mu = L.pm[j] * u, mu3 = mu * u * u;
                ph[k] -= mu;
                ax[k] += mu3 * rx;
                ay[k] += mu3 * ry;
                az[k] += mu3 * rz;
            }
        }
    }
    __device__ __forceinline__ void finish(const WalkArgs &A, uint32_t gf, uint32_t, int lane) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int li = lane + 32 * k;
            if (li < gc) {
                const uint32_t o = A.id[gf + li];
                if (A.acc64) {
                    A.acc64[o] = A.G64 * ax[k];
                    A.acc64[A.n + o] = A.G64 * ay[k];
                    A.acc64[2 * A.n + o] = A.G64 * az[k];
                }
                if (A.pot64) A.pot64[o] = A.G64 * ph[k];
            }
        }
    }
};

__device__ __forceinline__ void do_flush_pc(Fp64Policy &pol, const WarpLists64 &L, int hb, int cnt,
                                            int) {
    pol.flush_pc(L, hb, cnt);
}
__device__ __forceinline__ void do_flush_pp(Fp64Policy &pol, const WarpLists64 &L, int hb, int cnt,
                                            int) {
    pol.flush_pp(L, hb, cnt);
}

// ---------------------------------------------------------------------------
// List recording: the same walk, writing each group's accepted cells (node
// index) and opened-leaf particles (sorted index) in walk order at the
// group's offsets, so that the parity tests can compare list membership with
// the oracle's.  A group whose lists do not fit its offsets sets the
// overflow bit and writes nothing past its end.
// ---------------------------------------------------------------------------

struct ListPolicy : Fp32Rings {
    uint32_t *pc_out, *pp_out;
    int64_t pc_at, pc_end, pp_at, pp_end;
    bool over;

    __device__ __forceinline__ void begin(const WalkArgs &A, WarpTargets *, uint32_t g, uint32_t,
                                          uint32_t, float4, float4, int) {
        pc_out = A.lpc_out;
        pp_out = A.lpp_out;
        pc_at = A.lpc_off[g];
        pc_end = A.lpc_off[g + 1];
        pp_at = A.lpp_off[g];
        pp_end = A.lpp_off[g + 1];
        over = false;
    }
    __device__ __forceinline__ void flush_pc(const WarpLists &L, int hb, int cnt, int lane) {
        if (pc_at + cnt > pc_end) over = true;
        else if (lane < cnt) pc_out[pc_at + lane] = (uint32_t)L.cid[hb + lane];
        pc_at += cnt;
    }
    __device__ __forceinline__ void flush_pp(const WarpLists &L, int hb, int cnt, int lane) {
        if (pp_at + cnt > pp_end) over = true;
        else if (lane < cnt) pp_out[pp_at + lane] = (uint32_t)L.pid[hb + lane];
        pp_at += cnt;
    }
    __device__ __forceinline__ void finish(const WalkArgs &A, uint32_t, uint32_t, int lane) {
        if (lane == 0 && (over || pc_at != pc_end || pp_at != pp_end))
            atomicOr(&A.sc->status, ST_OVERFLOW);
    }
};

__device__ __forceinline__ void do_flush_pc(ListPolicy &pol, const WarpLists &L, int hb, int cnt,
                                            int lane) {
    pol.flush_pc(L, hb, cnt, lane);
}
__device__ __forceinline__ void do_flush_pp(ListPolicy &pol, const WarpLists &L, int hb, int cnt,
                                            int lane) {
    pol.flush_pp(L, hb, cnt, lane);
}

// ---------------------------------------------------------------------------
// The traversal
// ---------------------------------------------------------------------------

// The walk of group g's box, evaluated on tcnt of its targets starting at
// its target toff (the whole group, or one piece of it when the forward
// walk splits small workloads over more warps).
template <class P, class LT>
__device__ __forceinline__ void walk_group(const WalkArgs &A, LT &L, WarpTargets *tgt, P &pol,
                                           uint32_t g, uint32_t toff, uint32_t tcnt, uint32_t *fa,
                                           uint32_t *fb, int lane, uint32_t lt) {
    const uint32_t gf = A.gfirst[g] + toff, gc = tcnt;
    {
        const float4 box = A.gbox[g], clo = A.glo[g];
        if (lane == 0) {
            L.gbox = box;
            L.ghalf = A.ghalf[g];
            L.glo = clo;
            L.tsel = make_uint2(gf, gc);
        }
        pol.begin(A, tgt, g, gf, gc, box, clo, lane);
    }
    __syncwarp();

    // pc_tail and pp_tail count every entry ever appended: the list lengths
    uint32_t pc_head = 0, pc_tail = 0, pp_head = 0, pp_tail = 0;
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
            const float4 box = lds_f4(&L.gbox), half = lds_f4(&L.ghalf), clo = lds_f4(&L.glo);
            const bool open = mac_open(m, box, half);  // Sec. I.A opening test
            const bool leaf = (tp.y & LEAF_FLAG) != 0u;
            const bool accept = valid && !open;

            // accepted cells -> p-c ring
            const uint32_t am = __ballot_sync(0xffffffffu, accept);
            if (accept)
                pol.append_cell(A, L, (pc_tail + __popc(am & lt)) & (RING - 1), node, m, box, clo,
                                g);
            pc_tail += __popc(am);

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
            if (nnext + ntot > A.fcap) {
                overflow = true;
            } else {
                for (uint32_t k = 0; k < nch; ++k) nxt[nnext + noff + k] = tp.x + k;
                nnext += ntot;
            }

            // opened leaves -> p-p ring, 32 particles per round
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
                const float4 box = lds_f4(&L.gbox), clo = lds_f4(&L.glo);
                if (k < ltot)
                    pol.append_particle(A, L, (pp_tail + lane) & (RING - 1), sfirst + (k - soff),
                                        box, clo, g);
                pp_tail += min(32u, ltot - r);
                __syncwarp();
                if (pp_tail - pp_head >= 32u) {
                    // the head is a multiple of 32: the 32 entries do not wrap
                    do_flush_pp(pol, L, (int)(pp_head & (RING - 1)), 32, lane);
                    pp_head += 32;
                    __syncwarp();
                }
            }
            __syncwarp();
            while (pc_tail - pc_head >= 32u) {
                do_flush_pc(pol, L, (int)(pc_head & (RING - 1)), 32, lane);
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
    do_flush_pc(pol, L, (int)(pc_head & (RING - 1)), (int)(pc_tail - pc_head), lane);
    do_flush_pp(pol, L, (int)(pp_head & (RING - 1)), (int)(pp_tail - pp_head), lane);
    __syncwarp();
    const uint2 ts = lds_u2(&L.tsel);  // (gf, gc), not kept in registers through the walk
    pol.finish(A, ts.x, ts.y, lane);
    if (lane == 0) {
        if (A.gnpp) A.gnpp[g] = (int32_t)pp_tail;
        if (A.gnpc) A.gnpc[g] = (int32_t)pc_tail;
        atomicAdd((unsigned long long *)&A.sc->n_pp, (unsigned long long)ts.y * pp_tail);
        atomicAdd((unsigned long long *)&A.sc->n_pc, (unsigned long long)ts.y * pc_tail);
        atomicMax(&A.sc->max_frontier, (int)maxf);
        if (overflow) atomicOr(&A.sc->status, ST_OVERFLOW);
    }
    __syncwarp();
}

template <int SELF>
__global__ void __launch_bounds__(WALK_WARPS * 32) k_walk(const WalkArgs A) {
    __shared__ WarpLists lists[WALK_WARPS];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    const int64_t gw = (int64_t)blockIdx.x * WALK_WARPS + wib;
    uint32_t *fa = A.frontier + gw * 2 * FCAP;
    uint32_t *fb = fa + FCAP;
    // work item w: piece w % parts of group w / parts
    while (true) {
        uint32_t w = 0;
        if (lane == 0) w = atomicAdd(&A.sc->group_counter, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        const uint32_t parts = (uint32_t)A.parts;
        if (w >= (uint32_t)A.ngroups * parts) break;
        const uint32_t gi = w / parts, piece = w - gi * parts;
        const uint32_t g = A.gorder ? A.gorder[gi] : gi;
        const uint32_t gc = A.gcount[g], per = (gc + parts - 1u) / parts, tf = piece * per;
        if (tf >= gc) continue;
        ForwardPolicy<SELF> pol;
        walk_group(A, lists[wib], nullptr, pol, g, tf, min(per, gc - tf), fa, fb, lane, lt);
    }
}

__global__ void __launch_bounds__(WALK_WARPS * 32, 4) k_walk_adjoint(const WalkArgs A) {
    __shared__ WarpLists lists[WALK_WARPS];
    __shared__ WarpTargets targets[WALK_WARPS];
    __shared__ WarpAdjoint scratch[WALK_WARPS];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    const int64_t gw = (int64_t)blockIdx.x * WALK_WARPS + wib;
    uint32_t *fa = A.frontier + gw * 2 * FCAP;
    uint32_t *fb = fa + FCAP;
    // work item w: piece w % parts of group w / parts (as in k_walk)
    while (true) {
        uint32_t w = 0;
        if (lane == 0) w = atomicAdd(&A.sc->group_counter, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        const uint32_t parts = (uint32_t)A.parts;
        if (w >= (uint32_t)A.ngroups * parts) break;
        const uint32_t gi = w / parts, piece = w - gi * parts;
        const uint32_t g = A.gorder ? A.gorder[gi] : gi;
        const uint32_t gc = A.gcount[g], per = (gc + parts - 1u) / parts, tf = piece * per;
        if (tf >= gc) continue;
        AdjointPolicy pol;
        pol.cell_adj = A.cell_adj;
        pol.part_adj = A.part_adj;
        pol.nn = A.nn;
        pol.W = &scratch[wib];
        walk_group(A, lists[wib], &targets[wib], pol, g, tf, min(per, gc - tf), fa, fb, lane, lt);
    }
}

__global__ void __launch_bounds__(WALK_WARPS * 32) k_walk_lists(const WalkArgs A) {
    __shared__ WarpLists lists[WALK_WARPS];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    const int64_t gw = (int64_t)blockIdx.x * WALK_WARPS + wib;
    uint32_t *fa = A.frontier + gw * 2 * FCAP;
    uint32_t *fb = fa + FCAP;
    while (true) {
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(&A.sc->group_counter, 1u);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= A.ngroups) break;
        ListPolicy pol;
        walk_group(A, lists[wib], nullptr, pol, g, 0u, A.gcount[g], fa, fb, lane, lt);
    }
}

__global__ void __launch_bounds__(WALK_WARPS * 32) k_walk_fp64(const WalkArgs A) {
    __shared__ WarpLists64 lists[WALK_WARPS];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    const int64_t gw = (int64_t)blockIdx.x * WALK_WARPS + wib;
    uint32_t *fa = A.frontier + gw * 2 * FCAP;
    uint32_t *fb = fa + FCAP;
    while (true) {
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(&A.sc->group_counter, 1u);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= A.ngroups) break;
        Fp64Policy pol;
        walk_group(A, lists[wib], nullptr, pol, g, 0u, A.gcount[g], fa, fb, lane, lt);
    }
}

void fill_args(bonsai_ctx *c, float eps, WalkArgs &a) {
    a.mac = c->cell_mac.p;
    a.topo = c->cell_topo.p;
    a.ca = c->cell_a.p;
    a.cb = c->cell_b.p;
    a.cc = c->cell_c.p;
    a.body_hi = c->body_hi.p;
    a.body_lo = c->body_lo.p;
    a.src_hi = c->body_hi.p;
    a.src_lo = c->body_lo.p;
    a.accumulate = 0;
    a.parts = 1;
    a.gorder = nullptr;
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
    a.acc_c = nullptr;
    a.pot_c = nullptr;
    a.id = c->id.p;
    a.gnpp = c->grp_npp.p;
    a.gnpc = c->grp_npc.p;
    a.lam = nullptr;
    a.mu = nullptr;
    a.cell_adj = nullptr;
    a.part_adj = nullptr;
    a.nn = c->n_nodes;
    a.frontier = c->frontier.p;
    a.fcap = (c->walk_fcap > 0 && c->walk_fcap < FCAP) ? (uint32_t)c->walk_fcap : (uint32_t)FCAP;
    a.sc = c->dsc;
    a.pos64 = c->pos.p;
    a.mass64 = c->mass.p;
    a.gcentre = c->grp_centre.p;
    a.ndM = c->nd_M.p;
    a.ndcom = c->nd_com.p;
    a.ndQ = c->nd_Q.p;
    a.acc64 = nullptr;
    a.pot64 = nullptr;
    a.G64 = c->prm.G;
    a.eps2_64 = (double)eps * (double)eps;
    a.lpc_off = nullptr;
    a.lpp_off = nullptr;
    a.lpc_out = nullptr;
    a.lpp_out = nullptr;
}

}  // namespace

int walk_resident_warps(bonsai_ctx *c) {
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_walk<SELF_MASK>, WALK_WARPS * 32, 0) !=
            cudaSuccess || a < 1)
        a = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_walk<SELF_SUB>, WALK_WARPS * 32, 0) !=
            cudaSuccess || b < 1)
        b = 1;
    int d = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d, k_walk_adjoint, WALK_WARPS * 32, 0) !=
            cudaSuccess || d < 1)
        d = 1;
    const int per_sm = a > b ? (a > d ? a : d) : (b > d ? b : d);
    return per_sm * c->sm_count * WALK_WARPS;
}

size_t walk_frontier_elems(int warps) { return (size_t)warps * 2 * FCAP; }

static int launch_blocks(const void *fn, bonsai_ctx *c) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, WALK_WARPS * 32, 0) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    int blocks = per_sm * c->sm_count;
    const int cap = c->walk_warps / WALK_WARPS;  // frontier scratch is sized for this many
    return blocks < cap ? blocks : cap;
}

// Sort key of a group for the walk's fetch order: the largest FP32
// half-size of its box (the bit pattern of a non-negative float orders as
// the float).  64 particles in a small box sit in a dense region, whose
// lists are the longest, so ascending keys take the costliest groups first
// and leave the short walks for the end of the persistent grid's last wave.
__global__ void __launch_bounds__(256) k_group_order_keys(const float4 *__restrict__ half,
                                                          int64_t ng, uint64_t *__restrict__ key,
                                                          uint32_t *__restrict__ val) {
    for (int64_t g = blockIdx.x * 256ll + threadIdx.x; g < ng; g += (int64_t)gridDim.x * 256) {
        const float4 h = half[g];
        key[g] = (uint64_t)__float_as_uint(fmaxf(h.x, fmaxf(h.y, h.z)));
        val[g] = (uint32_t)g;
    }
}

// The groups in walk order (densest first) into grp_order; nullptr when the
// order is not used (the walk then fetches groups in index order).
static const uint32_t *walk_order(bonsai_ctx *c) {
    const int64_t ng = c->n_groups;
    if (ng < 2 || ensure(c->grp_okey, ng) || ensure(c->grp_okey2, ng) ||
        ensure(c->grp_order, ng) || ensure(c->grp_order2, ng))
        return nullptr;
    k_group_order_keys<<<grid_for(ng, 256, c->sm_count * 4), 256, 0, c->stream>>>(
        c->grp_half.p, ng, c->grp_okey.p, c->grp_order.p);
    // the particle sort's scratch is free once the tree is built
    c->launches += 1 + radix_sort_pairs_into(c->stream, c->sm_count, ng, c->grp_okey.p,
                                             c->grp_okey2.p, c->grp_order.p, c->grp_order2.p,
                                             c->hist.p, &c->dsc->status);
    return c->grp_order.p;
}

// With a few groups per warp, densest first (the order changes no result):
// there the last wave's long walks are a visible tail (at 2^20, 7.5 groups
// per warp: 7.49 -> 7.24 ms); with many groups per warp the tail is short
// and key order keeps neighbouring walks' records in L2 (at 2^23, 60 groups
// per warp: 61.60 ms in key order, 61.98 densest first).
static const uint32_t *walk_order_if_useful(bonsai_ctx *c, int parts, int blocks) {
    const int64_t warps = (int64_t)blocks * WALK_WARPS;
    if (parts == 1 && c->n_groups > warps && c->n_groups < 16 * warps) return walk_order(c);
    return nullptr;
}

// Pieces per group for the forward walk: when the groups are fewer than the
// resident warps (small N), each group's targets are split over up to
// MAX_PIECES warps that walk the same box (the same lists), so more warps
// share the evaluation; every target still sums its list in one warp.
constexpr int MAX_PIECES = 8;
static int walk_parts(int64_t ngroups, int blocks) {
    const int64_t warps = (int64_t)blocks * WALK_WARPS;
    const int64_t p = ngroups > 0 ? warps / ngroups : 1;
    return p >= MAX_PIECES ? MAX_PIECES : (p >= 1 ? (int)p : 1);
}

int walk_force(bonsai_ctx *c, float theta, float eps, float *acc_c, float *pot_c) {
    const bool mask_self = !(eps > 0.0f) || !(theta < 0.57f);
    WalkArgs a;
    fill_args(c, eps, a);
    a.acc_c = acc_c;
    a.pot_c = pot_c;
    const void *fn = mask_self ? (const void *)k_walk<SELF_MASK> : (const void *)k_walk<SELF_SUB>;
    const int blocks = launch_blocks(fn, c);
    a.parts = walk_parts(c->n_groups, blocks);
    a.gorder = walk_order_if_useful(c, a.parts, blocks);
    cudaEventRecord(c->ev[8], c->stream);
    if (mask_self)
        k_walk<SELF_MASK><<<blocks, WALK_WARPS * 32, 0, c->stream>>>(a);
    else
        k_walk<SELF_SUB><<<blocks, WALK_WARPS * 32, 0, c->stream>>>(a);
    cudaEventRecord(c->ev[9], c->stream);
    c->launches += 1;
    return cudaPeekAtLastError() == cudaSuccess ? BONSAI_OK : BONSAI_ECUDA;
}

// The walk of dst's groups over a local essential tree (cell records, leaf
// particle records); the forces are added to dst's key-order acc / pot.
int walk_let(bonsai_ctx *dst, const LetTree &t, float eps) {
    WalkArgs a;
    fill_args(dst, eps, a);
    a.mac = t.mac;
    a.topo = t.topo;
    a.ca = t.ca;
    a.cb = t.cb;
    a.cc = t.cc;
    a.src_hi = t.hi;
    a.src_lo = t.lo;
    a.nn = t.nn;
    a.accumulate = 1;
    const int blocks = launch_blocks((const void *)k_walk<SELF_NONE>, dst);
    a.parts = walk_parts(dst->n_groups, blocks);
    cudaEventRecord(dst->ev[8], dst->stream);
    k_walk<SELF_NONE><<<blocks, WALK_WARPS * 32, 0, dst->stream>>>(a);
    cudaEventRecord(dst->ev[9], dst->stream);
    dst->launches += 1;
    return cudaPeekAtLastError() == cudaSuccess ? BONSAI_OK : BONSAI_ECUDA;
}

// The adjoint walk: lam [3][n] and mu [n] (or null) in sorted order; adds the
// source-side and target-side gradients (times G) into part_adj [n] and the
// cell adjoints into cell_adj [3][nn].
int walk_adjoint(bonsai_ctx *c, float eps, const float *lam, const float *mu, float4 *cell_adj,
                 float4 *part_adj) {
    WalkArgs a;
    fill_args(c, eps, a);
    a.acc = nullptr;
    a.pot = nullptr;
    a.gnpp = nullptr;
    a.gnpc = nullptr;
    a.lam = lam;
    a.mu = mu;
    a.cell_adj = cell_adj;
    a.part_adj = part_adj;
    const int blocks = launch_blocks((const void *)k_walk_adjoint, c);
    a.parts = walk_parts(c->n_groups, blocks);
    a.gorder = walk_order_if_useful(c, a.parts, blocks);
    k_walk_adjoint<<<blocks, WALK_WARPS * 32, 0, c->stream>>>(a);
    c->launches += 1;
    return cudaPeekAtLastError() == cudaSuccess ? BONSAI_OK : BONSAI_ECUDA;
}

// The interaction lists of the current tree and packed opening test, at the
// caller's per-group offsets (device arrays, see ListPolicy).
int walk_lists(bonsai_ctx *c, const int64_t *pc_off, const int64_t *pp_off, uint32_t *pc_out,
               uint32_t *pp_out) {
    WalkArgs a;
    fill_args(c, 0.0f, a);
    a.acc = nullptr;
    a.pot = nullptr;
    a.gnpp = nullptr;
    a.gnpc = nullptr;
    a.lpc_off = pc_off;
    a.lpp_off = pp_off;
    a.lpc_out = pc_out;
    a.lpp_out = pp_out;
    k_walk_lists<<<launch_blocks((const void *)k_walk_lists, c), WALK_WARPS * 32, 0, c->stream>>>(a);
    c->launches += 1;
    return cudaPeekAtLastError() == cudaSuccess ? BONSAI_OK : BONSAI_ECUDA;
}

// The all-FP64 evaluation of the current tree and lists; outputs in caller order.
int walk_force_fp64(bonsai_ctx *c, float eps, double *acc, double *pot) {
    WalkArgs a;
    fill_args(c, eps, a);
    a.acc = nullptr;
    a.pot = nullptr;
    a.acc64 = acc;
    a.pot64 = pot;
    k_walk_fp64<<<launch_blocks((const void *)k_walk_fp64, c), WALK_WARPS * 32, 0, c->stream>>>(a);
    c->launches += 1;
    return cudaPeekAtLastError() == cudaSuccess ? BONSAI_OK : BONSAI_ECUDA;
}

}  // namespace bgb
