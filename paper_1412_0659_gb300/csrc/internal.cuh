// internal.cuh -- context layout, constants and kernel launchers shared by
// the translation units of the CUDA library.  Nothing here is part of the
// C ABI (include/bonsai_gb.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bonsai_gb.h"

namespace bgb {

constexpr int KEY_BITS = 21;   // bits per axis of the Peano-Hilbert key (63-bit key)
constexpr int MAX_LEVEL = 21;  // deepest octree level (one key value)
constexpr int NLEAF = 16;      // a node with more particles is split (Sec. I.A)
constexpr int NCRIT = 64;      // walk-group size
constexpr uint32_t LEAF_FLAG = 0x80000000u;  // topo.y: leaf marker, low bits = count

// device status word bits (set by kernels, read once per call)
constexpr int ST_BAD_INPUT = 1;      // non-finite position or mass <= 0
constexpr int ST_OVERFLOW = 2;       // a walk frontier overflowed
constexpr int ST_NODE_OVERFLOW = 4;  // node storage too small (host regrows)
constexpr int ST_TIMEOUT = 8;        // a bounded grid-barrier wait gave up
constexpr int ST_LONG_TIES = 16;     // a run of equal keys too long to fix in place
constexpr int BUILD_RETRY_EXACT = 1; // build_octree: sort again by the exact path

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

// cooperative octree build: threads per block, polls of a barrier wait
constexpr int OCT_BLOCK = 256;
constexpr int OCT_KEEP = 1 << 18;  // widest level whose child boundaries are kept between phases
constexpr uint32_t OCT_SPINS = 1u << 22;

// Device scalars written by kernels and read back in one copy.
struct DevScalars {
    double lo[3];     // bounding cube corner
    double L;         // cube side
    double scale;     // 2^21 / L
    uint64_t n_pp;    // interaction counters of the last walk
    uint64_t n_pc;
    int32_t status;        // ST_* bits
    int32_t max_frontier;
    uint32_t group_counter;  // dynamic scheduling of the walk
    uint32_t n_groups;
    int32_t pad;
    double mn[3], mx[3];  // componentwise bounds of the last bounding-box reduction
    // octree build: level starts, node count, depth, nodes needed after an
    // overflow, and the grid barrier's arrival counter and generation
    uint32_t oct_level[MAX_LEVEL + 2];
    uint32_t oct_nodes, oct_depth, oct_need;
    uint32_t bar_count, bar_gen;
};

// Bounding-cube reduction partials (per block)
struct BoxPartial {
    double mn[3], mx[3];
    int32_t bad;
    int32_t pad;
};

template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t cap = 0;  // elements
};

}  // namespace bgb

struct bonsai_ctx {
    bonsai_params prm;
    cudaStream_t stream;
    int device;
    int sm_count;

    int64_t n = 0;         // particles of the current tree
    int64_t n_nodes = 0;
    int64_t n_leaves = 0;
    int64_t n_groups = 0;
    int depth = 0;
    bool have_tree = false;
    bool have_forces = false;  // acc/pot in sorted order are valid
    bool have_vel = false;
    bool fixed_cube = false;         // keys in a given cube (a branch of a global octree)
    double cube[4] = {0, 0, 0, 0};   // lo[3], L of the current tree
    float packed_theta = -1.0f;  // theta of the current cell pack

    // particle state in key-sorted order (double buffers for the re-sort)
    bgb::DBuf<double> pos, pos2;     // [3][n]
    bgb::DBuf<double> vel, vel2;     // [3][n]
    bgb::DBuf<double> mass, mass2;   // [n]
    bgb::DBuf<uint32_t> id, id2;     // caller index of each sorted slot
    bgb::DBuf<float> acc;            // [3][n] sorted order, FP32, G applied
    bgb::DBuf<float> pot;            // [n]

    // keys and sort scratch
    bgb::DBuf<uint64_t> key, key2;
    bgb::DBuf<uint32_t> val, val2;
    bgb::DBuf<uint32_t> hist;        // radix histograms / scan
    bgb::DBuf<uint32_t> scan_tmp;
    bgb::DBuf<bgb::BoxPartial> box_part;

    // particle records for the walk: {x_hi, y_hi, z_hi, m} and {x_lo, y_lo, z_lo, 0}
    bgb::DBuf<float4> body_hi, body_lo;

    // nodes (breadth-first)
    bgb::DBuf<uint32_t> nd_first, nd_count, nd_child, nd_nchild, nd_level, nd_parent;
    bgb::DBuf<uint32_t> nd_scan;     // octree build: per-block child counts
    bgb::DBuf<uint32_t> nd_arrive;   // one-launch upward pass: finished children per node
    bgb::DBuf<uint32_t> nd_bounds;   // octree build: [7][OCT_KEEP] child boundaries of a level
    bgb::DBuf<double> nd_M;          // [nn]
    bgb::DBuf<double> nd_com;        // [3][nn]
    bgb::DBuf<double> nd_Q;          // [6][nn]
    // packed cell records for the walk
    bgb::DBuf<float4> cell_mac;      // {com_hi.xyz, r_open^2}
    bgb::DBuf<uint2> cell_topo;      // leaf: {first, count|LEAF}; internal: {child, nchild}
    bgb::DBuf<float4> cell_a;        // {com_lo.xyz, M}
    bgb::DBuf<float4> cell_b;        // -3 x {Qxx, Qyy, Qzz, Qxy}
    bgb::DBuf<float4> cell_c;        // {-3 Qxz, -3 Qyz, -trQ/2, -3/2 trQ}
    int64_t level_start[bgb::MAX_LEVEL + 2];

    // groups
    bgb::DBuf<uint32_t> grp_flag;    // [n+1] group-start flags / scan
    bgb::DBuf<uint32_t> grp_first, grp_count;
    bgb::DBuf<double> grp_centre;    // [3][ng] FP64 box centre
    bgb::DBuf<float4> grp_box;       // {c_f.xyz, 0}
    bgb::DBuf<float4> grp_half;      // {h_f.xyz (rounded up), 0}
    bgb::DBuf<float4> grp_lo;        // {c_lo.xyz, 0}: c = c_f + c_lo
    bgb::DBuf<int32_t> grp_npp, grp_npc;
    bgb::DBuf<uint64_t> grp_okey, grp_okey2;  // walk order: sort keys of the groups
    bgb::DBuf<uint32_t> grp_order, grp_order2;  // walk order: group indices, densest first

    // walk frontier scratch (per resident warp)
    bgb::DBuf<uint32_t> frontier;
    int walk_warps = 0;
    int walk_fcap = 0;  // 0: the full per-warp frontier; smaller values only for tests

    // device scalars + host mirror
    bgb::DevScalars *dsc = nullptr;
    bgb::DevScalars *hsc = nullptr;  // pinned host mirror

    // diagnostics scratch
    bgb::DBuf<double> diag_part;

    // adjoint
    float last_theta = 0.0f, last_eps = 0.0f;  // of the last force evaluation
    bgb::DBuf<float4> adj_cell;    // [3][nn] (com, M, Q) adjoint per node, FP32
    bgb::DBuf<float4> adj_part;    // [n] direct particle gradient {x, y, z, m}, key order
    bgb::DBuf<double> adj_node;    // [10][nn] accumulated alpha, B, beta
    bgb::DBuf<float> adj_lam, adj_mu;  // cotangents in key order
    bgb::DBuf<float> adj_ca;       // [3][n] cotangent in caller order (reverse chain)
    bgb::DBuf<uint32_t> leaf_of;   // leaf node of each key-order slot
    bgb::DBuf<double> adj_gpos, adj_gmass;  // gradient of one VJP, caller order
    // recorded run for the reverse chain: checkpoints of (pos, vel), caller order
    int run_steps = -1, run_ckpt = 1;
    double run_dt = 0.0;
    bgb::DBuf<double> run_mass;    // [n]
    bgb::DBuf<double> ckpt;        // [nck][6n]
    bgb::DBuf<double> seg_pos;     // [ckpt_every + 1][3n]

    // direct summation scratch
    bgb::DBuf<uint32_t> inv_id;    // [n] caller index -> key-order slot
    bgb::DBuf<double> dir_part;    // [chunks][4][nt] partial sums

    // pinned staging halves of the snapshot transfers (allocated on first use)
    void *stage[2] = {nullptr, nullptr};

    // timing events
    cudaEvent_t ev[10];
    bonsai_stats stats;
    uint64_t launches = 0;  // kernels launched by this context
};

namespace bgb {

// ---- allocation helpers (api.cu) ----
template <typename T>
int ensure(DBuf<T> &b, size_t n);
template <typename T>
void release(DBuf<T> &b);

// ---- context steps (api.cu) ----
int particle_buffers(bonsai_ctx *c, int64_t n);
// keys, sort, gather, octree, groups, multipoles, particle records;
// from_caller: pos/mass are caller-order arrays, else the context's state
int rebuild(bonsai_ctx *c, const double *pos, const double *mass, bool from_caller);

// ---- launchers (one per kernel family) ----
// keys.cu
void launch_bbox(bonsai_ctx *c, const double *pos, const double *mass, int64_t n);
// let.cu: overwrite the bounding cube with c->cube (keys in a given cube)
void launch_set_cube(bonsai_ctx *c);
// id non-null: pos is the key-ordered state with caller indices id; the
// keys are written in caller order and inv receives the inverse of id
void launch_keys(bonsai_ctx *c, const double *pos, int64_t n, const uint32_t *id = nullptr,
                 uint32_t *inv = nullptr);
// sort.cu
void radix_sort_pairs(bonsai_ctx *c, int64_t n);  // sorts key/val in place (ping-pong inside)
void exclusive_scan_u32(bonsai_ctx *c, const uint32_t *in, uint32_t *out, int64_t n,
                        uint32_t *total_dev);
void launch_gather_build(bonsai_ctx *c, const double *pos, const double *mass, int64_t n);
void launch_gather_step(bonsai_ctx *c, int64_t n, bool exact);
// tree.cu
int build_octree(bonsai_ctx *c);
int build_groups(bonsai_ctx *c);
int launch_multipoles(bonsai_ctx *c);
void launch_body_pack(bonsai_ctx *c);
void launch_cell_pack(bonsai_ctx *c, float theta);
// walk.cu
// A tree given by its walk records (a local essential tree, let.cu).
struct LetTree {
    const float4 *mac;
    const uint2 *topo;
    const float4 *ca, *cb, *cc;
    const float4 *hi, *lo;  // particle records of the opened leaves
    int64_t nn;
};
int walk_force(bonsai_ctx *c, float theta, float eps, float *acc_caller, float *pot_caller);
int walk_let(bonsai_ctx *dst, const LetTree &t, float eps);
int walk_force_fp64(bonsai_ctx *c, float eps, double *acc, double *pot);
int walk_lists(bonsai_ctx *c, const int64_t *pc_off, const int64_t *pp_off, uint32_t *pc_out,
               uint32_t *pp_out);
// direct.cu
int direct_forces(bonsai_ctx *c, const int64_t *targets, int64_t nt, float eps, double *acc,
                  double *pot);
// integrate.cu
void launch_kick(bonsai_ctx *c, double h);
void launch_drift(bonsai_ctx *c, double dt);
void launch_diagnostics(bonsai_ctx *c, double *out_dev);
int diag_blocks(bonsai_ctx *c);
int walk_resident_warps(bonsai_ctx *c);
size_t walk_frontier_elems(int warps);
// Tiles of the radix sort and of the scan, and the scratch sizes derived
// from them (constexpr, so that a fixed scratch layout can be checked at
// compile time).
constexpr int SORT_BLOCK = 256;
constexpr int SORT_IPT = 16;
constexpr int SORT_TILE = SORT_BLOCK * SORT_IPT;
constexpr int SCAN_BLOCK = 1024;
constexpr int SCAN_IPT = 4;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_IPT;
// entries of the scan's block-sum scratch for n inputs
constexpr size_t scan_tmp_elems(int64_t n) {
    size_t t = 0;
    int64_t m = n;
    while (m > SCAN_TILE) {
        m = (m + SCAN_TILE - 1) / SCAN_TILE;
        t += 2 * (size_t)m;
    }
    return t + 64;
}
// uint32 entries of the scratch of a sort of n pairs: one 64-bit look-back
// descriptor per tile and digit, then the 8 x 256 digit counts and the 8
// passes' tile counters
constexpr size_t sort_scratch_elems(int64_t n) {
    return 2 * 256 * (size_t)((n + SORT_TILE - 1) / SORT_TILE) + 8 * 256 + 64;
}
void launch_unpermute_state(bonsai_ctx *c, double *pos, double *vel, double *mass);
void launch_unpermute_forces(bonsai_ctx *c, float *acc, float *pot);
void launch_permute_in_vel(bonsai_ctx *c, const double *vel);
// adjoint.cu
int adjoint_buffers(bonsai_ctx *c);
int forces_vjp_sorted(bonsai_ctx *c, float theta, float eps, bool with_mu, double *gpos,
                      double *gmass);
void launch_cotangents_in(bonsai_ctx *c, const float *gacc, const float *gpot);
void launch_rev_drift(bonsai_ctx *c, double *vbar, const double *xbar, double dt, double coef);
void launch_rev_accum(bonsai_ctx *c, double *xbar, double *mbar);
// context-free variants on explicit buffers (noalloc.cu)
int launch_cube_keys_into(cudaStream_t s, int sm_count, const double *pos, const double *mass,
                          int64_t n, BoxPartial *part, int max_part, DevScalars *dsc,
                          uint64_t *key, uint32_t *val);
int radix_sort_pairs_into(cudaStream_t s, int sm_count, int64_t n, uint64_t *ka, uint64_t *kb,
                          uint32_t *va, uint32_t *vb, uint32_t *scratch, int32_t *status);

// Exclusive scan on explicit buffers (in and out must not alias; tmp holds
// scan_tmp_elems(n) entries); *total_dev receives the sum.  Returns the
// number of kernels launched.
int exclusive_scan_into(cudaStream_t s, const uint32_t *in, uint32_t *out, int64_t n,
                        uint32_t *tmp, uint32_t *total_dev);

// The opening test of Sec. I.A on FP32 records: m = {com_hi, r_open^2}, the
// group box centre and (rounded-up) half-size; the squared distance from the
// com to the box is formed with round-to-nearest in this fixed order.
__device__ __forceinline__ bool mac_open(float4 m, float4 box, float4 half) {
    const float dx = fmaxf(__fsub_rn(fabsf(__fsub_rn(m.x, box.x)), half.x), 0.0f);
    const float dy = fmaxf(__fsub_rn(fabsf(__fsub_rn(m.y, box.y)), half.y), 0.0f);
    const float dz = fmaxf(__fsub_rn(fabsf(__fsub_rn(m.z, box.z)), half.z), 0.0f);
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    return d2 < m.w;
}

inline int grid_for(int64_t n, int block, int max_blocks = 1 << 30) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

}  // namespace bgb

// Every host wait on the device is bounded (api.cu): the stream's work is
// polled through an event until it completes (BONSAI_OK), fails (ECUDA) or
// the process-wide limit passes (ETIMEOUT).
namespace bgb {
int wait_stream(cudaStream_t s);
}
#define BGB_WAIT(stream)                           \
    do {                                           \
        const int _w = bgb::wait_stream(stream);   \
        if (_w != BONSAI_OK) return _w;            \
    } while (0)

#define BGB_CUDA(call)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return BONSAI_ECUDA;     \
    } while (0)
