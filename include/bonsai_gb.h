/*
 * bonsai_gb.h -- C ABI of the GB300-native (sm_103a) tree-force library.
 *
 * The library computes, on one GPU, the per-step gravitational tree force of
 * Bonsai (Bedorf et al., SC14, Sec. III.A): Peano-Hilbert keys from the
 * bounding box (Sec. III.B.1), a key sort (Table 2 "Sorting SFC"), an octree
 * whose leaves hold at most 16 particles (Sec. I.A), a monopole+quadrupole
 * upward pass (Sec. VI.A, the 3x3 symmetric Q of Eq. 1-2), a group-wise walk
 * with an opening-angle criterion (Sec. I.A) fused with the softened
 * particle-particle and particle-cell evaluation of Eq. 1-2, and a
 * second-order kick-drift-kick leap-frog (Sec. III.B.2, last paragraph).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: BONSAI_OK (0) or a negative BONSAI_E* code.  No C++
 *   exception crosses this boundary.  bonsai_strerror() names a code.
 * - Pointers marked "device" must be CUDA device memory of the current
 *   device (e.g. a torch CUDA tensor's data_ptr()); "host" pointers are
 *   ordinary host memory (pinned memory makes the copies asynchronous).
 * - Positions and velocities are SoA float64 [3][n]: x[0..n), y[0..n),
 *   z[0..n).  Masses float64 [n].  Accelerations SoA float32 [3][n],
 *   potentials float32 [n].  Every input and output is in the caller's
 *   particle order; the key-sorted order is internal (see tree_debug_*).
 * - Ownership: the caller owns every pointer argument and keeps it valid
 *   for the duration of the call; the context owns its device scratch
 *   (allocated as n grows, freed by bonsai_destroy).
 * - Streams: all device work is enqueued on the context's stream.  Calls
 *   return after their work is complete (they synchronise the stream once
 *   to read the device status word), so outputs are ready on return.
 * - Units are the caller's: G is a parameter.
 */
#ifndef BONSAI_GB_H
#define BONSAI_GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BONSAI_OK 0
#define BONSAI_EINVAL (-1)    /* bad argument: null pointer, n <= 0, theta <= 0, eps < 0,
                                 non-finite position or mass <= 0 (found on the device) */
#define BONSAI_ENOMEM (-2)    /* a device allocation failed */
#define BONSAI_EOVERFLOW (-3) /* a bounded walk buffer overflowed (device status word) */
#define BONSAI_ECUDA (-4)     /* a CUDA runtime call failed */
#define BONSAI_ESTATE (-5)    /* call out of order, e.g. forces before a tree was built */
#define BONSAI_EIO (-6)       /* a snapshot file could not be opened, read or written, or
                                 is not a snapshot of this format (size, magic, version) */
#define BONSAI_ETIMEOUT (-7)  /* a host wait on the device exceeded the wait limit
                                 (bonsai_set_wait_timeout); the work stays queued.
                                 Also: a grid-wide barrier of the octree build gave
                                 up after about a second (the tree is not built) */

typedef struct bonsai_ctx bonsai_ctx;
typedef struct bonsai_let bonsai_let;

/* Parameters fixed at creation.  nleaf and ncrit must be 16 and 64: the
 * leaf size of Sec. I.A and the walk-group size; other values are EINVAL. */
typedef struct {
    double G;        /* gravitational constant in the caller's units */
    float theta;     /* opening angle used by tree_step (Sec. I.A; 0.4 in the paper) */
    float eps;       /* Plummer softening length used by tree_step */
    int32_t nleaf;   /* 16 */
    int32_t ncrit;   /* 64 */
    int32_t reserved[2];
} bonsai_params;

/* Statistics of the last tree_build / tree_forces. */
typedef struct {
    int64_t n;          /* particles */
    int64_t n_nodes;    /* octree nodes */
    int64_t n_groups;   /* walk groups */
    int32_t depth;      /* deepest level (root = 0) */
    int32_t max_frontier; /* largest per-group walk frontier seen */
    uint64_t n_pp;      /* sum over groups of |group| x |p-p list| (Sec. VI.A counts) */
    uint64_t n_pc;      /* sum over groups of |group| x |p-c list| */
    double flops;       /* 23 n_pp + 65 n_pc (Sec. VI.A convention) */
    float ms_keys;      /* bounding box + keys + sort + gather, last build */
    float ms_tree;      /* octree + groups + multipoles, last build */
    float ms_force;     /* cell pack + walk/force + scatter, last tree_forces */
    float ms_integrate; /* kicks + drift of the last tree_step */
    float ms_walk;      /* the fused walk/force kernel alone, last tree_forces */
    uint64_t launches;  /* kernels launched by this context since creation */
} bonsai_stats;

/* Create a context.  stream is a cudaStream_t (NULL = legacy default stream).
 * Errors: EINVAL (null out/params, nleaf != 16, ncrit != 64), ECUDA. */
int bonsai_create(bonsai_ctx **out, const bonsai_params *params, void *stream);

/* Destroy a context and free its device memory.  NULL is accepted. */
void bonsai_destroy(bonsai_ctx *ctx);

/* Replace the context's stream (cudaStream_t, NULL = legacy default). */
int bonsai_set_stream(bonsai_ctx *ctx, void *stream);

/* tree_build -- Sec. III.A "tree-construction" and "computation of multipole
 * moments" (with the keys and sort of Sec. III.B.1 / Table 2):
 *   bounding cube -> 21-bit Peano-Hilbert keys -> stable radix sort by
 *   (key, index) -> gather to key order -> octree (leaf <= 16 particles,
 *   children in key order, breadth-first numbering, built in one
 *   cooperative launch) -> walk groups (runs of consecutive sibling cells of
 *   <= 64 particles in all, under a parent with more) -> FP64 mass, centre
 *   of mass and non-traceless quadrupole per node.
 * pos: device [3][n] float64; mass: device [n] float64 (> 0, finite);
 * n >= 1.  The context copies what it needs; the caller's buffers are only
 * read during the call.  Velocities are reset to zero.
 * Errors: EINVAL (null pointer, n < 1 or > 2^31 - 1, non-finite position,
 * mass <= 0), ENOMEM, ECUDA, ETIMEOUT (see its definition). */
int tree_build(bonsai_ctx *ctx, const double *pos, const double *mass, int64_t n);

/* tree_forces -- Sec. III.A "tree-walk in which inter-particle gravitational
 * forces are computed", Eq. 1-2 of Sec. VI.A with Plummer softening:
 *   a_i = G sum_j [ m_j r/s^3 - 3/2 trQ_j r/s^5 - 3 Q_j r/s^5
 *                   + 15/2 (r^T Q_j r) r/s^7 ],
 *   phi_i = G sum_j [ -m_j/s + 1/2 trQ_j/s^3 - 3/2 r^T Q_j r/s^5 ],
 *   r = r_j - r_i, s = (|r|^2 + eps^2)^{1/2}, Q_j = 0 for particles; the
 *   self pair contributes nothing.  Sources are the cells accepted and the
 *   particles of the leaves opened by the group walk (opening test: a cell
 *   is opened when the squared distance from its centre of mass to the
 *   group's box is below (l/theta + |com - centre|)^2).
 * FP32 arithmetic on group-relative coordinates.  Interaction counts are in
 * tree_get_stats.  acc: device [3][n] float32 or NULL; pot: device [n]
 * float32 or NULL (caller order).  Requires a prior tree_build.
 * Errors: ESTATE (no tree), EINVAL (theta <= 0, eps < 0), EOVERFLOW, ECUDA. */
int tree_forces(bonsai_ctx *ctx, float theta, float eps, float *acc, float *pot);

/* tree_forces_fp64 -- the all-FP64 variant of tree_forces (the paper runs
 * FP32 only; this is the reference of a precision study): the same walk and
 * interaction lists (the opening test stays the FP32 test), with every p-p
 * and p-c term of Eq. 1-2 evaluated in FP64 on the FP64 multipoles and
 * positions relative to the FP64 group centre.  Much slower than
 * tree_forces (FP64 pipe).  acc: device float64 [3][n] or NULL; pot:
 * device float64 [n] or NULL (caller order).  The FP32 results of the last
 * tree_forces are left untouched.  Errors: as tree_forces. */
int tree_forces_fp64(bonsai_ctx *ctx, float theta, float eps, double *acc, double *pot);

/* Set the velocities of the particles of the last tree_build.
 * vel: device [3][n] float64, caller order.  Errors: ESTATE, EINVAL. */
int tree_set_velocities(bonsai_ctx *ctx, const double *vel);

/* tree_step -- one second-order leap-frog step (Sec. III.B.2, last
 * paragraph), kick-drift-kick in FP64:
 *   v += a dt/2;  x += v dt;  rebuild tree;  a = forces(x);  v += a dt/2,
 * with theta, eps and G from the creation parameters.  The forces at the
 * start of the step come from the previous tree_step or tree_forces (they
 * are computed here if there are none).  Errors: ESTATE, EOVERFLOW, ECUDA. */
int tree_step(bonsai_ctx *ctx, double dt);

/* Copy the FP64 state out in caller order; any pointer may be NULL.
 * pos, vel: device [3][n]; mass: device [n].  Errors: ESTATE. */
int tree_get_state(bonsai_ctx *ctx, double *pos, double *vel, double *mass);

/* Copy the accelerations and potentials of the last force evaluation out in
 * caller order; either pointer may be NULL.  acc: device [3][n] float32,
 * pot: device [n] float32.  Errors: ESTATE. */
int tree_get_forces(bonsai_ctx *ctx, float *acc, float *pot);

/* Energy and momentum diagnostics (Sec. VI: "gather and write statistics",
 * excluded from the flop count), FP64 on the device:
 *   out = {E_kin, E_pot, E_tot, Px, Py, Pz, Lx, Ly, Lz, M_total}, with
 *   E_kin = sum m v^2/2, E_pot = sum m phi/2 (phi of the last force
 *   evaluation), P = sum m v, L = sum m x cross v.  out: host double[10].
 * Errors: ESTATE (no forces yet), ECUDA. */
int bonsai_diagnostics(bonsai_ctx *ctx, double out[10]);

/* tree_direct_forces -- direct summation, the O(N^2) sum that the tree
 * approximates (Sec. I; the direct N-body kernel of Fig. 1), over all n
 * particles of the last tree_build for nt targets:
 *   a_i = G sum_{j != i} m_j r_ij / (|r_ij|^2 + eps^2)^{3/2},
 *   phi_i = -G sum_{j != i} m_j / (|r_ij|^2 + eps^2)^{1/2},  r_ij = x_j - x_i.
 * Pair terms in FP32 on coordinates split into an FP32 head and remainder
 * (differences accurate to FP32 relative to the separation), summed in FP32
 * within tiles of 256 sources and in FP64 across tiles, in a fixed order
 * (deterministic).  targets: device int64 [nt] caller indices, or NULL for
 * all particles (then nt must equal n).  acc: device float64 [3][nt], pot:
 * device float64 [nt], in the order of targets; either may be NULL.
 * Errors: EINVAL (null ctx, nt < 1, eps < 0, NULL targets with nt != n, an
 * index outside [0, n), found on the device), ESTATE (no tree), ENOMEM,
 * ECUDA. */
int tree_direct_forces(bonsai_ctx *ctx, const int64_t *targets, int64_t nt, float eps,
                       double *acc, double *pot);

/* ---- domains and local essential trees (Sec. III.B), on one GPU ------- */
/* The paper's processes each hold a piece of the global Peano-Hilbert
 * order, build their tree as a branch of the global octree, and send each
 * remote process the local essential tree (LET) it needs.  Here one context
 * stands for one process; the exchange is a device copy. */

/* tree_build_cube -- tree_build with the keys taken in the given cube
 * (cube = {lo_x, lo_y, lo_z, L}, host) instead of the particles' own
 * bounding cube, so that the trees of several domains are branches of one
 * global octree (Sec. III.B.1: the global bounding box maps every
 * process's coordinates to global PH keys).  Later tree_step calls keep the
 * cube.  Positions outside the cube are clamped to its edge cells.
 * Errors: as tree_build, and EINVAL for a non-finite cube or L <= 0. */
int tree_build_cube(bonsai_ctx *ctx, const double *pos, const double *mass, int64_t n,
                    const double cube[4]);

/* tree_domain_state -- copy the particles in key-order slots [first,
 * first + count) of the context's state out: pos, vel device float64
 * [3][count], mass [count], caller_id device uint32 [count] (the caller
 * index of each); any may be NULL.  With first = r n / R this is domain r of
 * R equal pieces of the Peano-Hilbert order (Sec. III.B.1).
 * Errors: EINVAL (bad range), ESTATE (no tree), ECUDA. */
int tree_domain_state(bonsai_ctx *ctx, int64_t first, int64_t count, double *pos, double *vel,
                      double *mass, uint32_t *caller_id);

/* A local essential tree: created empty, filled by let_build, read by
 * let_forces; owns its device arrays (the data a process sends).  stream:
 * a cudaStream_t for its kernels.  Errors: EINVAL, ENOMEM, ECUDA. */
int let_create(bonsai_let **out, void *stream);
void let_destroy(bonsai_let *let);

/* let_build -- the part of src's tree that dst's groups need (Sec. III.B.2):
 * src's tree is walked with the box of every group of dst (the opening test
 * of tree_forces at this theta); every cell reached is kept, an opened cell
 * with all its children, an opened leaf with its particles, a cell no group
 * opens as a leaf without particles.  Walking the LET with dst's groups
 * gives exactly the interaction lists of walking all of src's tree.  src
 * and dst must have been built with tree_build_cube in the same cube.
 * Errors: EINVAL (null, theta <= 0, different cubes), ESTATE (no tree),
 * EOVERFLOW (a marking walk's frontier overflowed), ENOMEM, ECUDA. */
int let_build(bonsai_let *let, bonsai_ctx *src, const bonsai_ctx *dst, float theta);

/* tree_get_group_boxes -- the walk's group boxes of the last build (Sec.
 * III.B.2: what a remote process needs to know of this one to build the
 * LET it sends here): box and half, device float [4][...] as float4 per
 * group, {centre.xyz (FP32, rounded to nearest), 0} and {half-size.xyz
 * (FP32, rounded up), 0}; either may be NULL; *ngroups (host, may be NULL)
 * receives the group count.  Errors: EINVAL, ESTATE (no tree), ECUDA. */
int tree_get_group_boxes(bonsai_ctx *ctx, float *box, float *half, int64_t *ngroups);

/* let_build_boxes -- let_build for group boxes received from a remote
 * process (tree_get_group_boxes there) instead of a context: the part of
 * src's tree that those groups need (Sec. III.B.2).  box, half: device
 * float4 [ngroups] as above; the remote tree must be a branch of the same
 * global octree (tree_build_cube in the same cube), which the caller
 * guarantees.  ngroups = 0 gives an empty LET.  Errors: EINVAL, ESTATE,
 * EOVERFLOW, ENOMEM, ECUDA. */
int let_build_boxes(bonsai_let *let, bonsai_ctx *src, const float *box, const float *half,
                    int64_t ngroups, float theta);

/* let_pack -- the LET as one contiguous buffer, the message a process sends
 * to another (Sec. III.B.2): a 64-byte header (magic "BGBLET01", cells,
 * particles, total bytes, theta), the cell records (4 x float4 per cell,
 * then the topology as uint2 per cell padded to 16 bytes) and the particle
 * records (2 x float4 per particle).  *bytes receives the packed size; with
 * buf NULL nothing else happens, otherwise buf (device, 16-byte aligned,
 * cap bytes >= *bytes, owned by the caller) receives the packed LET.
 * Errors: EINVAL (null, cap too small, misaligned buf), ECUDA. */
int let_pack(const bonsai_let *let, void *buf, int64_t cap, int64_t *bytes);

/* let_unpack -- a packed LET received from another process (buf: device,
 * 16-byte aligned, exactly the packed size) into let, ready for let_forces.
 * The header and the topology are checked (every internal cell's children
 * after it and inside the cell array, every leaf's particles inside the
 * particle array) before the LET is accepted.  The source-cell map of
 * let_debug_cells stays with the sender.  Errors: EINVAL (bad header,
 * size or topology; the LET is left empty), ENOMEM, ECUDA. */
int let_unpack(bonsai_let *let, const void *buf, int64_t bytes);

/* LET size: out = {cells, particles, bytes of its records, cells of the
 * source tree}.  Errors: EINVAL. */
int let_get_info(const bonsai_let *let, int64_t out[4]);

/* For tests: the source cell of each LET cell and its kind (0 used whole,
 * 1 opened cell, 2 opened leaf), device uint32 [cells] each; either may be
 * NULL.  Errors: EINVAL, ESTATE (empty LET, or one received by
 * let_unpack), ECUDA. */
int let_debug_cells(const bonsai_let *let, uint32_t *src_node, uint32_t *kind);

/* let_forces -- add the force of the LET's sources on dst's particles to
 * dst's current forces (those of its last tree_forces; read the sum with
 * tree_get_forces): dst's groups walk the LET like a local tree (Sec.
 * III.B.2: imported structures are processed separately as they arrive),
 * FP32 as tree_forces, no self pairs.  The per-group list lengths and the
 * counts of tree_get_stats become this walk's.
 * Errors: EINVAL, ESTATE (dst has no forces, empty LET), EOVERFLOW, ECUDA. */
int let_forces(bonsai_ctx *dst, const bonsai_let *let, float eps);

/* ---- snapshots and on-the-fly analysis (Sec. VI.C, Sec. IV Fig. 4) ---- */

/* tree_save_snapshot -- write the FP64 state of the context, in caller
 * order, to the file at path (Sec. VI.C: snapshots serve restarting and
 * analysis).  Format (little-endian): a 64-byte header {char magic[8] =
 * "BONSAIGB", uint32 version = 1, uint32 flags = 0, int64 n, double time,
 * double G, float theta, float eps, uint64 reserved[2]}, then pos [3][n],
 * vel [3][n], mass [n] as float64.  time is the caller's simulation time,
 * stored as given.  Streams through two 64 MB pinned staging buffers owned
 * by the context.  Errors: EINVAL (null ctx or path), ESTATE (no tree),
 * ENOMEM (staging), EIO, ECUDA. */
int tree_save_snapshot(bonsai_ctx *ctx, const char *path, double time);

/* tree_load_snapshot -- read a snapshot written by tree_save_snapshot into
 * the context: builds the tree of its positions and sets its velocities
 * (as tree_build followed by tree_set_velocities); *time (if non-NULL)
 * receives the stored time.  The context's creation parameters are kept.
 * Errors: EINVAL (null ctx or path, non-finite position or mass <= 0 in
 * the file), EIO (missing, short or foreign file), ENOMEM, ECUDA. */
int tree_load_snapshot(bonsai_ctx *ctx, const char *path, double *time);

/* tree_surface_density -- face-on (x-y) surface density of the particles
 * whose caller index is in [first, first + count) (for instance the disk
 * and bulge of Fig. 4), on an nx x ny grid over window = {xmin, xmax,
 * ymin, ymax}: each particle deposits m / (hx hy) onto the four pixel
 * centres nearest to it with bilinear (cloud-in-cell) weights, hx = (xmax -
 * xmin)/nx, hy = (ymax - ymin)/ny; deposits outside the grid are dropped.
 * FP64 with atomic additions (the order of the additions varies).  map:
 * device float64 [ny][nx], overwritten.  window: host double[4].
 * Errors: EINVAL (null pointer, nx or ny < 1, an empty or non-finite
 * window, a range outside [0, n)), ESTATE (no tree), ECUDA. */
int tree_surface_density(bonsai_ctx *ctx, int64_t first, int64_t count, const double window[4],
                         int nx, int ny, double *map);

/* ---- adjoint (vector-Jacobian products) ------------------------------- */
/* The paper has no adjoint.  These give the exact derivative of the forward
 * map with the tree and interaction lists of the forward evaluation held
 * fixed (node membership, opened cells and leaves are piecewise constant in
 * the positions; the multipoles stay functions of the particles). */

/* tree_forces_vjp -- for cotangents lambda = dL/da (device float32 [3][n])
 * and mu = dL/dphi (device float32 [n], or NULL for zero), writes
 *   gpos  = d(sum_i lambda_i.a_i + mu_i phi_i)/dx   (device float64 [3][n]),
 *   gmass = the same derivative with respect to the masses (device float64 [n]),
 * all in caller order, for the last tree_forces (same theta, eps, lists).
 * The walk is recomputed; p-c terms reach the particles through the
 * quadrupole upward pass (centre of mass and Q of every accepted cell).
 * FP32 evaluation, FP32 atomics per cell and particle, FP64 push-down.
 * Errors: EINVAL (null pointer), ESTATE (no forces yet), EOVERFLOW, ECUDA. */
int tree_forces_vjp(bonsai_ctx *ctx, const float *gacc, const float *gpot, double *gpos,
                    double *gmass);

/* tree_run -- nsteps calls of tree_step(dt) from the current state,
 * recording FP64 checkpoints of (pos, vel) every ckpt_every steps for
 * tree_run_vjp.  Errors: EINVAL, ESTATE, ENOMEM, as tree_step. */
int tree_run(bonsai_ctx *ctx, int nsteps, double dt, int ckpt_every);

/* tree_run_vjp -- reverse pass of the last tree_run.  In: xbar, vbar =
 * dL/dx_K, dL/dv_K (device float64 [3][n]) and mbar = dL/dm taken directly
 * (device float64 [n] or NULL).  Out: xbar0, vbar0 = dL/dx_0, dL/dv_0 and
 * mbar0 = dL/dm (device float64, caller order).  Each segment between
 * checkpoints is re-integrated to recover its positions; at every position
 * x_s the tree is rebuilt and the force VJP applied with the kick
 * cotangent (dt/2 v̄ at s = 0 and s = K, dt v̄ in between), the drift adding
 * dt x̄ to v̄.  The context's state afterwards is undefined (rebuild it).
 * Errors: EINVAL, ESTATE (no recorded run), ENOMEM, EOVERFLOW, ECUDA. */
int tree_run_vjp(bonsai_ctx *ctx, const double *xbar, const double *vbar, const double *mbar,
                 double *xbar0, double *vbar0, double *mbar0);

/* Statistics of the last build / force evaluation.  out: host. */
int tree_get_stats(bonsai_ctx *ctx, bonsai_stats *out);

/* End-to-end entry with HOST buffers: copies pos/mass (host [3][n] and [n]
 * float64) to the device, runs tree_build and tree_forces, and copies
 * acc/pot (host [3][n] and [n] float32) back, all on the context's stream.
 * Errors: as tree_build and tree_forces. */
int tree_solve_host(bonsai_ctx *ctx, const double *pos, const double *mass, int64_t n,
                    float theta, float eps, float *acc, float *pot);

/* ---- internal views for parity tests (key-sorted order) ---------------- */

/* Bounding cube of the last build: lo (host double[3]) and side L (host). */
int tree_debug_cube(bonsai_ctx *ctx, double lo[3], double *L);

/* Sorted keys (device uint64 [n]) and the caller index of each sorted slot
 * (device uint32 [n]); either may be NULL. */
int tree_debug_keys(bonsai_ctx *ctx, uint64_t *keys, uint32_t *perm);

/* Node arrays, breadth-first (device uint32 [n_nodes] each; any may be
 * NULL): first particle, particle count, first child, child count, level. */
int tree_debug_nodes(bonsai_ctx *ctx, uint32_t *first, uint32_t *count, uint32_t *child,
                     uint32_t *nchild, uint32_t *level);

/* FP64 multipoles (device): M [n_nodes], com [3][n_nodes], Q [6][n_nodes]
 * in the order xx, yy, zz, xy, xz, yz. */
int tree_debug_multipoles(bonsai_ctx *ctx, double *M, double *com, double *Q);

/* Groups (device uint32 [n_groups] first/count) and the p-p source count
 * and p-c list length of each group from the last tree_forces (device
 * int32 [n_groups]); any may be NULL. */
int tree_debug_groups(bonsai_ctx *ctx, uint32_t *first, uint32_t *count, int32_t *npp,
                      int32_t *npc);

/* The interaction lists of every group, as walked by the last tree_forces
 * (same tree, same opening angle; Sec. I.A: the walk accepts a cell as one
 * particle-cell interaction or opens it, an opened leaf giving its
 * particles as particle-particle interactions).  pc_off and pp_off are
 * device int64 [n_groups + 1]: exclusive prefix sums of the per-group p-c
 * list lengths and p-p source counts that tree_debug_groups returns.  Group
 * g's accepted cells (node indices, breadth-first numbering) go to
 * pc_cells[pc_off[g] .. pc_off[g+1]) and its p-p sources (key-sorted
 * particle indices) to pp_sources[pp_off[g] .. pp_off[g+1]), in walk
 * order; both device uint32, owned by the caller.  Nothing is written
 * outside a group's range.  Errors: EINVAL (null pointer), ESTATE (no
 * forces yet), EOVERFLOW (a group's lists do not have the lengths its
 * offsets give). */
int tree_debug_lists(bonsai_ctx *ctx, const int64_t *pc_off, const int64_t *pp_off,
                     uint32_t *pc_cells, uint32_t *pp_sources);

/* Limit the walk's per-warp frontier to cap entries (0 restores the full
 * capacity of 16384).  For tests of the overflow path: a walk that needs
 * more sets the device status word, and tree_forces / tree_forces_vjp
 * return BONSAI_EOVERFLOW; the context stays usable.  Errors: EINVAL. */
int tree_debug_set_frontier_capacity(bonsai_ctx *ctx, int cap);

/* Limit of every host wait on the device, in seconds, for all contexts of
 * the process (default 600).  Each call that needs a device result polls
 * an event recorded on its stream and returns BONSAI_ETIMEOUT once the
 * limit has passed; the work already queued still runs, and a later call
 * on the same stream is ordered after it.  (No paper counterpart: the
 * failure contract of this library.)  Errors: EINVAL (seconds not > 0 or
 * not finite). */
int bonsai_set_wait_timeout(double seconds);

/* Queue a host function on the context's stream that sleeps for the given
 * number of seconds (at most 60), holding back everything queued after it.
 * A test hook for the bounded waits: the device is not involved.  Errors:
 * EINVAL, ECUDA. */
int tree_debug_hold_stream(bonsai_ctx *ctx, double seconds);

/* tree_bounds -- the componentwise minimum mn[3] and maximum mx[3] (host)
 * of device positions pos [3][n] (with the input check of tree_build on
 * pos and mass [n]), by the bounding-box kernels of tree_build (Sec.
 * III.B.1); the context's tree is not touched.  Errors: EINVAL (null, bad
 * n, a non-finite position or a mass <= 0), ENOMEM, ECUDA. */
int tree_bounds(bonsai_ctx *ctx, const double *pos, const double *mass, int64_t n, double mn[3],
                double mx[3]);

/* bonsai_cube_from_bounds -- host: the cube the keys are taken in (Sec.
 * III.B.1: the global bounding box maps every coordinate to a global PH
 * key) from the componentwise minimum mn[3] and maximum mx[3] of all
 * positions, by the same FP64 steps as tree_build: side L = largest extent
 * x (1 + 2^-20) (1 when all points coincide), centred on the box.  For
 * processes that each hold part of the particles: reduce mn and mx over
 * them, then every process gets the same cube for tree_build_cube.
 * cube: host double[4] {lo_x, lo_y, lo_z, L}.  Errors: EINVAL (null,
 * non-finite, mn > mx). */
int bonsai_cube_from_bounds(const double mn[3], const double mx[3], double cube[4]);

/* Name of a status code. */
const char *bonsai_strerror(int code);

/* ---- space-filling-curve order without any device allocation ---------- */

/* Largest n accepted by bonsai_sfc_order_noalloc. */
#define BONSAI_NOALLOC_MAX_N (1 << 20)

/* bonsai_sfc_order_noalloc -- the bounding cube, the 63-bit Peano-Hilbert
 * keys and their stable sort, i.e. exactly the keys and the order that
 * tree_build computes for the same pos/mass (see tree_debug_keys), for
 * callers that must not allocate device memory.  There is no counterpart of
 * this entry point in the paper; it exists for users of the library.
 *
 * Who needs it: code that runs where cudaMalloc is not an option, e.g. a
 * host whose device memory is entirely owned by another allocator (a
 * framework's caching pool that has reserved the GPU, or a fixed memory
 * budget), a latency-critical loop that cannot afford the implicit
 * device-wide synchronisation of cudaMalloc/cudaFree, or a plugin that is
 * given buffers but no right to allocate.  It creates no context and calls
 * no cudaMalloc, cudaFree or allocating library routine.
 *
 * Scratch: a fixed static device array of about 13.2 MB (two ping-pong
 * halves of the sort for up to BONSAI_NOALLOC_MAX_N pairs, the sort's digit
 * counts and look-back descriptors, the bounding-box partials and a status
 * word), part of the library's
 * device code.  The CUDA runtime places it on a device when it loads that
 * code there: with the default lazy module loading at the first call on
 * the device, with CUDA_MODULE_LOADING=EAGER when the library is loaded.
 * The runtime, not this function, makes that placement, and it can fail
 * when another allocator already holds nearly all device memory; the first
 * call then returns ECUDA.  Once placed, the array stays on the device
 * until the process exits.  The first call on a device also looks up the
 * array's device address (with the device current) and caches it; make
 * that first call on each device before any stream capture begins.  Every
 * call on a device shares the same array, so calls whose
 * work overlaps on the GPU (different streams or threads without ordering)
 * race and must not be issued; calls on one stream are ordered and safe.
 *
 * pos: device [3][n] float64, mass: device [n] float64 (> 0, finite), both
 * read only.  keys: device uint64 [n], receives the sorted keys.  perm:
 * device uint32 [n], receives the caller index of each sorted slot.
 * cube: host double[4] or NULL, receives {lo_x, lo_y, lo_z, L}.  stream: a
 * cudaStream_t (NULL = legacy default stream).  The call returns after the
 * work is complete.
 * Errors: EINVAL (a null pointer, n < 1, n > BONSAI_NOALLOC_MAX_N, a
 * non-finite position or a mass <= 0), ECUDA, ETIMEOUT (a bounded wait of
 * the sort's look-back gave up; the output is then not sorted). */
int bonsai_sfc_order_noalloc(const double *pos, const double *mass, int64_t n, uint64_t *keys,
                             uint32_t *perm, double cube[4], void *stream);

/* ---- on-the-fly galaxy initial conditions (Sec. IV) ------------------ */
/* Sec. IV generates its Milky Way model on the fly instead of reading an
 * initial-condition file: an NFW dark-matter halo, an exponential stellar
 * disk and a Hernquist bulge.  These entry points build that model on the
 * GPU.  The halo and the bulge are sampled from their isotropic distribution
 * functions, obtained by Eddington's inversion in the spherically averaged
 * potential of all three components; each carries the outer taper
 * C(r) = erfc((r - r_t) / (sqrt(2) dr_t)) / 2.  The disk is exponential in
 * R (truncated at R_max) and sech^2 in z, with Gaussian velocities:
 * sigma_R^2 proportional to the surface density with Toomre's Q at R_Q,
 * the epicyclic azimuthal dispersion, the isothermal-sheet vertical
 * dispersion and the asymmetric-drift mean rotation held within [0, v_c]
 * (the epicyclic approximation, not a disk distribution function).  The
 * spheroids' distribution functions see the disk through its spherically
 * averaged mass, so they are in equilibrium in that potential; where the
 * flat disk dominates the inner mass the bulge adjusts.  Every particle
 * draws its uniforms from Philox4x32-10 (Salmon et al., SC11) with counter
 * (particle index, component, call, 0) and key (seed low word, seed high
 * word), so the output depends on the seed and n only, not on the launch
 * shape.  Units: kpc, Msun, Myr for the defaults. */

#define BONSAI_ICS_K 4096        /* radial nodes of the spheroid tables (1e-4 .. 600, log) */
#define BONSAI_ICS_V 256         /* speed-fraction nodes per velocity-table row */
#define BONSAI_ICS_KD 4096       /* radial nodes of the disk tables */
#define BONSAI_ICS_NRAD_OUT 15   /* rows of the radial table written by bonsai_galaxy_tables */
#define BONSAI_ICS_NDISK_OUT 7   /* rows of the disk table written by bonsai_galaxy_tables */

typedef struct {
    int64_t n_halo, n_disk, n_bulge;  /* particles per component (>= 0, sum < 2^32) */
    uint64_t seed;                    /* Philox key */
    double G;                         /* gravitational constant */
    double M_halo, a_halo;            /* NFW: total mass (with the taper), scale radius */
    double M_bulge, a_bulge;          /* Hernquist: total mass (with the taper), scale radius */
    double r_t, dr_t;                 /* outer taper of both spheroids */
    double M_disk, R_d, z0, R_max;    /* disk mass, scale length, sech^2 height, edge */
    double Q, R_Q;                    /* Toomre Q and the radius where it holds */
} bonsai_galaxy;

/* bonsai_galaxy_sec4 -- the Sec. IV model for n particles: component
 * masses 6.0e11 (halo), 5.0e10 (disk), 4.6e9 (bulge) Msun; counts in the
 * ratio of the paper's 51 G-particle realisation (bulge 994,689,024, disk
 * 2,945,105,920, halo 47,260,172,288: bulge and disk rounded down, the halo
 * takes the rest).  Scale lengths not given in the paper: a_halo = 15 kpc,
 * a_bulge = 0.5 kpc, r_t = 200 kpc, dr_t = 20 kpc, R_d = 2.5 kpc, z0 =
 * 0.3 kpc, R_max = 30 kpc, Q = 1.5 at R_Q = 2.43 R_d (Hernquist 1993);
 * G in kpc^3 Msun^-1 Myr^-2.
 * Errors: EINVAL (null, n < 1 or n >= 2^32). */
int bonsai_galaxy_sec4(bonsai_galaxy *g, int64_t n, uint64_t seed);

/* bonsai_galaxy_generate -- sample the model: pos, vel device float64
 * [3][n] SoA and mass device float64 [n], n = n_halo + n_disk + n_bulge;
 * halo first, then disk, then bulge; equal masses within a component; the
 * centre of mass and the mean velocity moved to zero.  Device scratch of
 * about 17 MB is allocated and freed stream-ordered (cudaMallocAsync).
 * Twelve kernels run on stream (a cudaStream_t, NULL = legacy default); the
 * call returns after they finish.  n = 0 does nothing.
 * Errors: EINVAL (null pointer with n > 0, a negative count, n >= 2^32, a
 * non-positive or non-finite length, G, Q or R_Q, R_max > 200 R_d, a
 * negative mass, zero mass for a component with particles), ENOMEM, ECUDA. */
int bonsai_galaxy_generate(const bonsai_galaxy *g, double *pos, double *vel, double *mass,
                           void *stream);

/* bonsai_galaxy_tables -- the generator's tables, for checks.  radial:
 * device float64 [BONSAI_ICS_NRAD_OUT][BONSAI_ICS_K], rows r, Psi (relative
 * potential), M(<r) total, M_halo(<r), M_bulge(<r), halo and bulge
 * cumulative mass fractions, halo and bulge d2rho/dPsi2, halo and bulge
 * f(E) at E = Psi, halo and bulge int_0^1 q^2 f dq, halo and bulge density.
 * vcdf: device float64 [2][K][V] (halo, bulge) normalised speed-fraction
 * cumulative distributions, or NULL.  disk: device float64
 * [BONSAI_ICS_NDISK_OUT][BONSAI_ICS_KD], rows: cumulative surface-mass
 * fraction at R = j R_max / (KD - 1); and at R = (j + 1/2) R_max / (KD - 1):
 * v_c^2, kappa, sigma_R, sigma_phi, sigma_z, mean v_phi.
 * Errors: as bonsai_galaxy_generate (null radial or disk: EINVAL). */
int bonsai_galaxy_tables(const bonsai_galaxy *g, double *radial, double *vcdf, double *disk,
                         void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BONSAI_GB_H */
