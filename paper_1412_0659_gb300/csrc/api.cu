// api.cu -- the C ABI of include/bonsai_gb.h: context, buffers, and the
// order of kernel launches for tree_build / tree_forces / tree_step.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <new>
#include <thread>

#include "internal.cuh"

namespace bgb {

template <typename T>
int ensure(DBuf<T> &b, size_t n) {
    if (n == 0) n = 1;
    if (b.cap >= n) return BONSAI_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    size_t cap = n + n / 8;
    if (cudaMalloc(&b.p, cap * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return BONSAI_ENOMEM;
    }
    b.cap = cap;
    return BONSAI_OK;
}

template <typename T>
void release(DBuf<T> &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

static std::atomic<double> g_wait_limit_s{600.0};

int wait_stream(cudaStream_t s) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return BONSAI_ECUDA;
    if (cudaEventRecord(e, s) != cudaSuccess) {
        cudaEventDestroy(e);
        return BONSAI_ECUDA;
    }
    const auto t0 = std::chrono::steady_clock::now();
    const double limit = g_wait_limit_s.load();
    int rc = BONSAI_OK;
    while (true) {
        const cudaError_t r = cudaEventQuery(e);
        if (r == cudaSuccess) break;
        if (r != cudaErrorNotReady) {
            rc = BONSAI_ECUDA;
            break;
        }
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > limit) {
            rc = BONSAI_ETIMEOUT;
            break;
        }
        // poll continuously for the first 2 ms (short calls), then every 50 us
        if (el > 2e-3) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    cudaEventDestroy(e);  // released by the runtime once the event completes
    return rc;
}

template int ensure<double>(DBuf<double> &, size_t);
template int ensure<float>(DBuf<float> &, size_t);
template int ensure<uint32_t>(DBuf<uint32_t> &, size_t);
template int ensure<int32_t>(DBuf<int32_t> &, size_t);
template int ensure<uint64_t>(DBuf<uint64_t> &, size_t);
template int ensure<float4>(DBuf<float4> &, size_t);
template int ensure<uint2>(DBuf<uint2> &, size_t);
template int ensure<BoxPartial>(DBuf<BoxPartial> &, size_t);
template void release<float4>(DBuf<float4> &);
template void release<uint2>(DBuf<uint2> &);
template void release<uint32_t>(DBuf<uint32_t> &);
template void release<int32_t>(DBuf<int32_t> &);

}  // namespace bgb

using namespace bgb;

namespace bgb {

// Bytes that ensure(b, n) would newly allocate, and the bytes it would free first.
template <typename T>
static void grow_bytes(const DBuf<T> &b, size_t n, size_t &alloc, size_t &freed) {
    if (n == 0) n = 1;
    if (b.cap >= n) return;
    alloc += (n + n / 8) * sizeof(T);
    freed += b.cap * sizeof(T);
}

int particle_buffers(bonsai_ctx *c, int64_t n) {
    const size_t n3 = 3 * (size_t)n;
    // the memory budget first: an n whose buffers cannot fit in the device
    // memory that is free (plus what the context would release to grow them)
    // fails with ENOMEM before anything is allocated or launched
    size_t alloc = 0, freed = 0;
    for (const DBuf<double> *b : {&c->pos, &c->pos2, &c->vel, &c->vel2}) grow_bytes(*b, n3, alloc, freed);
    grow_bytes(c->mass, n, alloc, freed);
    grow_bytes(c->mass2, n, alloc, freed);
    grow_bytes(c->id, n, alloc, freed);
    grow_bytes(c->id2, n, alloc, freed);
    grow_bytes(c->acc, n3, alloc, freed);
    grow_bytes(c->pot, n, alloc, freed);
    grow_bytes(c->key, n, alloc, freed);
    grow_bytes(c->key2, n, alloc, freed);
    grow_bytes(c->val, n, alloc, freed);
    grow_bytes(c->val2, n, alloc, freed);
    grow_bytes(c->body_hi, n, alloc, freed);
    grow_bytes(c->body_lo, n, alloc, freed);
    grow_bytes(c->grp_flag, 2 * (size_t)n + 2, alloc, freed);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return BONSAI_ECUDA;
    if (alloc > free_b + freed) return BONSAI_ENOMEM;
    if (ensure(c->pos, n3) || ensure(c->pos2, n3) || ensure(c->vel, n3) || ensure(c->vel2, n3) ||
        ensure(c->mass, n) || ensure(c->mass2, n) || ensure(c->id, n) || ensure(c->id2, n) ||
        ensure(c->acc, n3) || ensure(c->pot, n) || ensure(c->key, n) || ensure(c->key2, n) ||
        ensure(c->val, n) || ensure(c->val2, n) || ensure(c->hist, sort_scratch_elems(n)) ||
        ensure(c->scan_tmp, scan_tmp_elems(n)) ||
        ensure(c->box_part, (size_t)c->sm_count * 4 + 8) || ensure(c->body_hi, n) ||
        ensure(c->body_lo, n) || ensure(c->grp_flag, 2 * (size_t)n + 2) ||
        ensure(c->diag_part, (size_t)diag_blocks(c) * 10 + 16))
        return BONSAI_ENOMEM;
    return BONSAI_OK;
}

int node_buffers(bonsai_ctx *c) {
    const size_t nn = (size_t)c->n_nodes;
    if (ensure(c->nd_M, nn) || ensure(c->nd_com, 3 * nn) || ensure(c->nd_Q, 6 * nn) ||
        ensure(c->cell_mac, nn) || ensure(c->cell_a, nn) || ensure(c->cell_b, nn) ||
        ensure(c->cell_c, nn))
        return BONSAI_ENOMEM;
    return BONSAI_OK;
}

int read_scalars(bonsai_ctx *c) {
    BGB_CUDA(cudaMemcpyAsync(c->hsc, c->dsc, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                             c->stream));
    BGB_WAIT(c->stream);
    return BONSAI_OK;
}

// Keys, sort, gather, octree, groups, multipoles, particle records.
// from_caller: pos/mass are the caller's (caller order); otherwise the
// context's own state is re-sorted in place (tree_step): by default its keys
// are written in slot order and equal-key runs put in caller order after the
// sort; exact_ties writes each key at its caller index instead (taken when a
// run of equal keys is too long for the fix-up), and both give the (key,
// caller index) order.
static int rebuild_impl(bonsai_ctx *c, const double *pos, const double *mass, bool from_caller,
                        bool exact_ties);

int rebuild(bonsai_ctx *c, const double *pos, const double *mass, bool from_caller) {
    return rebuild_impl(c, pos, mass, from_caller, false);
}

static int rebuild_impl(bonsai_ctx *c, const double *pos, const double *mass, bool from_caller,
                        bool exact_ties) {
    const int64_t n = c->n;
    BGB_CUDA(cudaMemsetAsync(c->dsc, 0, sizeof(DevScalars), c->stream));
    BGB_CUDA(cudaEventRecord(c->ev[0], c->stream));
    const double *p = from_caller ? pos : c->pos.p;
    const double *m = from_caller ? mass : c->mass.p;
    launch_bbox(c, p, m, n);  // also checks the input
    if (c->fixed_cube) launch_set_cube(c);
    const bool scatter = !from_caller && exact_ties;
    if (scatter) {
        if (ensure(c->inv_id, (size_t)n)) return BONSAI_ENOMEM;
        launch_keys(c, p, n, c->id.p, c->inv_id.p);
    } else {
        launch_keys(c, p, n);
    }
    radix_sort_pairs(c, n);
    if (from_caller) {
        launch_gather_build(c, pos, mass, n);
    } else {
        launch_gather_step(c, n, scatter);  // also puts equal-key runs in caller order
    }
    BGB_CUDA(cudaEventRecord(c->ev[1], c->stream));
    BGB_CUDA(cudaGetLastError());
    c->have_tree = false;
    int rc = build_octree(c);
    if (rc == BUILD_RETRY_EXACT && !from_caller && !exact_ties)
        return rebuild_impl(c, nullptr, nullptr, false, true);
    if (rc) return rc;
    if ((rc = node_buffers(c))) return rc;
    if ((rc = build_groups(c))) return rc;
    if ((rc = launch_multipoles(c))) return rc;
    launch_body_pack(c);
    BGB_CUDA(cudaEventRecord(c->ev[2], c->stream));
    BGB_CUDA(cudaGetLastError());
    if ((rc = read_scalars(c))) return rc;
    if (c->hsc->status & ST_BAD_INPUT) {
        c->have_tree = false;
        return BONSAI_EINVAL;
    }
    if (c->hsc->status & ST_TIMEOUT) {  // a bounded device-side wait gave up
        c->have_tree = false;
        return BONSAI_ETIMEOUT;
    }
    if (!c->fixed_cube) {
        for (int d = 0; d < 3; ++d) c->cube[d] = c->hsc->lo[d];
        c->cube[3] = c->hsc->L;
    }
    cudaEventElapsedTime(&c->stats.ms_keys, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&c->stats.ms_tree, c->ev[1], c->ev[2]);
    c->have_tree = true;
    c->packed_theta = -1.0f;
    // leaves: nodes without children (counted from the level table on demand)
    return BONSAI_OK;
}

int forces_internal(bonsai_ctx *c, float theta, float eps, float *acc_c, float *pot_c) {
    if (!c->have_tree) return BONSAI_ESTATE;
    if (!(theta > 0.0f) || !(eps >= 0.0f) || !isfinite(theta) || !isfinite(eps))
        return BONSAI_EINVAL;
    if (c->walk_warps == 0) {
        c->walk_warps = walk_resident_warps(c);
        if (ensure(c->frontier, walk_frontier_elems(c->walk_warps))) return BONSAI_ENOMEM;
    }
    BGB_CUDA(cudaMemsetAsync(&c->dsc->n_pp, 0, 2 * sizeof(uint64_t), c->stream));
    BGB_CUDA(cudaMemsetAsync(&c->dsc->status, 0, 3 * sizeof(int32_t), c->stream));
    BGB_CUDA(cudaEventRecord(c->ev[3], c->stream));
    if (c->packed_theta != theta) {
        launch_cell_pack(c, theta);
        c->packed_theta = theta;
    }
    int rc = walk_force(c, theta, eps, acc_c, pot_c);
    if (rc) return rc;
    BGB_CUDA(cudaEventRecord(c->ev[4], c->stream));
    if ((rc = read_scalars(c))) return rc;
    cudaEventElapsedTime(&c->stats.ms_force, c->ev[3], c->ev[4]);
    cudaEventElapsedTime(&c->stats.ms_walk, c->ev[8], c->ev[9]);
    c->stats.n_pp = c->hsc->n_pp;
    c->stats.n_pc = c->hsc->n_pc;
    c->stats.flops = 23.0 * (double)c->hsc->n_pp + 65.0 * (double)c->hsc->n_pc;
    c->stats.max_frontier = c->hsc->max_frontier;
    if (c->hsc->status & ST_OVERFLOW) {
        c->have_forces = false;
        return BONSAI_EOVERFLOW;
    }
    if (c->hsc->status & ST_TIMEOUT) {  // the walk order's sort gave up: forces incomplete
        c->have_forces = false;
        return BONSAI_ETIMEOUT;
    }
    c->have_forces = true;
    c->last_theta = theta;
    c->last_eps = eps;
    return BONSAI_OK;
}

// One reverse force VJP at the current tree: cotangent already in adj_ca
// (caller order, FP32); adds the gradient into xbar, mbar (caller order).
int reverse_force_step(bonsai_ctx *c, double *xbar, double *mbar) {
    int rc = adjoint_buffers(c);
    if (rc) return rc;
    launch_cotangents_in(c, c->adj_ca.p, nullptr);
    rc = forces_vjp_sorted(c, c->prm.theta, c->prm.eps, false, c->adj_gpos.p, c->adj_gmass.p);
    if (rc) return rc;
    launch_rev_accum(c, xbar, mbar);
    return BONSAI_OK;
}

}  // namespace bgb

extern "C" {

int bonsai_create(bonsai_ctx **out, const bonsai_params *p, void *stream) {
    if (!out || !p) return BONSAI_EINVAL;
    *out = nullptr;
    if (p->nleaf != NLEAF || p->ncrit != NCRIT || !(p->theta > 0.0f) || !(p->eps >= 0.0f) ||
        !isfinite(p->G))
        return BONSAI_EINVAL;
    bonsai_ctx *c = new (std::nothrow) bonsai_ctx();
    if (!c) return BONSAI_ENOMEM;
    c->prm = *p;
    c->stream = (cudaStream_t)stream;
    memset(&c->stats, 0, sizeof(c->stats));
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) !=
            cudaSuccess) {
        delete c;
        return BONSAI_ECUDA;
    }
    if (cudaMalloc(&c->dsc, sizeof(DevScalars)) != cudaSuccess ||
        cudaMallocHost(&c->hsc, sizeof(DevScalars)) != cudaSuccess) {
        cudaFree(c->dsc);
        delete c;
        return BONSAI_ENOMEM;
    }
    for (int k = 0; k < 10; ++k) cudaEventCreate(&c->ev[k]);
    *out = c;
    return BONSAI_OK;
}

void bonsai_destroy(bonsai_ctx *c) {
    if (!c) return;
    wait_stream(c->stream);  // bounded; cudaFree below waits for the device in any case
    release(c->pos); release(c->pos2); release(c->vel); release(c->vel2);
    release(c->mass); release(c->mass2); release(c->id); release(c->id2);
    release(c->acc); release(c->pot); release(c->key); release(c->key2);
    release(c->val); release(c->val2); release(c->hist); release(c->scan_tmp);
    release(c->box_part); release(c->body_hi); release(c->body_lo);
    release(c->inv_id); release(c->dir_part);
    for (int k = 0; k < 2; ++k)
        if (c->stage[k]) cudaFreeHost(c->stage[k]);
    release(c->nd_first); release(c->nd_count); release(c->nd_child); release(c->nd_nchild);
    release(c->nd_level); release(c->nd_parent); release(c->nd_scan); release(c->nd_arrive); release(c->nd_bounds);
    release(c->grp_okey); release(c->grp_okey2); release(c->grp_order); release(c->grp_order2);
    release(c->nd_M); release(c->nd_com); release(c->nd_Q);
    release(c->cell_mac); release(c->cell_topo); release(c->cell_a); release(c->cell_b);
    release(c->cell_c);
    release(c->grp_flag); release(c->grp_first); release(c->grp_count); release(c->grp_centre);
    release(c->grp_box); release(c->grp_half); release(c->grp_lo); release(c->grp_npp);
    release(c->grp_npc); release(c->frontier); release(c->diag_part);
    release(c->adj_cell); release(c->adj_part); release(c->adj_node); release(c->adj_lam);
    release(c->adj_mu); release(c->adj_ca); release(c->leaf_of); release(c->adj_gpos);
    release(c->adj_gmass); release(c->run_mass); release(c->ckpt); release(c->seg_pos);
    cudaFree(c->dsc);
    cudaFreeHost(c->hsc);
    for (int k = 0; k < 10; ++k) cudaEventDestroy(c->ev[k]);
    delete c;
}

int bonsai_set_stream(bonsai_ctx *c, void *stream) {
    if (!c) return BONSAI_EINVAL;
    c->stream = (cudaStream_t)stream;
    return BONSAI_OK;
}

static int build_common(bonsai_ctx *c, const double *pos, const double *mass, int64_t n);

int tree_build(bonsai_ctx *c, const double *pos, const double *mass, int64_t n) {
    if (!c || !pos || !mass || n < 1 || n > 0x7fffffffll) return BONSAI_EINVAL;
    c->fixed_cube = false;
    return build_common(c, pos, mass, n);
}

int tree_build_cube(bonsai_ctx *c, const double *pos, const double *mass, int64_t n,
                    const double cube[4]) {
    if (!c || !pos || !mass || !cube || n < 1 || n > 0x7fffffffll) return BONSAI_EINVAL;
    for (int k = 0; k < 4; ++k)
        if (!isfinite(cube[k])) return BONSAI_EINVAL;
    if (!(cube[3] > 0.0)) return BONSAI_EINVAL;
    for (int k = 0; k < 4; ++k) c->cube[k] = cube[k];
    c->fixed_cube = true;
    return build_common(c, pos, mass, n);
}

static int build_common(bonsai_ctx *c, const double *pos, const double *mass, int64_t n) {
    c->have_tree = c->have_forces = c->have_vel = false;
    c->n = n;
    int rc = particle_buffers(c, n);
    if (rc) {
        c->n = 0;
        return rc;
    }
    rc = rebuild(c, pos, mass, true);
    if (rc) return rc;
    c->stats.n = n;
    c->stats.n_nodes = c->n_nodes;
    c->stats.n_groups = c->n_groups;
    c->stats.depth = c->depth;
    return BONSAI_OK;
}

int tree_forces(bonsai_ctx *c, float theta, float eps, float *acc, float *pot) {
    if (!c) return BONSAI_EINVAL;
    return forces_internal(c, theta, eps, acc, pot);
}

int tree_direct_forces(bonsai_ctx *c, const int64_t *targets, int64_t nt, float eps, double *acc,
                       double *pot) {
    if (!c || nt < 1 || !(eps >= 0.0f) || !isfinite(eps)) return BONSAI_EINVAL;
    if (!c->have_tree) return BONSAI_ESTATE;
    if (!targets && nt != c->n) return BONSAI_EINVAL;
    BGB_CUDA(cudaMemsetAsync(&c->dsc->status, 0, sizeof(int32_t), c->stream));
    int rc = direct_forces(c, targets, nt, eps, acc, pot);
    if (rc) return rc;
    if ((rc = read_scalars(c))) return rc;
    if (c->hsc->status & ST_BAD_INPUT) return BONSAI_EINVAL;
    return BONSAI_OK;
}

int tree_forces_fp64(bonsai_ctx *c, float theta, float eps, double *acc, double *pot) {
    if (!c) return BONSAI_EINVAL;
    if (!c->have_tree) return BONSAI_ESTATE;
    if (!(theta > 0.0f) || !(eps >= 0.0f) || !isfinite(theta) || !isfinite(eps))
        return BONSAI_EINVAL;
    if (c->walk_warps == 0) {
        c->walk_warps = walk_resident_warps(c);
        if (ensure(c->frontier, walk_frontier_elems(c->walk_warps))) return BONSAI_ENOMEM;
    }
    BGB_CUDA(cudaMemsetAsync(&c->dsc->n_pp, 0, 2 * sizeof(uint64_t), c->stream));
    BGB_CUDA(cudaMemsetAsync(&c->dsc->status, 0, 3 * sizeof(int32_t), c->stream));
    if (c->packed_theta != theta) {
        launch_cell_pack(c, theta);
        c->packed_theta = theta;
    }
    int rc = walk_force_fp64(c, eps, acc, pot);
    if (rc) return rc;
    if ((rc = read_scalars(c))) return rc;
    c->stats.n_pp = c->hsc->n_pp;
    c->stats.n_pc = c->hsc->n_pc;
    c->stats.flops = 23.0 * (double)c->hsc->n_pp + 65.0 * (double)c->hsc->n_pc;
    if (c->hsc->status & ST_OVERFLOW) return BONSAI_EOVERFLOW;
    return BONSAI_OK;
}

int tree_set_velocities(bonsai_ctx *c, const double *vel) {
    if (!c || !vel) return BONSAI_EINVAL;
    if (!c->have_tree) return BONSAI_ESTATE;
    launch_permute_in_vel(c, vel);
    BGB_WAIT(c->stream);
    c->have_vel = true;
    return BONSAI_OK;
}

int tree_step(bonsai_ctx *c, double dt) {
    if (!c || !isfinite(dt)) return BONSAI_EINVAL;
    if (!c->have_tree) return BONSAI_ESTATE;
    int rc;
    if (!c->have_forces && (rc = forces_internal(c, c->prm.theta, c->prm.eps, nullptr, nullptr)))
        return rc;
    BGB_CUDA(cudaEventRecord(c->ev[5], c->stream));
    launch_kick(c, 0.5 * dt);
    launch_drift(c, dt);
    BGB_CUDA(cudaEventRecord(c->ev[6], c->stream));
    c->have_forces = false;
    if ((rc = rebuild(c, nullptr, nullptr, false))) return rc;
    if ((rc = forces_internal(c, c->prm.theta, c->prm.eps, nullptr, nullptr))) return rc;
    BGB_CUDA(cudaEventRecord(c->ev[7], c->stream));
    launch_kick(c, 0.5 * dt);
    BGB_WAIT(c->stream);
    float a = 0.0f;
    cudaEventElapsedTime(&a, c->ev[5], c->ev[6]);
    c->stats.ms_integrate = 2.0f * a;
    c->stats.n_nodes = c->n_nodes;
    c->stats.n_groups = c->n_groups;
    c->stats.depth = c->depth;
    return BONSAI_OK;
}

int tree_get_state(bonsai_ctx *c, double *pos, double *vel, double *mass) {
    if (!c) return BONSAI_EINVAL;
    if (!c->have_tree) return BONSAI_ESTATE;
    launch_unpermute_state(c, pos, vel, mass);
    BGB_WAIT(c->stream);
    return BONSAI_OK;
}

int tree_get_forces(bonsai_ctx *c, float *acc, float *pot) {
    if (!c) return BONSAI_EINVAL;
    if (!c->have_forces) return BONSAI_ESTATE;
    launch_unpermute_forces(c, acc, pot);
    BGB_WAIT(c->stream);
    return BONSAI_OK;
}

int bonsai_diagnostics(bonsai_ctx *c, double out[10]) {
    if (!c || !out) return BONSAI_EINVAL;
    if (!c->have_forces) return BONSAI_ESTATE;
    double *dev = c->diag_part.p + (size_t)diag_blocks(c) * 10;
    launch_diagnostics(c, dev);
    BGB_CUDA(cudaMemcpyAsync(out, dev, 10 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    BGB_WAIT(c->stream);
    out[2] = out[0] + out[1];
    return BONSAI_OK;
}

int tree_get_stats(bonsai_ctx *c, bonsai_stats *out) {
    if (!c || !out) return BONSAI_EINVAL;
    c->stats.launches = c->launches;
    *out = c->stats;
    return BONSAI_OK;
}

int tree_forces_vjp(bonsai_ctx *c, const float *gacc, const float *gpot, double *gpos,
                    double *gmass) {
    if (!c || !gacc || !gpos || !gmass) return BONSAI_EINVAL;
    if (!c->have_forces) return BONSAI_ESTATE;
    int rc = adjoint_buffers(c);
    if (rc) return rc;
    launch_cotangents_in(c, gacc, gpot);
    rc = forces_vjp_sorted(c, c->last_theta, c->last_eps, gpot != nullptr, gpos, gmass);
    if (rc) return rc;
    if ((rc = read_scalars(c))) return rc;
    if (c->hsc->status & ST_OVERFLOW) return BONSAI_EOVERFLOW;
    return BONSAI_OK;
}

int tree_run(bonsai_ctx *c, int nsteps, double dt, int ckpt_every) {
    if (!c || nsteps < 0 || ckpt_every < 1 || !isfinite(dt)) return BONSAI_EINVAL;
    if (!c->have_tree) return BONSAI_ESTATE;
    const int64_t n = c->n;
    const int nck = (nsteps + ckpt_every - 1) / ckpt_every;
    if (ensure(c->ckpt, (size_t)(nck > 0 ? nck : 1) * 6 * n) || ensure(c->run_mass, n))
        return BONSAI_ENOMEM;
    c->run_steps = -1;
    launch_unpermute_state(c, nullptr, nullptr, c->run_mass.p);
    int rc;
    for (int s = 0; s < nsteps; ++s) {
        if (s % ckpt_every == 0) {
            double *ck = c->ckpt.p + (size_t)(s / ckpt_every) * 6 * n;
            launch_unpermute_state(c, ck, ck + 3 * n, nullptr);
        }
        if ((rc = tree_step(c, dt))) return rc;
    }
    BGB_WAIT(c->stream);
    c->run_steps = nsteps;
    c->run_ckpt = ckpt_every;
    c->run_dt = dt;
    return BONSAI_OK;
}

int tree_run_vjp(bonsai_ctx *c, const double *xbar, const double *vbar, const double *mbar,
                 double *xbar0, double *vbar0, double *mbar0) {
    if (!c || !xbar || !vbar || !xbar0 || !vbar0 || !mbar0) return BONSAI_EINVAL;
    if (c->run_steps < 0) return BONSAI_ESTATE;
    const int64_t n = c->n;
    const int K = c->run_steps, k = c->run_ckpt;
    const double dt = c->run_dt, h = 0.5 * dt;
    BGB_CUDA(cudaMemcpyAsync(xbar0, xbar, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    BGB_CUDA(cudaMemcpyAsync(vbar0, vbar, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if (mbar)
        BGB_CUDA(cudaMemcpyAsync(mbar0, mbar, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    else
        BGB_CUDA(cudaMemsetAsync(mbar0, 0, n * sizeof(double), c->stream));
    if (K == 0) {
        BGB_WAIT(c->stream);
        return BONSAI_OK;
    }
    // the reverse drift writes the kick cotangent (caller order) before the
    // first force VJP allocates the rest of the adjoint buffers
    if (ensure(c->seg_pos, (size_t)(k + 1) * 3 * n) || ensure(c->adj_ca, 3 * (size_t)n))
        return BONSAI_ENOMEM;
    int rc;
    const int nseg = (K + k - 1) / k;
    for (int j = nseg - 1; j >= 0; --j) {
        const int s0 = j * k, s1 = std::min(s0 + k, K);
        // re-run the segment from its checkpoint, keeping every position
        const double *ck = c->ckpt.p + (size_t)j * 6 * n;
        BGB_CUDA(cudaMemcpyAsync(c->seg_pos.p, ck, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice,
                                 c->stream));
        if ((rc = tree_build(c, ck, c->run_mass.p, n))) return rc;
        if ((rc = tree_set_velocities(c, ck + 3 * n))) return rc;
        for (int s = s0; s < s1; ++s) {
            if ((rc = tree_step(c, dt))) return rc;
            launch_unpermute_state(c, c->seg_pos.p + (size_t)(s + 1 - s0) * 3 * n, nullptr, nullptr);
        }
        // positions s1 .. s0 in reverse (s1 only when it is the last position)
        const int top = (s1 == K) ? s1 : s1 - 1;
        for (int s = top; s >= s0; --s) {
            // a_K enters only the last half kick; a_s (0 < s < K) both half
            // kicks around it; a_0 only the first; the drift adds dt xbar to
            // vbar before every position below K
            const double drift = (s == K) ? 0.0 : dt;
            const double coef = (s == K || s == 0) ? h : dt;
            launch_rev_drift(c, vbar0, xbar0, drift, coef);
            const double *xs = c->seg_pos.p + (size_t)(s - s0) * 3 * n;
            if ((rc = tree_build(c, xs, c->run_mass.p, n))) return rc;
            if ((rc = reverse_force_step(c, xbar0, mbar0))) return rc;
        }
    }
    if ((rc = read_scalars(c))) return rc;
    if (c->hsc->status & ST_OVERFLOW) return BONSAI_EOVERFLOW;
    return BONSAI_OK;
}

int tree_solve_host(bonsai_ctx *c, const double *pos, const double *mass, int64_t n, float theta,
                    float eps, float *acc, float *pot) {
    if (!c || !pos || !mass || n < 1 || n > 0x7fffffffll) return BONSAI_EINVAL;
    c->have_tree = c->have_forces = c->have_vel = false;
    c->n = n;
    int rc = particle_buffers(c, n);
    if (rc) {
        c->n = 0;
        return rc;
    }
    // stage the caller's arrays in the second state buffers, then build from them
    BGB_CUDA(cudaMemcpyAsync(c->pos2.p, pos, 3 * n * sizeof(double), cudaMemcpyHostToDevice,
                             c->stream));
    BGB_CUDA(cudaMemcpyAsync(c->mass2.p, mass, n * sizeof(double), cudaMemcpyHostToDevice,
                             c->stream));
    rc = rebuild(c, c->pos2.p, c->mass2.p, true);
    if (rc) return rc;
    rc = forces_internal(c, theta, eps, nullptr, nullptr);
    if (rc) return rc;
    // caller-order results staged in the key buffer's space, then copied to the host
    float *stage = reinterpret_cast<float *>(c->pos2.p);
    launch_unpermute_forces(c, stage, stage + 3 * n);
    if (acc)
        BGB_CUDA(cudaMemcpyAsync(acc, stage, 3 * n * sizeof(float), cudaMemcpyDeviceToHost,
                                 c->stream));
    if (pot)
        BGB_CUDA(cudaMemcpyAsync(pot, stage + 3 * n, n * sizeof(float), cudaMemcpyDeviceToHost,
                                 c->stream));
    BGB_WAIT(c->stream);
    c->stats.n = n;
    c->stats.n_nodes = c->n_nodes;
    c->stats.n_groups = c->n_groups;
    c->stats.depth = c->depth;
    return BONSAI_OK;
}

int tree_debug_cube(bonsai_ctx *c, double lo[3], double *L) {
    if (!c || !lo || !L) return BONSAI_EINVAL;
    if (!c->have_tree) return BONSAI_ESTATE;
    BGB_CUDA(cudaMemcpyAsync(c->hsc, c->dsc, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                             c->stream));
    BGB_WAIT(c->stream);
    for (int d = 0; d < 3; ++d) lo[d] = c->hsc->lo[d];
    *L = c->hsc->L;
    return BONSAI_OK;
}

int tree_debug_keys(bonsai_ctx *c, uint64_t *keys, uint32_t *perm) {
    if (!c) return BONSAI_EINVAL;
    if (!c->have_tree) return BONSAI_ESTATE;
    if (keys)
        BGB_CUDA(cudaMemcpyAsync(keys, c->key.p, c->n * sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                                 c->stream));
    if (perm)
        BGB_CUDA(cudaMemcpyAsync(perm, c->id.p, c->n * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                                 c->stream));
    BGB_WAIT(c->stream);
    return BONSAI_OK;
}

int tree_debug_nodes(bonsai_ctx *c, uint32_t *first, uint32_t *count, uint32_t *child,
                     uint32_t *nchild, uint32_t *level) {
    if (!c) return BONSAI_EINVAL;
    if (!c->have_tree) return BONSAI_ESTATE;
    const size_t b = c->n_nodes * sizeof(uint32_t);
    uint32_t *dst[5] = {first, count, child, nchild, level};
    uint32_t *src[5] = {c->nd_first.p, c->nd_count.p, c->nd_child.p, c->nd_nchild.p,
                        c->nd_level.p};
    for (int k = 0; k < 5; ++k)
        if (dst[k])
            BGB_CUDA(cudaMemcpyAsync(dst[k], src[k], b, cudaMemcpyDeviceToDevice, c->stream));
    BGB_WAIT(c->stream);
    return BONSAI_OK;
}

int tree_debug_multipoles(bonsai_ctx *c, double *M, double *com, double *Q) {
    if (!c) return BONSAI_EINVAL;
    if (!c->have_tree) return BONSAI_ESTATE;
    const size_t nn = c->n_nodes;
    if (M) BGB_CUDA(cudaMemcpyAsync(M, c->nd_M.p, nn * 8, cudaMemcpyDeviceToDevice, c->stream));
    if (com)
        BGB_CUDA(cudaMemcpyAsync(com, c->nd_com.p, 3 * nn * 8, cudaMemcpyDeviceToDevice, c->stream));
    if (Q) BGB_CUDA(cudaMemcpyAsync(Q, c->nd_Q.p, 6 * nn * 8, cudaMemcpyDeviceToDevice, c->stream));
    BGB_WAIT(c->stream);
    return BONSAI_OK;
}

int tree_debug_groups(bonsai_ctx *c, uint32_t *first, uint32_t *count, int32_t *npp,
                      int32_t *npc) {
    if (!c) return BONSAI_EINVAL;
    if (!c->have_tree) return BONSAI_ESTATE;
    if ((npp || npc) && !c->have_forces) return BONSAI_ESTATE;
    const size_t ng = c->n_groups;
    if (first)
        BGB_CUDA(cudaMemcpyAsync(first, c->grp_first.p, ng * 4, cudaMemcpyDeviceToDevice, c->stream));
    if (count)
        BGB_CUDA(cudaMemcpyAsync(count, c->grp_count.p, ng * 4, cudaMemcpyDeviceToDevice, c->stream));
    if (npp) BGB_CUDA(cudaMemcpyAsync(npp, c->grp_npp.p, ng * 4, cudaMemcpyDeviceToDevice, c->stream));
    if (npc) BGB_CUDA(cudaMemcpyAsync(npc, c->grp_npc.p, ng * 4, cudaMemcpyDeviceToDevice, c->stream));
    BGB_WAIT(c->stream);
    return BONSAI_OK;
}

int tree_debug_lists(bonsai_ctx *c, const int64_t *pc_off, const int64_t *pp_off,
                     uint32_t *pc_cells, uint32_t *pp_sources) {
    if (!c || !pc_off || !pp_off || !pc_cells || !pp_sources) return BONSAI_EINVAL;
    if (!c->have_tree || !c->have_forces) return BONSAI_ESTATE;
    BGB_CUDA(cudaMemsetAsync(&c->dsc->status, 0, 3 * sizeof(int32_t), c->stream));
    int rc = walk_lists(c, pc_off, pp_off, pc_cells, pp_sources);
    if (rc) return rc;
    if ((rc = read_scalars(c))) return rc;
    return (c->hsc->status & ST_OVERFLOW) ? BONSAI_EOVERFLOW : BONSAI_OK;
}

int tree_bounds(bonsai_ctx *c, const double *pos, const double *mass, int64_t n, double mn[3],
                double mx[3]) {
    if (!c || !pos || !mass || !mn || !mx || n < 1 || n > 0x7fffffffll) return BONSAI_EINVAL;
    if (ensure(c->box_part, (size_t)c->sm_count * 4 + 8)) return BONSAI_ENOMEM;
    BGB_CUDA(cudaMemsetAsync(&c->dsc->status, 0, sizeof(int32_t), c->stream));
    launch_bbox(c, pos, mass, n);  // also checks the input
    BGB_CUDA(cudaPeekAtLastError());
    int rc = read_scalars(c);
    if (rc) return rc;
    if (c->hsc->status & ST_BAD_INPUT) return BONSAI_EINVAL;
    for (int d = 0; d < 3; ++d) {
        mn[d] = c->hsc->mn[d];
        mx[d] = c->hsc->mx[d];
    }
    return BONSAI_OK;
}

int bonsai_set_wait_timeout(double seconds) {
    if (!(seconds > 0.0) || !isfinite(seconds)) return BONSAI_EINVAL;
    g_wait_limit_s.store(seconds);
    return BONSAI_OK;
}

static void CUDART_CB hold_host(void *arg) {
    const double s = *static_cast<double *>(arg);
    delete static_cast<double *>(arg);
    std::this_thread::sleep_for(std::chrono::duration<double>(s));
}

int tree_debug_hold_stream(bonsai_ctx *c, double seconds) {
    if (!c || !(seconds >= 0.0) || !(seconds <= 60.0)) return BONSAI_EINVAL;
    double *arg = new (std::nothrow) double(seconds);
    if (!arg) return BONSAI_ENOMEM;
    if (cudaLaunchHostFunc(c->stream, hold_host, arg) != cudaSuccess) {
        delete arg;
        return BONSAI_ECUDA;
    }
    return BONSAI_OK;
}

int tree_debug_set_frontier_capacity(bonsai_ctx *c, int cap) {
    if (!c || cap < 0) return BONSAI_EINVAL;
    c->walk_fcap = cap;
    return BONSAI_OK;
}

const char *bonsai_strerror(int code) {
    switch (code) {
        case BONSAI_OK: return "ok";
        case BONSAI_EINVAL: return "invalid argument";
        case BONSAI_ENOMEM: return "device allocation failed";
        case BONSAI_EOVERFLOW: return "walk buffer overflow";
        case BONSAI_ECUDA: return "CUDA runtime error";
        case BONSAI_ESTATE: return "call out of order";
        case BONSAI_EIO: return "snapshot file could not be opened, read or written, or has the wrong format";
        case BONSAI_ETIMEOUT: return "a wait on the device exceeded the wait limit";
        default: return "unknown status";
    }
}

}  // extern "C"
