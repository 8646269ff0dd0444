// adjoint.cu -- vector-Jacobian products of the tree forces with the tree
// and interaction lists held fixed, and of a chain of kick-drift-kick steps
// (reverse pass with checkpoints).  The paper has no adjoint; it is the
// exact derivative of the forward map of Eq. 1-2 for the lists the forward
// walk produced.
//
// tree_forces_vjp:
//   1. cotangents (caller order) -> key order (FP32);
//   2. k_walk_adjoint (walk.cu): recomputes the walk, adds the p-p source
//      and target gradients per particle and the (com, M, Q) adjoint per cell;
//   3. the cell adjoints reach the particles of each cell through
//      com = sum m x / M and Q = sum m (x - com)(x - com)^T:
//        dL/dx_k += m_k (gcom/M + 2 gQ (x_k - com)),
//        dL/dm_k += gM + gcom.(x_k - com)/M + (x_k - com)^T gQ (x_k - com).
//      Summed over the ancestors of a particle this is
//        dL/dx_k += m_k (alpha + 2 B x_k),  dL/dm_k += beta + alpha.x_k + x_k^T B x_k
//      with per-node alpha = gcom/M - 2 gQ com, B = gQ,
//      beta = gM - gcom.com/M + com^T gQ com, accumulated top-down by level
//      (FP64, HBM-bound);
//   4. back to caller order (FP64).
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace bgb {

int walk_adjoint(bonsai_ctx *c, float eps, const float *lam, const float *mu, float4 *cell_adj,
                 float4 *part_adj);

namespace {

constexpr int NADJ = 10;  // alpha (3), B (6: xx yy zz xy xz yz), beta

__global__ void __launch_bounds__(256) k_cotangents_in(const float *__restrict__ gacc,
                                                       const float *__restrict__ gpot,
                                                       const uint32_t *__restrict__ id, int64_t n,
                                                       float *__restrict__ lam,
                                                       float *__restrict__ mu) {
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const uint32_t o = id[i];
        lam[i] = gacc[o];
        lam[n + i] = gacc[n + o];
        lam[2 * n + i] = gacc[2 * n + o];
        if (gpot) mu[i] = gpot[o];
    }
}

__global__ void __launch_bounds__(256) k_leaf_of(const uint2 *__restrict__ topo, int64_t nn,
                                                 uint32_t *__restrict__ leaf_of) {
    int64_t c = blockIdx.x * 256ll + threadIdx.x;
    if (c >= nn) return;
    const uint2 t = topo[c];
    if (t.y & LEAF_FLAG) {
        const uint32_t cnt = t.y & ~LEAF_FLAG;
        for (uint32_t k = 0; k < cnt; ++k) leaf_of[t.x + k] = (uint32_t)c;
    }
}

// own alpha, B, beta of every node from its (com, M, Q) adjoint
__global__ void __launch_bounds__(256) k_adj_node_terms(const float4 *__restrict__ cell_adj,
                                                        const double *__restrict__ M,
                                                        const double *__restrict__ com, int64_t nn,
                                                        double *__restrict__ acc) {
    int64_t c = blockIdx.x * 256ll + threadIdx.x;
    if (c >= nn) return;
    const float4 a = cell_adj[c], b = cell_adj[nn + c], d = cell_adj[2 * nn + c];
    const double gcx = a.x, gcy = a.y, gcz = a.z, gM = a.w;
    const double qxx = b.x, qyy = b.y, qzz = b.z, qxy = b.w, qxz = d.x, qyz = d.y;
    const double Mi = 1.0 / M[c];
    const double cx = com[c], cy = com[nn + c], cz = com[2 * nn + c];
    const double bx = qxx * cx + qxy * cy + qxz * cz;
    const double by = qxy * cx + qyy * cy + qyz * cz;
    const double bz = qxz * cx + qyz * cy + qzz * cz;
    acc[c] = gcx * Mi - 2.0 * bx;
    acc[nn + c] = gcy * Mi - 2.0 * by;
    acc[2 * nn + c] = gcz * Mi - 2.0 * bz;
    acc[3 * nn + c] = qxx;
    acc[4 * nn + c] = qyy;
    acc[5 * nn + c] = qzz;
    acc[6 * nn + c] = qxy;
    acc[7 * nn + c] = qxz;
    acc[8 * nn + c] = qyz;
    acc[9 * nn + c] = gM - (gcx * cx + gcy * cy + gcz * cz) * Mi + (cx * bx + cy * by + cz * bz);
}

// add the parent's accumulated terms (the parent's level is complete)
__global__ void __launch_bounds__(256) k_adj_topdown(const uint32_t *__restrict__ parent,
                                                     int64_t nn, int64_t s, int64_t m,
                                                     double *__restrict__ acc) {
    int64_t t = blockIdx.x * 256ll + threadIdx.x;
    if (t >= m) return;
    const int64_t c = s + t;
    const uint32_t p = parent[c];
#pragma unroll
    for (int k = 0; k < NADJ; ++k) acc[k * nn + c] += acc[k * nn + p];
}

__global__ void __launch_bounds__(256) k_adj_particles(
    const double *__restrict__ pos, const double *__restrict__ mass,
    const uint32_t *__restrict__ leaf_of, const double *__restrict__ acc, int64_t nn,
    const float4 *__restrict__ part_adj, const uint32_t *__restrict__ id, int64_t n,
    double *__restrict__ gpos, double *__restrict__ gmass) {
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const uint32_t l = leaf_of[i];
        const double x = pos[i], y = pos[n + i], z = pos[2 * n + i], m = mass[i];
        const double ax = acc[l], ay = acc[nn + l], az = acc[2 * nn + l];
        const double qxx = acc[3 * nn + l], qyy = acc[4 * nn + l], qzz = acc[5 * nn + l];
        const double qxy = acc[6 * nn + l], qxz = acc[7 * nn + l], qyz = acc[8 * nn + l];
        const double beta = acc[9 * nn + l];
        const double bx = qxx * x + qxy * y + qxz * z;
        const double by = qxy * x + qyy * y + qyz * z;
        const double bz = qxz * x + qyz * y + qzz * z;
        const float4 d = part_adj[i];
        const uint32_t o = id[i];
        gpos[o] = (double)d.x + m * (ax + 2.0 * bx);
        gpos[n + o] = (double)d.y + m * (ay + 2.0 * by);
        gpos[2 * n + o] = (double)d.z + m * (az + 2.0 * bz);
        gmass[o] = (double)d.w + beta + (ax * x + ay * y + az * z) + (x * bx + y * by + z * bz);
    }
}

// ---- elementwise FP64 steps of the reverse kick-drift-kick chain ----

// vbar += dt xbar (dt may be 0); lam = (float)(c vbar), caller order
__global__ void __launch_bounds__(256) k_rev_drift(double *__restrict__ vbar,
                                                   const double *__restrict__ xbar, int64_t n3,
                                                   double dt, double c, float *__restrict__ lam) {
    for (int64_t k = blockIdx.x * 256ll + threadIdx.x; k < n3; k += (int64_t)gridDim.x * 256) {
        const double v = vbar[k] + dt * xbar[k];
        vbar[k] = v;
        lam[k] = (float)(c * v);
    }
}

// xbar += gpos; mbar += gmass
__global__ void __launch_bounds__(256) k_rev_accum(double *__restrict__ xbar,
                                                   const double *__restrict__ gpos,
                                                   double *__restrict__ mbar,
                                                   const double *__restrict__ gmass, int64_t n) {
    for (int64_t k = blockIdx.x * 256ll + threadIdx.x; k < 3 * n; k += (int64_t)gridDim.x * 256) {
        xbar[k] += gpos[k];
        if (k < n) mbar[k] += gmass[k];
    }
}

}  // namespace

int adjoint_buffers(bonsai_ctx *c) {
    const size_t n = (size_t)c->n, nn = (size_t)c->n_nodes;
    if (ensure(c->adj_cell, 3 * nn) || ensure(c->adj_part, n) || ensure(c->adj_node, NADJ * nn) ||
        ensure(c->adj_lam, 3 * n) || ensure(c->adj_mu, n) || ensure(c->leaf_of, n) ||
        ensure(c->adj_gpos, 3 * n) || ensure(c->adj_gmass, n) || ensure(c->adj_ca, 3 * n))
        return BONSAI_ENOMEM;
    return BONSAI_OK;
}

// VJP of the forces of the current tree at (theta, eps), cotangents in key
// order already in adj_lam / adj_mu (mu may be null); gradients (FP64,
// caller order) to gpos / gmass.
int forces_vjp_sorted(bonsai_ctx *c, float theta, float eps, bool with_mu, double *gpos,
                      double *gmass) {
    const int64_t n = c->n, nn = c->n_nodes;
    if (c->packed_theta != theta) {
        launch_cell_pack(c, theta);
        c->packed_theta = theta;
    }
    BGB_CUDA(cudaMemsetAsync(c->adj_cell.p, 0, 3 * nn * sizeof(float4), c->stream));
    BGB_CUDA(cudaMemsetAsync(c->adj_part.p, 0, n * sizeof(float4), c->stream));
    BGB_CUDA(cudaMemsetAsync(&c->dsc->status, 0, 3 * sizeof(int32_t), c->stream));
    int rc = walk_adjoint(c, eps, c->adj_lam.p, with_mu ? c->adj_mu.p : nullptr, c->adj_cell.p,
                          c->adj_part.p);
    if (rc) return rc;
    k_leaf_of<<<grid_for(nn, 256), 256, 0, c->stream>>>(c->cell_topo.p, nn, c->leaf_of.p);
    k_adj_node_terms<<<grid_for(nn, 256), 256, 0, c->stream>>>(c->adj_cell.p, c->nd_M.p,
                                                               c->nd_com.p, nn, c->adj_node.p);
    c->launches += 2;
    for (int l = 1; l <= c->depth; ++l) {
        const int64_t s = c->level_start[l], m = c->level_start[l + 1] - s;
        if (m <= 0) continue;
        k_adj_topdown<<<grid_for(m, 256), 256, 0, c->stream>>>(c->nd_parent.p, nn, s, m,
                                                               c->adj_node.p);
        c->launches += 1;
    }
    k_adj_particles<<<grid_for(n, 256, c->sm_count * 16), 256, 0, c->stream>>>(
        c->pos.p, c->mass.p, c->leaf_of.p, c->adj_node.p, nn, c->adj_part.p, c->id.p, n, gpos,
        gmass);
    c->launches += 1;
    BGB_CUDA(cudaGetLastError());
    return BONSAI_OK;
}

void launch_cotangents_in(bonsai_ctx *c, const float *gacc, const float *gpot) {
    k_cotangents_in<<<grid_for(c->n, 256, c->sm_count * 16), 256, 0, c->stream>>>(
        gacc, gpot, c->id.p, c->n, c->adj_lam.p, c->adj_mu.p);
    c->launches += 1;
}

void launch_rev_drift(bonsai_ctx *c, double *vbar, const double *xbar, double dt, double coef) {
    const int64_t n3 = 3 * c->n;
    k_rev_drift<<<grid_for(n3, 256, c->sm_count * 16), 256, 0, c->stream>>>(vbar, xbar, n3, dt, coef,
                                                                            c->adj_ca.p);
    c->launches += 1;
}

void launch_rev_accum(bonsai_ctx *c, double *xbar, double *mbar) {
    k_rev_accum<<<grid_for(3 * c->n, 256, c->sm_count * 16), 256, 0, c->stream>>>(
        xbar, c->adj_gpos.p, mbar, c->adj_gmass.p, c->n);
    c->launches += 1;
}

}  // namespace bgb
