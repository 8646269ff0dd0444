// direct.cu -- direct summation on the GPU: the O(N^2) sum that the tree
// approximates (Sec. I; the direct N-body kernel of Fig. 1), for a set of
// targets over all particles of the current tree.  It is the accuracy
// reference of the tree at sizes where a CPU sum is out of reach.
//
// Layout: a block owns DB x DT targets (DT per thread) and one chunk of the
// sources; the chunk is staged through shared memory in tiles of DTILE
// particle records.  Pair terms are FP32 on coordinates split into an FP32
// head and remainder (the difference (x_j,hi - x_i,hi) + (x_j,lo - x_i,lo) is
// accurate to FP32 relative to the separation), summed in FP32 within a
// tile and in FP64 across tiles.  Each source chunk writes its own FP64
// partial sums; a second kernel adds the chunks in order, so the result is
// deterministic.
#include "internal.cuh"

namespace bgb {

namespace {

constexpr int DB = 256;     // threads per block
constexpr int DT = 2;       // targets per thread
constexpr int DTILE = 256;  // source records per shared-memory tile
constexpr int MAX_CHUNKS = 64;

// caller index -> key-order slot
__global__ void __launch_bounds__(256) k_inverse_id(const uint32_t *__restrict__ id, int64_t n,
                                                    uint32_t *__restrict__ inv) {
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256)
        inv[id[i]] = (uint32_t)i;
}

// Partial sums of source chunk blockIdx.y for the block's targets:
// part[(chunk * 4 + c) * nt + t], c = ax, ay, az, phi (without G).
__global__ void __launch_bounds__(DB) k_direct(const float4 *__restrict__ hi,
                                               const float4 *__restrict__ lo, int64_t n,
                                               const int64_t *__restrict__ targets,
                                               const uint32_t *__restrict__ inv, int64_t nt,
                                               float eps2, int64_t chunk,
                                               double *__restrict__ part,
                                               DevScalars *__restrict__ sc) {
    __shared__ float4 sh[DTILE], sl[DTILE];
    float4 th[DT], tl[DT];
    int slot[DT];
    bool tv[DT];
    double ax[DT], ay[DT], az[DT], ph[DT];
#pragma unroll
    for (int d = 0; d < DT; ++d) {
        const int64_t t = ((int64_t)blockIdx.x * DT + d) * DB + threadIdx.x;
        tv[d] = t < nt;
        int64_t c = tv[d] ? (targets ? targets[t] : t) : 0;
        if (c < 0 || c >= n) {  // a bad caller index: reported, not read
            if (tv[d] && blockIdx.y == 0) atomicOr(&sc->status, ST_BAD_INPUT);
            c = 0;
        }
        slot[d] = (int)inv[c];
        th[d] = hi[slot[d]];
        tl[d] = lo[slot[d]];
        ax[d] = ay[d] = az[d] = ph[d] = 0.0;
    }
    const int64_t s0 = (int64_t)blockIdx.y * chunk;
    const int64_t s1 = min(n, s0 + chunk);
    for (int64_t base = s0; base < s1; base += DTILE) {
        __syncthreads();
        for (int k = threadIdx.x; k < DTILE; k += DB) {
            const int64_t j = base + k;
            if (j < s1) {
                sh[k] = hi[j];
                sl[k] = lo[j];
            }
        }
        __syncthreads();
        const int cnt = (int)min((int64_t)DTILE, s1 - base);
        float fx[DT], fy[DT], fz[DT], fp[DT];
#pragma unroll
        for (int d = 0; d < DT; ++d) fx[d] = fy[d] = fz[d] = fp[d] = 0.0f;
        const int jb = (int)base;
#pragma unroll 4
        for (int k = 0; k < cnt; ++k) {
            const float4 a = sh[k], b = sl[k];
#pragma unroll
            for (int d = 0; d < DT; ++d) {
                const float dx = (a.x - th[d].x) + (b.x - tl[d].x);
                const float dy = (a.y - th[d].y) + (b.y - tl[d].y);
                const float dz = (a.z - th[d].z) + (b.z - tl[d].z);
                float r2 = fmaf(dx, dx, eps2);
                r2 = fmaf(dy, dy, r2);
                r2 = fmaf(dz, dz, r2);
                const float rinv = (jb + k == slot[d]) ? 0.0f : rsqrtf(r2);  // j = i: nothing
                const float mr = a.w * rinv;
                const float mr3 = mr * rinv * rinv;
                fp[d] -= mr;
                fx[d] = fmaf(mr3, dx, fx[d]);
                fy[d] = fmaf(mr3, dy, fy[d]);
                fz[d] = fmaf(mr3, dz, fz[d]);
            }
        }
#pragma unroll
        for (int d = 0; d < DT; ++d) {
            ax[d] += (double)fx[d];
            ay[d] += (double)fy[d];
            az[d] += (double)fz[d];
            ph[d] += (double)fp[d];
        }
    }
#pragma unroll
    for (int d = 0; d < DT; ++d) {
        const int64_t t = ((int64_t)blockIdx.x * DT + d) * DB + threadIdx.x;
        if (!tv[d]) continue;
        double *p = part + (int64_t)blockIdx.y * 4 * nt;
        p[t] = ax[d];
        p[nt + t] = ay[d];
        p[2 * nt + t] = az[d];
        p[3 * nt + t] = ph[d];
    }
}

// Add the chunks in order and apply G.
__global__ void __launch_bounds__(256) k_direct_final(const double *__restrict__ part, int nchunks,
                                                      int64_t nt, double G, double *__restrict__ acc,
                                                      double *__restrict__ pot) {
    for (int64_t t = blockIdx.x * 256ll + threadIdx.x; t < nt; t += (int64_t)gridDim.x * 256) {
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int c = 0; c < nchunks; ++c)
            for (int k = 0; k < 4; ++k) s[k] += part[((int64_t)c * 4 + k) * nt + t];
        if (acc) {
            acc[t] = G * s[0];
            acc[nt + t] = G * s[1];
            acc[2 * nt + t] = G * s[2];
        }
        if (pot) pot[t] = G * s[3];
    }
}

}  // namespace

int direct_forces(bonsai_ctx *c, const int64_t *targets, int64_t nt, float eps, double *acc,
                  double *pot) {
    const int64_t n = c->n;
    if (ensure(c->inv_id, (size_t)n)) return BONSAI_ENOMEM;
    const int64_t tblocks = (nt + DB * DT - 1) / (DB * DT);
    int64_t nchunks = (8ll * c->sm_count + tblocks - 1) / tblocks;
    const int64_t max_chunks = (n + DTILE - 1) / DTILE;
    if (nchunks > MAX_CHUNKS) nchunks = MAX_CHUNKS;
    if (nchunks > max_chunks) nchunks = max_chunks;
    if (nchunks < 1) nchunks = 1;
    int64_t chunk = (n + nchunks - 1) / nchunks;
    chunk = (chunk + DTILE - 1) / DTILE * DTILE;
    nchunks = (n + chunk - 1) / chunk;
    if (ensure(c->dir_part, (size_t)(nchunks * 4 * nt))) return BONSAI_ENOMEM;
    k_inverse_id<<<grid_for(n, 256, c->sm_count * 16), 256, 0, c->stream>>>(c->id.p, n, c->inv_id.p);
    const dim3 grid((unsigned)tblocks, (unsigned)nchunks);
    k_direct<<<grid, DB, 0, c->stream>>>(c->body_hi.p, c->body_lo.p, n, targets, c->inv_id.p, nt,
                                         eps * eps, chunk, c->dir_part.p, c->dsc);
    k_direct_final<<<grid_for(nt, 256, c->sm_count * 16), 256, 0, c->stream>>>(
        c->dir_part.p, (int)nchunks, nt, c->prm.G, acc, pot);
    c->launches += 3;
    return cudaPeekAtLastError() == cudaSuccess ? BONSAI_OK : BONSAI_ECUDA;
}

}  // namespace bgb
