// direct.cu -- direct summation on the GPU: the O(N^2) sum that the tree
// approximates (Sec. I; the direct N-body kernel of Fig. 1), for a set of
// targets over all particles of the current tree.  It is the accuracy
// reference of the tree at sizes where a CPU sum is out of reach.
//
// Layout: a block owns DB x 2 DP targets (DP pairs per thread, the two
// targets of a pair in one packed FP32 register pair, so that each packed
// instruction evaluates two pair terms) and one chunk of the sources; the
// chunk is staged through shared memory in tiles of DTILE particle records,
// each record feeding 2 DP pair terms per thread.  Pair terms are FP32 on
// tile-relative coordinates taken from the FP32 head and remainder of each
// FP64 position (see k_direct), summed in FP32 within a tile and in FP64
// across tiles (the FP64 running sums live in shared memory).  Each source chunk writes its
// own FP64 partial sums; a second kernel adds the chunks in order, so the
// result is deterministic.  The self pair (j = i) contributes nothing: it is
// masked per pair, but only in the tiles that hold the self source of one
// of the block's targets (with eps = 0 in every tile).
#include <algorithm>

#include "internal.cuh"
#include "packed.cuh"

namespace bgb {

namespace {

constexpr int DB = 128;     // threads per block
constexpr int DP = 3;       // target pairs per thread (6 blocks of 80 registers per SM)
constexpr int DTG = 2 * DP; // targets per thread
constexpr int DTILE = 256;  // source records per shared-memory tile
constexpr int MAX_CHUNKS = 64;

// caller index -> key-order slot
__global__ void __launch_bounds__(256) k_inverse_id(const uint32_t *__restrict__ id, int64_t n,
                                                    uint32_t *__restrict__ inv) {
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256)
        inv[id[i]] = (uint32_t)i;
}

// One tile of cnt staged sources (tile-relative coordinates and mass) on
// the thread's DP target pairs (tile-relative), FP32 sums into f*.  MASK:
// the self pair (tile source ks[d] of target d) contributes nothing.
template <bool MASK>
__device__ __forceinline__ void tile_pairs(const float4 *sr, int cnt, const int *ks, const f32x2 *tx,
                                           const f32x2 *ty, const f32x2 *tz, f32x2 e2, f32x2 *fx,
                                           f32x2 *fy, f32x2 *fz, f32x2 *fp) {
#pragma unroll 2
    for (int k = 0; k < cnt; ++k) {
        const float4 a = sr[k];
        const f32x2 ax = dup2(a.x), ay = dup2(a.y), az = dup2(a.z), am = dup2(a.w);
#pragma unroll
        for (int p = 0; p < DP; ++p) {
            const f32x2 dx = sub2(ax, tx[p]);
            const f32x2 dy = sub2(ay, ty[p]);
            const f32x2 dz = sub2(az, tz[p]);
            f32x2 r2 = fma2(dx, dx, e2);
            r2 = fma2(dy, dy, r2);
            r2 = fma2(dz, dz, r2);
            float r0, r1;
            u2(r2, r0, r1);
            float q0 = rsqrtf(r0), q1 = rsqrtf(r1);
            if (MASK) {  // j = i: nothing
                q0 = (k == ks[2 * p]) ? 0.0f : q0;
                q1 = (k == ks[2 * p + 1]) ? 0.0f : q1;
            }
            const f32x2 rinv = p2(q0, q1);
            const f32x2 mr = mul2(am, rinv);
            const f32x2 mr3 = mul2(mr, mul2(rinv, rinv));
            fp[p] = sub2(fp[p], mr);
            fx[p] = fma2(mr3, dx, fx[p]);
            fy[p] = fma2(mr3, dy, fy[p]);
            fz[p] = fma2(mr3, dz, fz[p]);
        }
    }
}

// Partial sums of source chunk blockIdx.y for the block's targets:
// part[(chunk * 4 + c) * nt + t], c = ax, ay, az, phi (without G).
// Target d of thread x is t = (blockIdx.x * DTG + d) * DB + x.  Each tile's
// coordinates are taken relative to its first source R (FP32 head and
// remainder): sources and targets become (x_hi - R_hi) + (x_lo - R_lo),
// one rounding each, so a pair's separation is a single FP32 difference,
// accurate relative to the distances from R (a tile of consecutive sources
// in key order is compact).  The self pair is masked in the tiles that
// hold a self source of some target of the block (a block-uniform choice;
// with eps = 0, ALL_MASK, in every tile), and the other tiles run without
// the per-pair test.
template <bool ALL_MASK>
__global__ void __launch_bounds__(DB, 6) k_direct(const float4 *__restrict__ hi,
                                                  const float4 *__restrict__ lo, int64_t n,
                                                  const int64_t *__restrict__ targets,
                                                  const uint32_t *__restrict__ inv, int64_t nt,
                                                  float eps2, int64_t chunk,
                                                  double *__restrict__ part,
                                                  DevScalars *__restrict__ sc) {
    __shared__ float4 sr[DTILE];             // {x - R, y - R, z - R, m} of the tile's sources
    __shared__ double acc64[4 * DTG * DB];  // [c][d][thread]: FP64 running sums
    __shared__ int sslot[DTG * DB];         // [d][thread]: key-order slot of each target
    const int x = threadIdx.x;
#pragma unroll
    for (int d = 0; d < DTG; ++d) {
        const int64_t t = ((int64_t)blockIdx.x * DTG + d) * DB + x;
        const bool tv = t < nt;
        int64_t c = tv ? (targets ? targets[t] : t) : 0;
        if (c < 0 || c >= n) {  // a bad caller index: reported, not read
            if (tv && blockIdx.y == 0) atomicOr(&sc->status, ST_BAD_INPUT);
            c = 0;
        }
        sslot[d * DB + x] = (int)inv[c];
#pragma unroll
        for (int k = 0; k < 4; ++k) acc64[(k * DTG + d) * DB + x] = 0.0;
    }
    const f32x2 e2 = dup2(eps2);
    const int64_t s0 = (int64_t)blockIdx.y * chunk;
    const int64_t s1 = min(n, s0 + chunk);
    for (int64_t base = s0; base < s1; base += DTILE) {
        const float4 rh = hi[base], rl = lo[base];  // the tile's reference R
        __syncthreads();
        for (int k = x; k < DTILE; k += DB) {
            const int64_t j = base + k;
            if (j < s1) {
                const float4 a = hi[j], b = lo[j];
                sr[k] = make_float4((a.x - rh.x) + (b.x - rl.x), (a.y - rh.y) + (b.y - rl.y),
                                    (a.z - rh.z) + (b.z - rl.z), a.w);
            }
        }
        const int cnt = (int)min((int64_t)DTILE, s1 - base);
        int ks[DTG];  // each target's self source in this tile, or -1
        bool mine = false;
#pragma unroll
        for (int d = 0; d < DTG; ++d) {
            const int64_t o = (int64_t)sslot[d * DB + x] - base;
            ks[d] = (o >= 0 && o < cnt) ? (int)o : -1;
            mine |= ks[d] >= 0;
        }
        const bool mask = ALL_MASK || __syncthreads_or(mine);
        if (ALL_MASK) __syncthreads();
        // the targets relative to R (their records are read again per tile
        // from L1/L2 rather than kept in registers through the tile loop)
        f32x2 tx[DP], ty[DP], tz[DP];
#pragma unroll
        for (int p = 0; p < DP; ++p) {
            const int i0 = sslot[(2 * p) * DB + x], i1 = sslot[(2 * p + 1) * DB + x];
            const float4 h0 = hi[i0], h1 = hi[i1], l0 = lo[i0], l1 = lo[i1];
            tx[p] = p2((h0.x - rh.x) + (l0.x - rl.x), (h1.x - rh.x) + (l1.x - rl.x));
            ty[p] = p2((h0.y - rh.y) + (l0.y - rl.y), (h1.y - rh.y) + (l1.y - rl.y));
            tz[p] = p2((h0.z - rh.z) + (l0.z - rl.z), (h1.z - rh.z) + (l1.z - rl.z));
        }
        f32x2 fx[DP], fy[DP], fz[DP], fp[DP];
#pragma unroll
        for (int p = 0; p < DP; ++p) fx[p] = fy[p] = fz[p] = fp[p] = 0ull;
        if (mask)
            tile_pairs<true>(sr, cnt, ks, tx, ty, tz, e2, fx, fy, fz, fp);
        else
            tile_pairs<false>(sr, cnt, ks, tx, ty, tz, e2, fx, fy, fz, fp);
#pragma unroll
        for (int p = 0; p < DP; ++p) {
            float v[4][2];
            u2(fx[p], v[0][0], v[0][1]);
            u2(fy[p], v[1][0], v[1][1]);
            u2(fz[p], v[2][0], v[2][1]);
            u2(fp[p], v[3][0], v[3][1]);
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int h = 0; h < 2; ++h) acc64[(k * DTG + 2 * p + h) * DB + x] += (double)v[k][h];
        }
    }
#pragma unroll
    for (int d = 0; d < DTG; ++d) {
        const int64_t t = ((int64_t)blockIdx.x * DTG + d) * DB + x;
        if (t >= nt) continue;
        double *pt = part + (int64_t)blockIdx.y * 4 * nt;
        pt[t] = acc64[(0 * DTG + d) * DB + x];
        pt[nt + t] = acc64[(1 * DTG + d) * DB + x];
        pt[2 * nt + t] = acc64[(2 * DTG + d) * DB + x];
        pt[3 * nt + t] = acc64[(3 * DTG + d) * DB + x];
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
    const int64_t tblocks = (nt + DB * DTG - 1) / (DB * DTG);
    // source chunks: the count (at most MAX_CHUNKS, each chunk at least one
    // tile) whose blocks fill the resident slots of the whole GPU best,
    // counting the idle slots of the last wave
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_direct<false>, DB, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t slots = (int64_t)per_sm * c->sm_count;
    const int64_t max_chunks = std::min<int64_t>(MAX_CHUNKS, (n + DTILE - 1) / DTILE);
    int64_t nchunks = 1;
    double best = -1.0;
    for (int64_t k = 1; k <= max_chunks; ++k) {
        const int64_t blocks = k * tblocks;
        const int64_t waves = (blocks + slots - 1) / slots;
        // filled fraction, with a small preference for more (shorter) chunks
        const double fill = (double)blocks / (double)(waves * slots) + 1e-3 * (double)waves;
        if (blocks >= slots / 2 && fill > best + 1e-9) {
            best = fill;
            nchunks = k;
        }
    }
    if (best < 0.0) nchunks = max_chunks;  // too few targets to fill the GPU: all chunks
    int64_t chunk = (n + nchunks - 1) / nchunks;
    chunk = (chunk + DTILE - 1) / DTILE * DTILE;
    nchunks = (n + chunk - 1) / chunk;
    if (ensure(c->dir_part, (size_t)(nchunks * 4 * nt))) return BONSAI_ENOMEM;
    k_inverse_id<<<grid_for(n, 256, c->sm_count * 16), 256, 0, c->stream>>>(c->id.p, n, c->inv_id.p);
    const dim3 grid((unsigned)tblocks, (unsigned)nchunks);
    if (eps > 0.0f)
        k_direct<false><<<grid, DB, 0, c->stream>>>(c->body_hi.p, c->body_lo.p, n, targets,
                                                    c->inv_id.p, nt, eps * eps, chunk,
                                                    c->dir_part.p, c->dsc);
    else
        k_direct<true><<<grid, DB, 0, c->stream>>>(c->body_hi.p, c->body_lo.p, n, targets,
                                                   c->inv_id.p, nt, eps * eps, chunk,
                                                   c->dir_part.p, c->dsc);
    k_direct_final<<<grid_for(nt, 256, c->sm_count * 16), 256, 0, c->stream>>>(
        c->dir_part.p, (int)nchunks, nt, c->prm.G, acc, pot);
    c->launches += 3;
    return cudaPeekAtLastError() == cudaSuccess ? BONSAI_OK : BONSAI_ECUDA;
}

}  // namespace bgb
