// sort.cu -- stable LSD radix sort of (key, index) pairs, an exclusive
// scan, and the gathers that move particle state into key order
// (Table 2 "Sorting SFC").
//
// The sort is 8 passes of 8 bits.  Each pass is a per-tile histogram, an
// exclusive scan of the digit-major histogram table (which yields every
// tile's output offset per digit), and a stable scatter that ranks the
// tile's keys with warp match/popc and writes them digit by digit.  Stability plus the index payload
// starting at 0..n-1 makes the order identical to sorting by (key, index).
#include <utility>

#include "internal.cuh"

namespace bgb {

namespace {

// SORT_BLOCK, SORT_IPT, SORT_TILE, SCAN_BLOCK, SCAN_IPT and SCAN_TILE are
// in internal.cuh: the scratch sizes of every caller derive from them.
constexpr int SORT_WARPS = SORT_BLOCK / 32;

__device__ inline uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__global__ void __launch_bounds__(SORT_BLOCK) k_hist(const uint64_t *__restrict__ kin, int64_t n,
                                                     int shift, uint32_t *__restrict__ hist,
                                                     int nb) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    for (int r = 0; r < SORT_IPT; ++r) {
        int64_t i = base + r * SORT_BLOCK + threadIdx.x;
        uint32_t d = i < n ? (uint32_t)(kin[i] >> shift) & 255u : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (d < 256u && (peers & lanemask_lt()) == 0u) atomicAdd(&cnt[d], __popc(peers));
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one tile, in two halves of 2048 pairs.  Each warp owns
// a contiguous run of 256 pairs of the half and ranks them by digit with
// match_any against warp-private digit counts; a scan over the digits then
// gives every pair its place in a digit-sorted copy of the half in shared
// memory, from which the pairs of each digit are written to global memory
// as one contiguous run (instead of one scattered store per pair).  Warps
// own consecutive positions, so the order within a digit is the input order.
__global__ void __launch_bounds__(SORT_BLOCK) k_scatter(const uint64_t *__restrict__ kin,
                                                        const uint32_t *__restrict__ vin,
                                                        uint64_t *__restrict__ kout,
                                                        uint32_t *__restrict__ vout, int64_t n,
                                                        int shift,
                                                        const uint32_t *__restrict__ offs,
                                                        int nb) {
    constexpr int HALF = SORT_TILE / 2;
    constexpr int PER_WARP = HALF / SORT_WARPS;
    constexpr int ROUNDS = PER_WARP / 32;
    __shared__ uint64_t sk[HALF];
    __shared__ uint32_t sv[HALF];
    __shared__ uint32_t wh[SORT_WARPS][256];
    __shared__ uint32_t gbase[256], lstart[256], wsum[SORT_WARPS];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lt = lanemask_lt();
    gbase[tid] = offs[(int64_t)tid * nb + blockIdx.x];
    for (int h = 0; h < 2; ++h) {
        const int64_t h0 = (int64_t)blockIdx.x * SORT_TILE + (int64_t)h * HALF;
#pragma unroll
        for (int w = 0; w < SORT_WARPS; ++w) wh[w][tid] = 0u;
        __syncthreads();
        uint64_t key[ROUNDS];
        uint32_t val[ROUNDS], dg[ROUNDS], rk[ROUNDS];
#pragma unroll
        for (int r = 0; r < ROUNDS; ++r) {
            const int64_t i = h0 + warp * PER_WARP + r * 32 + lane;
            const bool valid = i < n;
            key[r] = valid ? kin[i] : 0ull;
            val[r] = valid ? vin[i] : 0u;
            const uint32_t d = valid ? (uint32_t)(key[r] >> shift) & 255u : 256u;
            dg[r] = d;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const uint32_t prev = d < 256u ? wh[warp][d] : 0u;
            rk[r] = prev + __popc(peers & lt);
            __syncwarp();
            if (d < 256u && (peers & lt) == 0u) wh[warp][d] = prev + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // digit tid: offsets of the warps' runs, and the half's count
        uint32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < SORT_WARPS; ++w) {
            const uint32_t c = wh[w][tid];
            wh[w][tid] = cnt;
            cnt += c;
        }
        // exclusive scan of the counts over the 256 digits
        uint32_t inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        uint32_t add = 0;
        for (int w = 0; w < warp; ++w) add += wsum[w];
        lstart[tid] = add + inc - cnt;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < ROUNDS; ++r) {
            const uint32_t d = dg[r];
            if (d < 256u) {
                const uint32_t p = lstart[d] + wh[warp][d] + rk[r];
                sk[p] = key[r];
                sv[p] = val[r];
            }
        }
        __syncthreads();
        const int64_t left = n - h0;
        const int nh = left <= 0 ? 0 : (left < HALF ? (int)left : HALF);
        for (int p = tid; p < nh; p += SORT_BLOCK) {
            const uint64_t k = sk[p];
            const uint32_t d = (uint32_t)(k >> shift) & 255u;
            const uint32_t dst = gbase[d] + ((uint32_t)p - lstart[d]);
            kout[dst] = k;
            vout[dst] = sv[p];
        }
        __syncthreads();
        gbase[tid] += cnt;
    }
}

// Exclusive scan of one tile per block; block sums go to bsum.
// in and out may alias (the sort scans its histogram table in place).
__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_tile(const uint32_t *in, uint32_t *out, int64_t n,
                                                          uint32_t *__restrict__ bsum) {
    __shared__ uint32_t wsum[SCAN_BLOCK / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IPT;
    uint32_t v[SCAN_IPT], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0u;
        s += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = wsum[lane];
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        wsum[lane] = wi - w;
        if (lane == 31 && bsum) bsum[blockIdx.x] = wi;
    }
    __syncthreads();
    uint32_t run = wsum[warp] + inc - s;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_add(uint32_t *__restrict__ out, int64_t n,
                                                         const uint32_t *__restrict__ boff) {
    const uint32_t add = boff[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int k = threadIdx.x; k < SCAN_TILE; k += SCAN_BLOCK)
        if (base + k < n) out[base + k] += add;
}

__global__ void k_scan_total(const uint32_t *in, const uint32_t *out, int64_t n, uint32_t *total) {
    *total = n > 0 ? out[n - 1] + in[n - 1] : 0u;
}

// Returns the number of kernels launched.
int scan_rec(cudaStream_t s, const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp) {
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb <= 1) {
        k_scan_tile<<<1, SCAN_BLOCK, 0, s>>>(in, out, n, nullptr);
        return 1;
    }
    uint32_t *bsum = tmp, *boff = tmp + nb;
    k_scan_tile<<<(unsigned)nb, SCAN_BLOCK, 0, s>>>(in, out, n, bsum);
    int k = scan_rec(s, bsum, boff, nb, tmp + 2 * nb);
    k_scan_add<<<(unsigned)nb, SCAN_BLOCK, 0, s>>>(out, n, boff);
    return k + 2;
}

__global__ void __launch_bounds__(256) k_gather_build(const double *__restrict__ pos_c,
                                                      const double *__restrict__ mass_c,
                                                      const uint32_t *__restrict__ perm, int64_t n,
                                                      double *__restrict__ pos,
                                                      double *__restrict__ vel,
                                                      double *__restrict__ mass,
                                                      uint32_t *__restrict__ id) {
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        uint32_t j = perm[i];
        pos[i] = pos_c[j];
        pos[n + i] = pos_c[n + j];
        pos[2 * n + i] = pos_c[2 * n + j];
        vel[i] = 0.0;
        vel[n + i] = 0.0;
        vel[2 * n + i] = 0.0;
        mass[i] = mass_c[j];
        id[i] = j;
    }
}

// Re-sort of the context's state: perm holds the caller index of each new
// slot, inv the old slot of each caller index.
__global__ void __launch_bounds__(256) k_gather_step(
    const double *__restrict__ pos_o, const double *__restrict__ vel_o,
    const double *__restrict__ mass_o, const uint32_t *__restrict__ inv,
    const uint32_t *__restrict__ perm, int64_t n, double *__restrict__ pos,
    double *__restrict__ vel, double *__restrict__ mass, uint32_t *__restrict__ id) {
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const uint32_t c = perm[i];
        const uint32_t j = inv[c];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            pos[d * n + i] = pos_o[d * n + j];
            vel[d * n + i] = vel_o[d * n + j];
        }
        mass[i] = mass_o[j];
        id[i] = c;
    }
}

}  // namespace

void exclusive_scan_u32(bonsai_ctx *c, const uint32_t *in, uint32_t *out, int64_t n,
                        uint32_t *total_dev) {
    if (n > 0) c->launches += scan_rec(c->stream, in, out, n, c->scan_tmp.p);
    if (total_dev) {
        k_scan_total<<<1, 1, 0, c->stream>>>(in, out, n, total_dev);
        c->launches += 1;
    }
}

int exclusive_scan_into(cudaStream_t s, const uint32_t *in, uint32_t *out, int64_t n,
                        uint32_t *tmp, uint32_t *total_dev) {
    int launches = n > 0 ? scan_rec(s, in, out, n, tmp) : 0;
    if (total_dev) {
        k_scan_total<<<1, 1, 0, s>>>(in, out, n, total_dev);
        launches += 1;
    }
    return launches;
}

// The same eight passes on explicit buffers: (ka, va) hold the input and the
// result, (kb, vb) are the second ping-pong half, hist holds
// sort_hist_elems(n) entries and tmp scan_tmp_elems(256 * tiles) entries.
// Returns the number of kernels launched.
int radix_sort_pairs_into(cudaStream_t s, int64_t n, uint64_t *ka, uint64_t *kb, uint32_t *va,
                          uint32_t *vb, uint32_t *hist, uint32_t *tmp) {
    const int nb = (int)((n + SORT_TILE - 1) / SORT_TILE);
    const int64_t nh = 256ll * nb;
    int launches = 0;
    for (int shift = 0; shift < 64; shift += 8) {
        k_hist<<<nb, SORT_BLOCK, 0, s>>>(ka, n, shift, hist, nb);
        launches += scan_rec(s, hist, hist, nh, tmp) + 2;
        k_scatter<<<nb, SORT_BLOCK, 0, s>>>(ka, va, kb, vb, n, shift, hist, nb);
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    return launches;
}

void radix_sort_pairs(bonsai_ctx *c, int64_t n) {
    const int nb = (int)((n + SORT_TILE - 1) / SORT_TILE);
    const int64_t nh = 256ll * nb;
    uint64_t *ka = c->key.p, *kb = c->key2.p;
    uint32_t *va = c->val.p, *vb = c->val2.p;
    for (int shift = 0; shift < 64; shift += 8) {
        k_hist<<<nb, SORT_BLOCK, 0, c->stream>>>(ka, n, shift, c->hist.p, nb);
        c->launches += scan_rec(c->stream, c->hist.p, c->hist.p, nh, c->scan_tmp.p) + 2;
        k_scatter<<<nb, SORT_BLOCK, 0, c->stream>>>(ka, va, kb, vb, n, shift, c->hist.p, nb);
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    // eight passes: the result is back in key/val
}

void launch_gather_build(bonsai_ctx *c, const double *pos, const double *mass, int64_t n) {
    k_gather_build<<<grid_for(n, 256, c->sm_count * 16), 256, 0, c->stream>>>(
        pos, mass, c->val.p, n, c->pos.p, c->vel.p, c->mass.p, c->id.p);
    c->launches += 1;
}

void launch_gather_step(bonsai_ctx *c, int64_t n) {
    k_gather_step<<<grid_for(n, 256, c->sm_count * 16), 256, 0, c->stream>>>(
        c->pos.p, c->vel.p, c->mass.p, c->inv_id.p, c->val.p, n, c->pos2.p, c->vel2.p, c->mass2.p,
        c->id2.p);
    c->launches += 1;
    std::swap(c->pos, c->pos2);
    std::swap(c->vel, c->vel2);
    std::swap(c->mass, c->mass2);
    std::swap(c->id, c->id2);
}

}  // namespace bgb
