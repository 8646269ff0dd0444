// sort.cu -- stable LSD radix sort of (key, index) pairs, an exclusive
// scan, and the gathers that move particle state into key order
// (Table 2 "Sorting SFC").
//
// The sort is 8 passes of 8 bits after one count of all digits; each pass
// is one kernel (a one-sweep pass with decoupled look-back, below).
// Stability plus the index payload starting at 0..n-1 makes the order
// identical to sorting by (key, index).
#include <utility>

#include "internal.cuh"

namespace bgb {

namespace {

// SORT_BLOCK, SORT_IPT, SORT_TILE, SCAN_BLOCK, SCAN_IPT and SCAN_TILE are
// in internal.cuh: the scratch sizes of every caller derive from them.
// ---- one-sweep LSD radix sort ----
// Digit d of pass p is bits [8p, 8p + 8) of the key.  k_sort_counts counts
// every pass's digits in one read of the keys.  Each pass is then a single
// kernel over tiles of SORT_TILE pairs, taken in launch order from a
// counter: a tile ranks its pairs by digit (warp match/popc against
// warp-private counts, so equal digits keep their input order), publishes
// its per-digit counts, and finds its global offset per digit by a
// decoupled look-back over the descriptors of the tiles before it (the
// exclusive sum of their counts), stopping at the first tile that already
// published its inclusive prefix.  A descriptor is one 64-bit word: the pass
// (plus one) in bits 56-63, the kind (1 = this tile's count, 2 = inclusive
// prefix) in bits 54-55, the value below; words of another pass read as not
// yet published, and the whole array is cleared once per sort.  A tile
// waits only on tiles that started before it, so the look-back always
// ends; its polling is bounded all the same, and a wait that gives up sets
// ST_TIMEOUT.
constexpr int SORT_WARPS = SORT_BLOCK / 32;
constexpr int PER_WARP = SORT_TILE / SORT_WARPS;  // contiguous pairs of one warp
constexpr int ROUNDS = PER_WARP / 32;
constexpr uint64_t DESC_VALUE = (1ull << 54) - 1ull;
constexpr uint64_t DESC_COUNT = 1ull << 54, DESC_PREFIX = 2ull << 54;
constexpr uint32_t LOOKBACK_SPINS = 1u << 22;
constexpr int LOOKBACK_W = 8;  // predecessors read per look-back round trip

__device__ inline uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// The digit counts of all eight passes: cnt[p * 256 + d] (zeroed by the
// caller), from block-private shared counters.  Per warp and pass, a digit
// shared by all 32 lanes (the usual case for the high digits of nearly
// sorted keys) is one add; otherwise every lane adds its own.
__global__ void __launch_bounds__(SORT_BLOCK) k_sort_counts(const uint64_t *__restrict__ kin,
                                                            int64_t n, uint32_t *__restrict__ cnt) {
    __shared__ uint32_t sc[8][256];
    for (int k = threadIdx.x; k < 8 * 256; k += SORT_BLOCK) (&sc[0][0])[k] = 0u;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * SORT_BLOCK;
    const int64_t end = (n + 31) / 32 * 32;  // whole warps take part in the votes
    constexpr int U = 4;  // keys loaded ahead, so that their loads overlap
    for (int64_t i0 = (int64_t)blockIdx.x * SORT_BLOCK + threadIdx.x; i0 < end; i0 += U * stride) {
        uint64_t ks[U];
        bool vs[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * stride;
            vs[u] = i < n;
            ks[u] = vs[u] ? kin[i] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (i0 + u * stride >= end) break;  // uniform within a warp
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                const uint32_t d = vs[u] ? (uint32_t)(ks[u] >> (8 * p)) & 255u : 256u;
                const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
                if (__all_sync(0xffffffffu, d == d0)) {
                    if ((threadIdx.x & 31) == 0 && d0 < 256u) atomicAdd(&sc[p][d0], 32u);
                } else if (d < 256u) {
                    atomicAdd(&sc[p][d], 1u);
                }
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 8 * 256; k += SORT_BLOCK) {
        const uint32_t v = (&sc[0][0])[k];
        if (v) atomicAdd(cnt + k, v);
    }
}

// One pass (digit shift 8 * pass) over one tile per block.  Shared memory:
// the tile's pairs in digit order (sk, sv), the warps' digit counts, and per
// digit the tile's local start and global base.
struct SweepShared {
    uint64_t sk[SORT_TILE];
    uint32_t sv[SORT_TILE];
    uint32_t wh[SORT_WARPS][256];
    uint32_t lstart[256], gbase[256], wsum[SORT_WARPS];
    uint32_t tile;
};

__global__ void __launch_bounds__(SORT_BLOCK, 3) k_sort_pass(const uint64_t *__restrict__ kin,
                                                          const uint32_t *__restrict__ vin,
                                                          uint64_t *__restrict__ kout,
                                                          uint32_t *__restrict__ vout, int64_t n,
                                                          int pass, uint64_t *desc,
                                                          const uint32_t *__restrict__ cnt,
                                                          uint32_t *tile_counter,
                                                          int32_t *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SweepShared &S = *reinterpret_cast<SweepShared *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int shift = 8 * pass;
    const uint32_t lt = lanemask_lt();
    if (tid == 0) S.tile = atomicAdd(tile_counter + pass, 1u);
#pragma unroll
    for (int w = 0; w < SORT_WARPS; ++w) S.wh[w][tid] = 0u;
    __syncthreads();
    const uint32_t tile = S.tile;
    const int64_t t0 = (int64_t)tile * SORT_TILE;
    // 1. ranks within the warp's contiguous run.  The digits of all rounds
    // are loaded first, so that their loads are in flight together (the
    // keys are read again in step 3, from L2, rather than held in registers
    // through the look-back).
    uint32_t dr[ROUNDS];  // digit (bits 0-8, 256 = past the end) | rank in warp << 9
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const int64_t i = t0 + warp * PER_WARP + r * 32 + lane;
        dr[r] = i < n ? (uint32_t)(kin[i] >> shift) & 255u : 256u;
    }
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const uint32_t d = dr[r];
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t prev = d < 256u ? S.wh[warp][d] : 0u;
        dr[r] = d | ((prev + __popc(peers & lt)) << 9);
        __syncwarp();
        if (d < 256u && (peers & lt) == 0u) S.wh[warp][d] = prev + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // 2. digit tid: the warps' offsets within the digit and the tile's count
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < SORT_WARPS; ++w) {
        const uint32_t x = S.wh[w][tid];
        S.wh[w][tid] = c;
        c += x;
    }
    // publish this tile's count, then look back for the exclusive prefix
    const uint64_t epoch = (uint64_t)(pass + 1) << 56;
    uint64_t *my = desc + (int64_t)tile * 256 + tid;
    volatile uint64_t *vmy = my;
    uint64_t excl = 0;
    if (tile == 0) {
        *vmy = epoch | DESC_PREFIX | (uint64_t)c;
    } else {
        *vmy = epoch | DESC_COUNT | (uint64_t)c;
        // LOOKBACK_W predecessors per round trip (independent loads), taken
        // nearest first; an unpublished one is polled again from there
        int64_t t = (int64_t)tile - 1;
        uint32_t spins = 0;
        while (t >= 0) {
            uint64_t v[LOOKBACK_W];
#pragma unroll
            for (int w = 0; w < LOOKBACK_W; ++w)  // before tile 0: a zero prefix
                v[w] = t - w >= 0 ? *(volatile uint64_t *)(desc + (t - w) * 256 + tid)
                                  : (epoch | DESC_PREFIX);
            int used = LOOKBACK_W;
            bool done = false;
#pragma unroll
            for (int w = 0; w < LOOKBACK_W; ++w) {
                if ((v[w] & (255ull << 56)) != epoch) {
                    used = w;
                    break;
                }
                excl += v[w] & DESC_VALUE;
                if ((v[w] & (3ull << 54)) == DESC_PREFIX) {
                    done = true;
                    break;
                }
            }
            if (done) break;
            t -= used;
            if (used < LOOKBACK_W) {
                if (++spins > LOOKBACK_SPINS || (*(volatile int32_t *)status & ST_TIMEOUT)) {
                    atomicOr(status, ST_TIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
        }
        *vmy = epoch | DESC_PREFIX | (excl + c);
    }
    // global base of digit tid: pairs of smaller digits in all tiles, plus
    // pairs of this digit in the tiles before this one
    uint32_t inc = __ldg(cnt + pass * 256 + tid), lc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t a = __shfl_up_sync(0xffffffffu, inc, o);
        const uint32_t b = __shfl_up_sync(0xffffffffu, lc, o);
        if (lane >= o) {
            inc += a;
            lc += b;
        }
    }
    // inc: inclusive scan of the global counts over this warp's digits; lc:
    // the same for the tile's counts
    __shared__ uint32_t gsum[SORT_WARPS];
    if (lane == 31) {
        gsum[warp] = inc;
        S.wsum[warp] = lc;
    }
    __syncthreads();
    uint32_t gadd = 0, ladd = 0;
    for (int w = 0; w < warp; ++w) {
        gadd += gsum[w];
        ladd += S.wsum[w];
    }
    const uint32_t gcount = __ldg(cnt + pass * 256 + tid);
    S.gbase[tid] = (gadd + inc - gcount) + (uint32_t)excl;
    S.lstart[tid] = ladd + lc - c;
    __syncthreads();
    // 3. the tile's pairs in digit order in shared memory (values read now)
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const uint32_t d = dr[r] & 511u;
        if (d < 256u) {
            const int64_t i = t0 + warp * PER_WARP + r * 32 + lane;
            const uint32_t p = S.lstart[d] + S.wh[warp][d] + (dr[r] >> 9);
            S.sk[p] = kin[i];
            S.sv[p] = vin[i];
        }
    }
    __syncthreads();
    // 4. each digit's pairs as one contiguous run of the output
    const int64_t left = n - t0;
    const int nt = left < SORT_TILE ? (int)left : SORT_TILE;
    for (int p = tid; p < nt; p += SORT_BLOCK) {
        const uint64_t k = S.sk[p];
        const uint32_t d = (uint32_t)(k >> shift) & 255u;
        const int64_t dst = (int64_t)S.gbase[d] + (p - (int64_t)S.lstart[d]);
        kout[dst] = k;
        vout[dst] = S.sv[p];
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

// Re-sort of the context's state.  With inv (the exact path), perm holds the
// caller index of each new slot and inv the old slot of each caller index.
// Without it, perm holds the old slot of each new slot and id_o the caller
// index of each old slot: the sort ran on (key, old slot) pairs in old-slot
// order, so equal keys came out in old-slot order, and each slot of a run of
// equal keys takes instead the run's element whose caller index has the
// slot's rank in the run, which makes the order (key, caller index).  A run
// longer than TIE_RUN_MAX is left alone and reported (ST_LONG_TIES): the
// caller then sorts again by the exact path.
constexpr int TIE_RUN_MAX = 32;
__global__ void __launch_bounds__(256) k_gather_step(
    const double *__restrict__ pos_o, const double *__restrict__ vel_o,
    const double *__restrict__ mass_o, const uint32_t *__restrict__ inv,
    const uint32_t *__restrict__ id_o, const uint32_t *__restrict__ perm,
    const uint64_t *__restrict__ key, int64_t n, double *__restrict__ pos,
    double *__restrict__ vel, double *__restrict__ mass, uint32_t *__restrict__ id,
    int32_t *status) {
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        uint32_t c, j;
        if (inv) {
            c = perm[i];
            j = inv[c];
        } else {
            j = perm[i];
            const uint64_t k = key[i];
            if ((i > 0 && key[i - 1] == k) || (i + 1 < n && key[i + 1] == k)) {
                int64_t s = i, e = i + 1;  // the run [s, e), looked for up to TIE_RUN_MAX + 1
                while (s > 0 && e - s <= TIE_RUN_MAX && key[s - 1] == k) --s;
                while (e < n && e - s <= TIE_RUN_MAX && key[e] == k) ++e;
                if (e - s > TIE_RUN_MAX) {
                    atomicOr(status, ST_LONG_TIES);
                } else {
                    for (int64_t a = s; a < e; ++a) {  // the element of rank i - s
                        const uint32_t ca = id_o[perm[a]];
                        int64_t r = 0;
                        for (int64_t b = s; b < e; ++b) r += id_o[perm[b]] < ca ? 1 : 0;
                        if (r == i - s) {
                            j = perm[a];
                            break;
                        }
                    }
                }
            }
            c = id_o[j];
        }
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

// The sort on explicit buffers: (ka, va) hold the input and the result,
// (kb, vb) are the second ping-pong half, scratch holds
// sort_scratch_elems(n) entries (cleared here; 8-byte aligned), status
// receives ST_TIMEOUT if a look-back wait gave up.  Returns the number of
// kernels launched.
int radix_sort_pairs_into(cudaStream_t s, int sm_count, int64_t n, uint64_t *ka, uint64_t *kb,
                          uint32_t *va, uint32_t *vb, uint32_t *scratch, int32_t *status) {
    const int64_t tiles = (n + SORT_TILE - 1) / SORT_TILE;
    uint64_t *desc = reinterpret_cast<uint64_t *>(scratch);
    uint32_t *cnt = scratch + 2 * 256 * tiles;
    uint32_t *tile_counter = cnt + 8 * 256;
    cudaMemsetAsync(scratch, 0, sort_scratch_elems(n) * sizeof(uint32_t), s);
    k_sort_counts<<<grid_for(n, SORT_BLOCK * 4, sm_count * 8), SORT_BLOCK, 0, s>>>(ka, n, cnt);
    cudaFuncSetAttribute(k_sort_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(SweepShared));
    for (int pass = 0; pass < 8; ++pass) {
        k_sort_pass<<<(unsigned)tiles, SORT_BLOCK, sizeof(SweepShared), s>>>(
            ka, va, kb, vb, n, pass, desc, cnt, tile_counter, status);
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    // eight passes: the result is back in (ka, va)
    return 9;
}

void radix_sort_pairs(bonsai_ctx *c, int64_t n) {
    c->launches += radix_sort_pairs_into(c->stream, c->sm_count, n, c->key.p, c->key2.p, c->val.p,
                                         c->val2.p, c->hist.p, &c->dsc->status);
}

void launch_gather_build(bonsai_ctx *c, const double *pos, const double *mass, int64_t n) {
    k_gather_build<<<grid_for(n, 256, c->sm_count * 16), 256, 0, c->stream>>>(
        pos, mass, c->val.p, n, c->pos.p, c->vel.p, c->mass.p, c->id.p);
    c->launches += 1;
}

void launch_gather_step(bonsai_ctx *c, int64_t n, bool exact) {
    k_gather_step<<<grid_for(n, 256, c->sm_count * 16), 256, 0, c->stream>>>(
        c->pos.p, c->vel.p, c->mass.p, exact ? c->inv_id.p : nullptr, c->id.p, c->val.p,
        c->key.p, n, c->pos2.p, c->vel2.p, c->mass2.p, c->id2.p, &c->dsc->status);
    c->launches += 1;
    std::swap(c->pos, c->pos2);
    std::swap(c->vel, c->vel2);
    std::swap(c->mass, c->mass2);
    std::swap(c->id, c->id2);
}

}  // namespace bgb
