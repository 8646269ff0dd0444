// keys.cu -- bounding cube reduction and Peano-Hilbert keys (Sec. III.B.1:
// the bounding box maps coordinates to PH keys; Fig. 2 shows the curve).
//
// Both kernels stream the FP64 SoA positions once.  Every FP64 operation
// that feeds a key is an explicit round-to-nearest intrinsic so the keys are
// bit-identical to any IEEE implementation of the same formula; the Hilbert
// transform runs as a table-driven state machine, two levels per lookup.
#include <math.h>

#include <climits>
#include <cmath>

#include "internal.cuh"

namespace bgb {

namespace {

constexpr int BOX_BLOCK = 256;

__device__ inline double warp_min(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}
__device__ inline double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Per-block min/max of x, y, z plus an input check (finite positions,
// finite positive masses).  The minima and maxima are taken on the
// order-preserving integer images of the doubles and the checks on their
// bit patterns, so the loop uses no FP64 instruction.
__device__ inline long long warp_min_k(long long v) {
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}
__device__ inline long long warp_max_k(long long v) {
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

__global__ void __launch_bounds__(BOX_BLOCK) k_box_partial(const double *__restrict__ pos,
                                                           const double *__restrict__ mass,
                                                           int64_t n, BoxPartial *part) {
    constexpr long long EXP = 0x7ff0000000000000ll;  // exponent field: all ones = inf / NaN
    long long mn[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, mx[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)BOX_BLOCK + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * BOX_BLOCK) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double v = pos[d * n + i];
            bad |= (__double_as_longlong(v) & EXP) == EXP;
            const long long k = order_key(v);
            mn[d] = min(mn[d], k);
            mx[d] = max(mx[d], k);
        }
        // positive, finite and not zero: the bit pattern lies in (0, +inf)
        const long long mb = __double_as_longlong(mass[i]);
        bad |= !(mb > 0ll && mb < EXP);
    }
    __shared__ long long smn[3][BOX_BLOCK / 32], smx[3][BOX_BLOCK / 32];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        long long a = warp_min_k(mn[d]), b = warp_max_k(mx[d]);
        if (l == 0) { smn[d][w] = a; smx[d][w] = b; }
    }
    if (bad) atomicOr(&sbad, 1);
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            long long a = l < BOX_BLOCK / 32 ? smn[d][l] : LLONG_MAX;
            long long b = l < BOX_BLOCK / 32 ? smx[d][l] : LLONG_MIN;
            a = warp_min_k(a);
            b = warp_max_k(b);
            if (l == 0) {
                part[blockIdx.x].mn[d] = from_order_key(a);
                part[blockIdx.x].mx[d] = from_order_key(b);
            }
        }
        if (l == 0) part[blockIdx.x].bad = sbad;
    }
}

// Final reduction and the cube: side L = (largest extent) * (1 + 2^-20)
// (1 when every point coincides), centred on the box; scale = 2^21 / L.
__global__ void __launch_bounds__(BOX_BLOCK) k_box_final(const BoxPartial *part, int nb,
                                                         DevScalars *sc) {
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    int bad = 0;
    for (int b = threadIdx.x; b < nb; b += BOX_BLOCK) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            mn[d] = fmin(mn[d], part[b].mn[d]);
            mx[d] = fmax(mx[d], part[b].mx[d]);
        }
        bad |= part[b].bad;
    }
    __shared__ double smn[3][BOX_BLOCK / 32], smx[3][BOX_BLOCK / 32];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double a = warp_min(mn[d]), b = warp_max(mx[d]);
        if (l == 0) { smn[d][w] = a; smx[d][w] = b; }
    }
    if (bad) atomicOr(&sbad, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        double lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            lo[d] = smn[d][0];
            hi[d] = smx[d][0];
            for (int k = 1; k < BOX_BLOCK / 32; ++k) {
                lo[d] = fmin(lo[d], smn[d][k]);
                hi[d] = fmax(hi[d], smx[d][k]);
            }
        }
        double ext = __dsub_rn(hi[0], lo[0]);
        double e1 = __dsub_rn(hi[1], lo[1]), e2 = __dsub_rn(hi[2], lo[2]);
        if (e1 > ext) ext = e1;
        if (e2 > ext) ext = e2;
        double L = __dmul_rn(ext, 1.0 + 0x1p-20);
        if (ext == 0.0) L = 1.0;
        for (int d = 0; d < 3; ++d) {
            double w = __dsub_rn(hi[d], lo[d]);
            sc->lo[d] = __dsub_rn(lo[d], __dmul_rn(__dsub_rn(L, w), 0.5));
        }
        sc->L = L;
        sc->scale = __ddiv_rn(0x1p21, L);
        for (int d = 0; d < 3; ++d) {
            sc->mn[d] = lo[d];
            sc->mx[d] = hi[d];
        }
        if (sbad) atomicOr(&sc->status, ST_BAD_INPUT);
    }
}

// floor((x - lo) * scale) clamped to [0, 2^21 - 1], each FP64 step rounded
// to nearest.  The floor and the clamp are taken on the bit pattern of the
// product, on the integer pipes: negative values (and -0) and values below
// 1 give 0, values of 2^21 or more give 2^21 - 1, and otherwise the
// mantissa with its leading bit, shifted right by 52 minus the exponent, is
// the integer part.  (A NaN, which the input check rejects, gives 2^21 - 1.)
__device__ inline uint32_t quantise(double x, double lo, double scale) {
    const long long b = __double_as_longlong(__dmul_rn(__dsub_rn(x, lo), scale));
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    if (b < 0 || e < 0) return 0u;
    if (e >= KEY_BITS) return (1u << KEY_BITS) - 1u;
    const unsigned long long m = ((unsigned long long)b & 0xfffffffffffffull) | (1ull << 52);
    return (uint32_t)(m >> (52 - e));
}

}  // namespace

// Hilbert index of a 21-bit cell after J. Skilling, "Programming the Hilbert
// curve" (AIP Conf. Proc. 707, 2004): the transpose form, then bit
// interleaving with axis 0 most significant in each 3-bit digit.
//
// Evaluated as a finite-state machine over the levels, from the top.  At
// each level Skilling's loop reads one bit per axis and then only inverts
// the lower bits of axis 0 or swaps the lower bits of axis 0 with those of
// axis i, the same for every lower bit; so the lower bits of the current
// axes are always the original ones permuted (pi) and inverted (m), and the
// final Gray step adds one bit of state, the parity P of the Gray code's
// last axis above the level.  A state is (pi, m, P): 6 x 8 x 2 = 96 codes
// (48 reachable).  With c_a = o_{pi(a)} ^ m_a the level's current bits (o
// the original ones), the key digit is (g0 ^ P, g1 ^ P, g2 ^ P) with g0 =
// c0, g1 = c0 ^ c1, g2 = c0 ^ c1 ^ c2; then P ^= g2, and for axis i = 0, 1,
// 2: if c_i, m_0 is flipped, else (i > 0) the entries of axes 0 and i of
// (pi, m) are swapped.
namespace {

// The six permutations of three axes, 2 bits per axis (pi(0) lowest).
__device__ __forceinline__ uint32_t perm_code(int k) {
    constexpr uint32_t P[6] = {0u | 1u << 2 | 2u << 4, 0u | 2u << 2 | 1u << 4,
                               1u | 0u << 2 | 2u << 4, 1u | 2u << 2 | 0u << 4,
                               2u | 0u << 2 | 1u << 4, 2u | 1u << 2 | 0u << 4};
    return P[k];
}

// One level: state s = perm index * 16 + m * 2 + P, original bits o (axis a
// in bit a) -> digit (3 bits) | next state << 3.
__device__ uint32_t ph_level(uint32_t s, uint32_t o) {
    uint32_t pi = perm_code((int)(s >> 4));
    uint32_t m = (s >> 1) & 7u, P = s & 1u;
    uint32_t c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) c[a] = ((o >> ((pi >> (2 * a)) & 3u)) & 1u) ^ ((m >> a) & 1u);
    const uint32_t g0 = c[0], g1 = c[0] ^ c[1], g2 = c[0] ^ c[1] ^ c[2];
    const uint32_t digit = ((g0 ^ P) << 2) | ((g1 ^ P) << 1) | (g2 ^ P);
    P ^= g2;
    if (c[0]) m ^= 1u;
#pragma unroll
    for (int i = 1; i < 3; ++i) {
        if (c[i]) {
            m ^= 1u;
        } else {  // swap axes 0 and i of pi and m
            const uint32_t p0 = pi & 3u, pii = (pi >> (2 * i)) & 3u;
            pi = (pi & ~(3u | (3u << (2 * i)))) | pii | (p0 << (2 * i));
            const uint32_t m0 = m & 1u, mi = (m >> i) & 1u;
            m = (m & ~(1u | (1u << i))) | mi | (m0 << i);
        }
    }
    uint32_t k = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j)
        if (perm_code(j) == pi) k = (uint32_t)j;
    return digit | ((k * 16u + m * 2u + P) << 3);
}

constexpr int PH_STATES = 96;

}  // namespace

// Spread the low 21 bits of v to every third bit of a 64-bit word.
__device__ inline uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// The machine's tables in shared memory: one level per entry (t1[s * 8 +
// o]) and two levels per entry (t2[s * 64 + (o_high << 3 | o_low)] = 6
// digit bits | next state << 6), built by each block from ph_level.
struct PhTables {
    uint16_t t1[PH_STATES * 8];
    uint16_t t2[PH_STATES * 64];
};

__device__ void ph_build(PhTables &T) {
    for (int k = threadIdx.x; k < PH_STATES * 8; k += blockDim.x)
        T.t1[k] = (uint16_t)ph_level((uint32_t)(k >> 3), (uint32_t)(k & 7));
    __syncthreads();
    for (int k = threadIdx.x; k < PH_STATES * 64; k += blockDim.x) {
        const uint32_t s = (uint32_t)k >> 6, hi = ((uint32_t)k >> 3) & 7u, lo = (uint32_t)k & 7u;
        const uint32_t e1 = T.t1[s * 8 + hi], e2 = T.t1[(e1 >> 3) * 8 + lo];
        T.t2[k] = (uint16_t)((((e1 & 7u) << 3) | (e2 & 7u)) | ((e2 >> 3) << 6));
    }
    __syncthreads();
}

// The key of cell (x0, x1, x2): the top level with t1, then ten pairs of
// levels with t2, reading the original bits from the Morton interleaving
// (axis a in bit a of each 3-bit group).
__device__ __forceinline__ uint64_t ph_key(const PhTables &T, uint32_t x0, uint32_t x1,
                                           uint32_t x2) {
    const uint64_t mo = spread3(x0) | (spread3(x1) << 1) | (spread3(x2) << 2);
    uint32_t e = T.t1[(uint32_t)(mo >> 60) & 7u];
    uint64_t key = e & 7u;
    uint32_t s = e >> 3;
#pragma unroll
    for (int l = 19; l > 0; l -= 2) {  // levels l and l - 1
        e = T.t2[s * 64u + ((uint32_t)(mo >> (3 * (l - 1))) & 63u)];
        key = (key << 6) | (e & 63u);
        s = e >> 6;
    }
    return key;
}

namespace {

// Keys of the particles at pos.  With id (the caller index of each slot of
// a key-ordered state), key and payload go to the caller index, so that the
// stable sort breaks ties by caller index as the order rule asks, and
// inv[caller index] = slot records where each particle was.
__global__ void __launch_bounds__(256) k_keys(const double *__restrict__ pos, int64_t n,
                                              const DevScalars *__restrict__ sc,
                                              uint64_t *__restrict__ key,
                                              uint32_t *__restrict__ val,
                                              const uint32_t *__restrict__ id,
                                              uint32_t *__restrict__ inv) {
    __shared__ PhTables T;
    ph_build(T);
    const double lo0 = sc->lo[0], lo1 = sc->lo[1], lo2 = sc->lo[2], s = sc->scale;
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        uint32_t q0 = quantise(pos[i], lo0, s);
        uint32_t q1 = quantise(pos[n + i], lo1, s);
        uint32_t q2 = quantise(pos[2 * n + i], lo2, s);
        const uint32_t o = id ? id[i] : (uint32_t)i;
        key[o] = ph_key(T, q0, q1, q2);
        val[o] = o;
        if (id) inv[o] = (uint32_t)i;
    }
}

}  // namespace

void launch_bbox(bonsai_ctx *c, const double *pos, const double *mass, int64_t n) {
    int nb = grid_for(n, BOX_BLOCK * 4, c->sm_count * 4);
    k_box_partial<<<nb, BOX_BLOCK, 0, c->stream>>>(pos, mass, n, c->box_part.p);
    k_box_final<<<1, BOX_BLOCK, 0, c->stream>>>(c->box_part.p, nb, c->dsc);
    c->launches += 2;
}

// Bounding cube and keys into explicit buffers (no context): part holds at
// most max_part block partials.  Returns the number of kernels launched.
int launch_cube_keys_into(cudaStream_t s, int sm_count, const double *pos, const double *mass,
                          int64_t n, BoxPartial *part, int max_part, DevScalars *dsc,
                          uint64_t *key, uint32_t *val) {
    const int cap = sm_count * 4 < max_part ? sm_count * 4 : max_part;
    const int nb = grid_for(n, BOX_BLOCK * 4, cap);
    k_box_partial<<<nb, BOX_BLOCK, 0, s>>>(pos, mass, n, part);
    k_box_final<<<1, BOX_BLOCK, 0, s>>>(part, nb, dsc);
    k_keys<<<grid_for(n, 256, sm_count * 4), 256, 0, s>>>(pos, n, dsc, key, val, nullptr, nullptr);
    return 3;
}

void launch_keys(bonsai_ctx *c, const double *pos, int64_t n, const uint32_t *id, uint32_t *inv) {
    k_keys<<<grid_for(n, 256, c->sm_count * 4), 256, 0, c->stream>>>(pos, n, c->dsc, c->key.p,
                                                                       c->val.p, id, inv);
    c->launches += 1;
}

}  // namespace bgb

// The cube of k_box_final, on the host, for bounds reduced over processes.
// Each step is one IEEE FP64 operation in the kernel's order (the product
// by 0.5 is exact, so a fused multiply-add could not change the result).
extern "C" int bonsai_cube_from_bounds(const double mn[3], const double mx[3], double cube[4]) {
    if (!mn || !mx || !cube) return BONSAI_EINVAL;
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(mn[d]) || !std::isfinite(mx[d]) || mn[d] > mx[d]) return BONSAI_EINVAL;
    double ext = mx[0] - mn[0];
    const double e1 = mx[1] - mn[1], e2 = mx[2] - mn[2];
    if (e1 > ext) ext = e1;
    if (e2 > ext) ext = e2;
    double L = ext * (1.0 + 0x1p-20);
    if (ext == 0.0) L = 1.0;
    for (int d = 0; d < 3; ++d) {
        const double w = mx[d] - mn[d];
        cube[d] = mn[d] - (L - w) * 0.5;
    }
    cube[3] = L;
    return BONSAI_OK;
}
