// integrate.cu -- the leap-frog (Sec. III.B.2, last paragraph: a
// second-order leap-frog ends the step), the energy/momentum diagnostics
// ("gather and write statistics", Table 2's "Other"), and the copies
// between key order and the caller's order.  All FP64 and HBM-bound.
#include "internal.cuh"

namespace bgb {

namespace {

constexpr int DIAG_BLOCK = 256;
constexpr int NDIAG = 10;

// v += a h (a in FP32, promoted), all three components.
__global__ void __launch_bounds__(256) k_kick(double *__restrict__ vel,
                                              const float *__restrict__ acc, int64_t n3, double h) {
    for (int64_t k = blockIdx.x * 256ll + threadIdx.x; k < n3; k += (int64_t)gridDim.x * 256)
        vel[k] = __dadd_rn(vel[k], __dmul_rn((double)acc[k], h));
}

// x += v dt.
__global__ void __launch_bounds__(256) k_drift(double *__restrict__ pos,
                                               const double *__restrict__ vel, int64_t n3,
                                               double dt) {
    for (int64_t k = blockIdx.x * 256ll + threadIdx.x; k < n3; k += (int64_t)gridDim.x * 256)
        pos[k] = __dadd_rn(pos[k], __dmul_rn(vel[k], dt));
}

__device__ inline double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < DIAG_BLOCK / 32; ++k) r += sh[k];
    return r;
}

// Per-block partial sums of {E_kin, E_pot, P, L, M}.
__global__ void __launch_bounds__(DIAG_BLOCK) k_diag_partial(const double *__restrict__ pos,
                                                             const double *__restrict__ vel,
                                                             const double *__restrict__ mass,
                                                             const float *__restrict__ pot,
                                                             int64_t n, double *__restrict__ part) {
    double s[NDIAG] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)DIAG_BLOCK + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * DIAG_BLOCK) {
        const double m = mass[i];
        const double x = pos[i], y = pos[n + i], z = pos[2 * n + i];
        const double vx = vel[i], vy = vel[n + i], vz = vel[2 * n + i];
        s[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        s[1] += 0.5 * m * (double)pot[i];
        s[3] += m * vx;
        s[4] += m * vy;
        s[5] += m * vz;
        s[6] += m * (y * vz - z * vy);
        s[7] += m * (z * vx - x * vz);
        s[8] += m * (x * vy - y * vx);
        s[9] += m;
    }
    __shared__ double sh[DIAG_BLOCK / 32];
#pragma unroll
    for (int k = 0; k < NDIAG; ++k) {
        double r = block_sum(s[k], sh);
        if (threadIdx.x == 0) part[blockIdx.x * NDIAG + k] = r;
    }
}

__global__ void __launch_bounds__(32) k_diag_final(const double *__restrict__ part, int nb,
                                                   double *__restrict__ out) {
    const int k = threadIdx.x;
    if (k >= NDIAG) return;
    double r = 0.0;
    for (int b = 0; b < nb; ++b) r += part[b * NDIAG + k];
    out[k] = r;  // out[2] (E_tot) is formed on the host
}

__global__ void __launch_bounds__(256) k_unpermute_state(const double *__restrict__ pos,
                                                         const double *__restrict__ vel,
                                                         const double *__restrict__ mass,
                                                         const uint32_t *__restrict__ id,
                                                         int64_t n, double *__restrict__ pos_c,
                                                         double *__restrict__ vel_c,
                                                         double *__restrict__ mass_c) {
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const uint32_t o = id[i];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (pos_c) pos_c[d * n + o] = pos[d * n + i];
            if (vel_c) vel_c[d * n + o] = vel[d * n + i];
        }
        if (mass_c) mass_c[o] = mass[i];
    }
}

__global__ void __launch_bounds__(256) k_unpermute_forces(const float *__restrict__ acc,
                                                          const float *__restrict__ pot,
                                                          const uint32_t *__restrict__ id,
                                                          int64_t n, float *__restrict__ acc_c,
                                                          float *__restrict__ pot_c) {
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const uint32_t o = id[i];
        if (acc_c) {
            acc_c[o] = acc[i];
            acc_c[n + o] = acc[n + i];
            acc_c[2 * n + o] = acc[2 * n + i];
        }
        if (pot_c) pot_c[o] = pot[i];
    }
}

__global__ void __launch_bounds__(256) k_permute_in_vel(const double *__restrict__ vel_c,
                                                        const uint32_t *__restrict__ id, int64_t n,
                                                        double *__restrict__ vel) {
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const uint32_t o = id[i];
#pragma unroll
        for (int d = 0; d < 3; ++d) vel[d * n + i] = vel_c[d * n + o];
    }
}

}  // namespace

void launch_kick(bonsai_ctx *c, double h) {
    const int64_t n3 = 3 * c->n;
    k_kick<<<grid_for(n3, 256, c->sm_count * 16), 256, 0, c->stream>>>(c->vel.p, c->acc.p, n3, h);
    c->launches += 1;
}

void launch_drift(bonsai_ctx *c, double dt) {
    const int64_t n3 = 3 * c->n;
    k_drift<<<grid_for(n3, 256, c->sm_count * 16), 256, 0, c->stream>>>(c->pos.p, c->vel.p, n3,
                                                                          dt);
    c->launches += 1;
}

int diag_blocks(bonsai_ctx *c) { return c->sm_count * 2; }

void launch_diagnostics(bonsai_ctx *c, double *out_dev) {
    const int nb = diag_blocks(c);
    k_diag_partial<<<nb, DIAG_BLOCK, 0, c->stream>>>(c->pos.p, c->vel.p, c->mass.p, c->pot.p, c->n,
                                                     c->diag_part.p);
    k_diag_final<<<1, 32, 0, c->stream>>>(c->diag_part.p, nb, out_dev);
    c->launches += 2;
}

void launch_unpermute_state(bonsai_ctx *c, double *pos, double *vel, double *mass) {
    k_unpermute_state<<<grid_for(c->n, 256, c->sm_count * 16), 256, 0, c->stream>>>(
        c->pos.p, c->vel.p, c->mass.p, c->id.p, c->n, pos, vel, mass);
    c->launches += 1;
}

void launch_unpermute_forces(bonsai_ctx *c, float *acc, float *pot) {
    k_unpermute_forces<<<grid_for(c->n, 256, c->sm_count * 16), 256, 0, c->stream>>>(
        c->acc.p, c->pot.p, c->id.p, c->n, acc, pot);
    c->launches += 1;
}

void launch_permute_in_vel(bonsai_ctx *c, const double *vel) {
    k_permute_in_vel<<<grid_for(c->n, 256, c->sm_count * 16), 256, 0, c->stream>>>(
        vel, c->id.p, c->n, c->vel.p);
    c->launches += 1;
}

}  // namespace bgb
