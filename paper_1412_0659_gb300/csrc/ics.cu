// ics.cu -- on-the-fly galaxy initial conditions on the GPU (Sec. IV: the
// Milky Way model -- NFW halo, exponential disk, Hernquist bulge -- is
// generated on the fly rather than read from an initial-condition file).
//
// Steps (each a kernel below):
//   1. k_shapes: a logarithmic radial grid r_k = R_MIN e^{k dl}; for both
//      spheroids the tapered shape C(r) / (x (1+x)^beta) (beta = 2 NFW, 3
//      Hernquist; C = erfc((r - r_t)/(sqrt(2) dr_t))/2) and its first two
//      radial derivatives in closed form; the sech^2 exponential disk's
//      spherical shell mass rate (Simpson in the polar angle).
//   2. k_cumulative: enclosed shape masses (closed form below the first
//      node, trapezoid rule in ln r above), one block per spheroid and one
//      for the disk.
//   3. k_profiles: normalised densities, masses and cumulative fractions.
//   4. k_potential: Psi = G M(<r)/r + G int_r dM/dr' d ln r' (reverse scan),
//      Psi', Psi'' and d2rho/dPsi2 = (rho'' Psi' - rho' Psi'')/Psi'^3.
//   5. k_eddington: each spheroid's isotropic distribution function by
//      Eddington's formula, the integral exact for a piecewise-linear
//      integrand between nodes (one warp per energy).
//   6. k_speed_cdf: per radius, the cumulative distribution of the speed
//      fraction q = v/v_esc, density q^2 f(Psi_min + (1 - q^2)(Psi - Psi_min)).
//   7. k_disk_*: the disk's cumulative surface mass, its rotation in the
//      spheroids' enclosed mass plus the midplane force of the sech^2
//      exponential disk (Hankel integral in k), the epicyclic frequency, the
//      dispersions (sigma_R^2 ~ Sigma with Toomre's Q at R_Q, epicyclic
//      sigma_phi, isothermal-sheet sigma_z) and the asymmetric-drift
//      rotation.
//   8. k_sample: every particle draws Philox4x32-10 uniforms (counter =
//      particle, component, call, 0; key = seed) and inverts the tables.
//   9. k_moments / k_shift: centre of mass and mean velocity to zero.
//
// All arithmetic is FP64.  The tables are a few MB and stay in L2 while the
// sampler reads them.
#include <math.h>

#include "internal.cuh"

namespace {

constexpr int K = BONSAI_ICS_K;
constexpr int V = BONSAI_ICS_V;
constexpr int KD = BONSAI_ICS_KD;
constexpr double R_MIN = 1.0e-4;
constexpr double R_MAX = 600.0;
constexpr double PI = 3.141592653589793238462643383279502884;
constexpr int SHELL_N = 2048;   // Simpson intervals of the disk's spherical shell average
constexpr int VC_NK = 4000;     // Simpson intervals of the disk's Hankel integral in k
constexpr double VC_KMAX = 40.0;  // k range, in units of 1 / R_d
constexpr int IZ_NT = 4096;     // Simpson intervals of the vertical factor in t = z / z0
constexpr double IZ_TMAX = 40.0;

// rows of the radial table
enum {
    RR = 0, RPSI, RMT, RMH, RMB, RPH, RPB, RG2H, RG2B, RFH, RFB, RVNH, RVNB, RRHOH, RRHOB,
    RLOGR, RS1H, RS2H, RS1B, RS2B, RFH_INT, RFB_INT, RSH, RSB, RDMT, RMD, RDMD, RS0H, RS0B,
    RSLH, RSLB,  // d2rho/dPsi2 slope of segment [Psi_{k+1}, Psi_k]
    RFD_INT,     // r dM/dr of the disk (integrand in ln r)
    NRAD
};
static_assert(BONSAI_ICS_NRAD_OUT <= NRAD, "exported radial rows");
// rows of the disk table
enum { DCDF = 0, DVC2, DKAP, DSR, DSPHI, DSZ, DVPHI, DOM2, DKAP2, NDISK };
static_assert(BONSAI_ICS_NDISK_OUT <= NDISK, "exported disk rows");

struct IcsTables {
    double *rad;   // [NRAD][K]
    double *vcdf;  // [2][K][V]
    double *disk;  // [NDISK][KD]
    double *iz;    // [VC_NK + 1]: the disk's vertical factor I(k z0) on the k grid
};

// Simpson weight of node j of n intervals (n even), without the h/3
__device__ __forceinline__ double simpson_w(int j, int n) {
    return (j == 0 || j == n) ? 1.0 : ((j & 1) ? 4.0 : 2.0);
}

// Central surface density of the truncated disk (total mass M_disk)
__device__ double disk_sigma0(const bonsai_galaxy &g);

__device__ __forceinline__ double *row(double *t, int r) { return t + (size_t)r * K; }
__device__ __forceinline__ const double *row(const double *t, int r) { return t + (size_t)r * K; }

// 1 - (1 + x) e^-x: the alternating series sum_{k>=2} (-1)^k (k-1) x^k / k!
// (22 terms) below x = 1/2, where the closed form cancels; the closed form
// above.
__device__ double disk_fraction(double x) {
    if (x >= 0.5) return 1.0 - (1.0 + x) * exp(-x);
    double s = 0.0, t = 0.5 * x * x;
    for (int k = 2; k < 24; ++k) {
        s += ((k & 1) ? -1.0 : 1.0) * (k - 1) * t;
        t = t * x / (k + 1);
    }
    return s;
}

__device__ double disk_sigma0(const bonsai_galaxy &g) {
    return g.M_disk / (2.0 * PI * g.R_d * g.R_d * disk_fraction(g.R_max / g.R_d));
}

// ---------------------------------------------------------------- step 1
__global__ void k_shapes(bonsai_galaxy g, double *rad) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const double dl = log(R_MAX / R_MIN) / (K - 1);
    const double r = R_MIN * exp(dl * k);
    row(rad, RR)[k] = r;
    row(rad, RLOGR)[k] = log(r);
    const double y = (r - g.r_t) / (sqrt(2.0) * g.dr_t);
    const double C = 0.5 * erfc(y);
    const double C1 = -exp(-y * y) / (sqrt(2.0 * PI) * g.dr_t);
    const double C2 = -C1 * (r - g.r_t) / (g.dr_t * g.dr_t);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const double a = c == 0 ? g.a_halo : g.a_bulge;
        const double beta = c == 0 ? 2.0 : 3.0;
        const double x = r / a;
        const double h = 1.0 / (x * pow(1.0 + x, beta));
        const double L1 = -1.0 / r - beta / (a + r);
        const double L1p = 1.0 / (r * r) + beta / ((a + r) * (a + r));
        const double h1 = h * L1, h2 = h * (L1 * L1 + L1p);
        const double s0 = h * C;
        row(rad, c == 0 ? RS0H : RS0B)[k] = s0;
        row(rad, c == 0 ? RS1H : RS1B)[k] = h1 * C + h * C1;
        row(rad, c == 0 ? RS2H : RS2B)[k] = h2 * C + 2.0 * h1 * C1 + h * C2;
        row(rad, c == 0 ? RFH_INT : RFB_INT)[k] = 4.0 * PI * r * r * r * s0;
    }
}

// Sum over the 32 lanes of a warp (every lane gets the total).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The disk: 4 pi r^2 times its density averaged over the sphere, rho =
// Sigma0 e^{-R/R_d} sech^2(z/z0) / (2 z0) for R <= R_max, by Simpson's rule
// in the polar angle phi (R = r cos phi, z = r sin phi) on
// [acos(min(1, R_max/r)), asin(min(1, 40 z0/r))].  A warp per radius node,
// its lanes taking every 32nd term.
__global__ void k_disk_shell(bonsai_galaxy g, double *rad) {
    const int k = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= K) return;
    const double dl = log(R_MAX / R_MIN) / (K - 1);
    const double r = R_MIN * exp(dl * k);
    const double sig0 = disk_sigma0(g);
    const double hi = asin(fmin(1.0, IZ_TMAX * g.z0 / r));
    const double lo = acos(fmin(1.0, g.R_max / r));
    double dM = 0.0;
    if (hi > lo) {
        const double hp = (hi - lo) / SHELL_N;
        double acc = 0.0;
        for (int j = lane; j <= SHELL_N; j += 32) {
            const double phi = lo + (hi - lo) * j / SHELL_N;
            const double cph = cos(phi);
            const double ch = cosh(r * sin(phi) / g.z0);
            acc += simpson_w(j, SHELL_N) * (sig0 * exp(-r * cph / g.R_d) / (2.0 * g.z0) / (ch * ch)) * cph;
        }
        dM = 4.0 * PI * r * r * (hp / 3.0 * warp_sum(acc));
    }
    if (lane == 0) {
        row(rad, RDMD)[k] = dM;
        row(rad, RFD_INT)[k] = r * dM;
    }
}

// Exclusive scan of one double per thread over a block of 1024 threads.
__device__ double block_exclusive_scan(double v, double *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        double s = sh[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    const double pre = w > 0 ? sh[w - 1] : 0.0;
    __syncthreads();
    return pre + x - v;
}

constexpr int SCAN_T = 1024;
constexpr int PER_T = K / SCAN_T;
static_assert(K % SCAN_T == 0, "scan shape");
static_assert(KD % 256 == 0 && KD % 64 == 0, "disk launch shapes");

// ---------------------------------------------------------------- step 2
// S[k] = S0 + sum_{j<k} (F_j + F_{j+1}) dl / 2, S0 the closed-form mass of
// the untapered cusp below r_0 times C(r_0).  Block 0: halo, block 1: bulge,
// block 2: the disk (S0: the central density times the volume below r_0).
__global__ void __launch_bounds__(SCAN_T) k_cumulative(bonsai_galaxy g, double *rad) {
    __shared__ double sh[32];
    const int c = blockIdx.x;
    const double dl = log(R_MAX / R_MIN) / (K - 1);
    const double *F = row(rad, c == 0 ? RFH_INT : (c == 1 ? RFB_INT : RFD_INT));
    double *S = row(rad, c == 0 ? RSH : (c == 1 ? RSB : RMD));
    const double r0 = R_MIN;
    double S0;
    if (c == 2) {
        S0 = 4.0 / 3.0 * PI * r0 * r0 * r0 * disk_sigma0(g) / (2.0 * g.z0);
    } else {
        const double a = c == 0 ? g.a_halo : g.a_bulge;
        const double x0 = r0 / a;
        const double C0 = 0.5 * erfc((r0 - g.r_t) / (sqrt(2.0) * g.dr_t));
        const double I = c == 0 ? log1p(x0) - x0 / (1.0 + x0) : x0 * x0 / (2.0 * (1.0 + x0) * (1.0 + x0));
        S0 = 4.0 * PI * a * a * a * C0 * I;
    }
    const int j0 = threadIdx.x * PER_T;
    double seg[PER_T], tot = 0.0;
#pragma unroll
    for (int i = 0; i < PER_T; ++i) {
        const int j = j0 + i;
        seg[i] = j < K - 1 ? 0.5 * (F[j] + F[j + 1]) * dl : 0.0;
        tot += seg[i];
    }
    double run = S0 + block_exclusive_scan(tot, sh);
#pragma unroll
    for (int i = 0; i < PER_T; ++i) {
        S[j0 + i] = run;
        run += seg[i];
    }
}

// ---------------------------------------------------------------- step 3
__global__ void k_profiles(bonsai_galaxy g, double *rad) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const double r = row(rad, RR)[k];
    double Mt = row(rad, RMD)[k], rho_t = 0.0;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const double *S = row(rad, c == 0 ? RSH : RSB);
        const double M = c == 0 ? g.M_halo : g.M_bulge;
        const double rho0 = M / S[K - 1];
        const double rho = rho0 * row(rad, c == 0 ? RS0H : RS0B)[k];
        row(rad, c == 0 ? RRHOH : RRHOB)[k] = rho;
        row(rad, c == 0 ? RS1H : RS1B)[k] *= rho0;  // rho'
        row(rad, c == 0 ? RS2H : RS2B)[k] *= rho0;  // rho''
        const double Mc = rho0 * S[k];
        row(rad, c == 0 ? RMH : RMB)[k] = Mc;
        row(rad, c == 0 ? RPH : RPB)[k] = S[k] / S[K - 1];
        Mt += Mc;
        rho_t += rho;
    }
    row(rad, RMT)[k] = Mt;
    row(rad, RDMT)[k] = 4.0 * PI * r * r * rho_t + row(rad, RDMD)[k];
}

// ---------------------------------------------------------------- step 4
// O[k] = sum_{j=k}^{K-2} (dMt_j + dMt_{j+1}) dl / 2 as an exclusive scan of
// the reversed segments; then Psi and d2rho/dPsi2 of both spheroids.
__global__ void __launch_bounds__(SCAN_T) k_potential(bonsai_galaxy g, double *rad) {
    __shared__ double sh[32];
    const double dl = log(R_MAX / R_MIN) / (K - 1);
    const double *dMt = row(rad, RDMT);
    const int e0 = threadIdx.x * PER_T;  // reversed index e: k = K - 1 - e
    double seg[PER_T], tot = 0.0;
#pragma unroll
    for (int i = 0; i < PER_T; ++i) {
        const int e = e0 + i;
        const int j = K - 2 - e;  // segment j spans nodes j, j + 1
        seg[i] = j >= 0 ? 0.5 * (dMt[j] + dMt[j + 1]) * dl : 0.0;
        tot += seg[i];
    }
    double run = block_exclusive_scan(tot, sh);
#pragma unroll
    for (int i = 0; i < PER_T; ++i) {
        const int k = K - 1 - (e0 + i);
        const double r = row(rad, RR)[k];
        const double Mt = row(rad, RMT)[k];
        const double Psi = g.G * (Mt / r + run);
        const double P1 = -g.G * Mt / (r * r);
        const double P2 = 2.0 * g.G * Mt / (r * r * r) - g.G * dMt[k] / (r * r);
        row(rad, RPSI)[k] = Psi;
        const double P13 = P1 * P1 * P1;
        row(rad, RG2H)[k] = (row(rad, RS2H)[k] * P1 - row(rad, RS1H)[k] * P2) / P13;
        row(rad, RG2B)[k] = (row(rad, RS2B)[k] * P1 - row(rad, RS1B)[k] * P2) / P13;
        run += seg[i];
    }
    __syncthreads();
    // slope of the linear d2rho/dPsi2 on each segment [Psi_{k+1}, Psi_k]
    for (int k = threadIdx.x; k < K - 1; k += SCAN_T) {
        const double *Ps = row(rad, RPSI);
        const double dP = Ps[k] - Ps[k + 1];
        row(rad, RSLH)[k] = (row(rad, RG2H)[k] - row(rad, RG2H)[k + 1]) / dP;
        row(rad, RSLB)[k] = (row(rad, RG2B)[k] - row(rad, RG2B)[k + 1]) / dP;
    }
}

// ---------------------------------------------------------------- step 5
// f(E_j), E_j = Psi_j: (1/(sqrt(8) pi^2)) sum over segments [Psi_{k+1},
// Psi_k], k >= j, of the exact integral of the linear g2 / sqrt(E - Psi).
// Each lane takes a contiguous run of segments, so that sqrt(E - Psi_k) of
// a node shared by two segments is taken once.
constexpr int EDD_WARPS = 8;
__global__ void __launch_bounds__(EDD_WARPS * 32) k_eddington(double *rad) {
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * EDD_WARPS + (threadIdx.x >> 5);
    if (wid >= 2 * K) return;
    const int c = wid / K, j = wid % K;
    const double *Psi = row(rad, RPSI);
    const double *g2 = row(rad, c == 0 ? RG2H : RG2B);
    const double *sl = row(rad, c == 0 ? RSLH : RSLB);
    const double E = Psi[j];
    const int nseg = K - 1 - j;
    const int per = (nseg + 31) / 32;
    const int k0 = j + lane * per;
    const int k1 = min(k0 + per, K - 1);
    double s = 0.0;
    if (k0 < k1) {
        double sb = E - Psi[k0];
        double rsb = sqrt(sb);
        for (int k = k0; k < k1; ++k) {
            const double pa = Psi[k + 1], pb = Psi[k];
            const double slope = sl[k];
            const double sa = E - pa;
            const double rsa = sqrt(sa);
            const double D = (pb - pa) / (rsa + rsb);
            const double A = g2[k + 1] + slope * sa;
            s += 2.0 * A * D - (2.0 / 3.0) * slope * D * (sa + rsa * rsb + sb);
            sb = sa;
            rsb = rsa;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const double f = s * (1.0 / (sqrt(8.0) * PI * PI));
        row(rad, c == 0 ? RFH : RFB)[j] = f > 0.0 ? f : 0.0;
    }
}

// Largest m in [0, n - 2] with T[m] <= u (bisection).
__device__ __forceinline__ int bisect(const double *T, int n, double u) {
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (T[mid] <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

// f at energy E by linear interpolation on the decreasing Psi nodes,
// clamped outside them.
__device__ double f_at(const double *Psi, const double *f, double E) {
    if (E >= Psi[0]) return f[0];
    if (E <= Psi[K - 1]) return f[K - 1];
    int lo = 0, hi = K - 1;  // Psi[lo] > E >= Psi[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (Psi[mid] > E) lo = mid;
        else hi = mid;
    }
    // -Psi increases with the index: interpolate in x = -E between lo, hi
    const double x0 = -Psi[lo], x1 = -Psi[hi];
    return (f[hi] - f[lo]) / (x1 - x0) * (-E - x0) + f[lo];
}

// ---------------------------------------------------------------- step 6
constexpr int VPL = V / 32;  // speed nodes per lane
__global__ void __launch_bounds__(EDD_WARPS * 32) k_speed_cdf(double *rad, double *vcdf) {
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * EDD_WARPS + (threadIdx.x >> 5);
    if (wid >= 2 * K) return;
    const int c = wid / K, k = wid % K;
    const double *Psi = row(rad, RPSI);
    const double *f = row(rad, c == 0 ? RFH : RFB);
    const double pmin = Psi[K - 1];
    const double w = Psi[k] - pmin;
    double p[VPL];
#pragma unroll
    for (int i = 0; i < VPL; ++i) {
        const double q = (lane * VPL + i) / (V - 1.0);
        p[i] = q * q * f_at(Psi, f, pmin + (1.0 - q * q) * w);
    }
    // trapezoid segments ending at each node; the first node's is zero
    double prev = __shfl_up_sync(0xffffffffu, p[VPL - 1], 1);
    double seg[VPL], tot = 0.0;
#pragma unroll
    for (int i = 0; i < VPL; ++i) {
        const double pm = i == 0 ? prev : p[i - 1];
        seg[i] = (lane == 0 && i == 0) ? 0.0 : 0.5 * (pm + p[i]) / (V - 1.0);
        tot += seg[i];
    }
    double x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    double run = x - tot;
    const double all = __shfl_sync(0xffffffffu, x, 31);
    double *C = vcdf + ((size_t)c * K + k) * V + lane * VPL;
#pragma unroll
    for (int i = 0; i < VPL; ++i) {
        run += seg[i];
        const double q = (lane * VPL + i) / (V - 1.0);
        C[i] = all > 0.0 ? run / all : q;
    }
    if (lane == 0) row(rad, c == 0 ? RVNH : RVNB)[k] = all;
}

// ---------------------------------------------------------------- step 7
// The disk's vertical factor on the k grid k_j = j (40 / R_d) / VC_NK:
// I(k z0) = int_0^inf sech^2(t) e^{-k z0 t} dt (the sech^2 layer's weight of
// e^{-k|z|}; 1 for a thin disk), Simpson's rule on t in [0, 40].
// A warp per k node, its lanes taking every 32nd term.
__global__ void k_disk_vertical(bonsai_galaxy g, double *iz) {
    const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (j > VC_NK) return;
    const double hk = VC_KMAX / g.R_d / VC_NK;
    const double kz = hk * j * g.z0;
    const double ht = IZ_TMAX / IZ_NT;
    double acc = 0.0;
    for (int i = lane; i <= IZ_NT; i += 32) {
        const double t = IZ_TMAX * i / IZ_NT;
        const double ch = cosh(t);
        acc += simpson_w(i, IZ_NT) * (exp(-kz * t) / (ch * ch));
    }
    acc = warp_sum(acc);
    if (lane == 0) iz[j] = ht / 3.0 * acc;
}

__device__ __forceinline__ double central(const double *y, int j, double h) {
    if (j == 0) return (y[1] - y[0]) / h;
    if (j == KD - 1) return (y[KD - 1] - y[KD - 2]) / h;
    return (y[j + 1] - y[j - 1]) / (2.0 * h);
}

// Enclosed spheroid mass at radius R: linear in ln r between nodes, ~ r^2
// below the first node.
__device__ double sph_mass_at(const double *rad, int rowM, double R) {
    const double *M = row(rad, rowM);
    const double *lr = row(rad, RLOGR);
    const double r0 = row(rad, RR)[0];
    if (R < r0) return M[0] * (R / r0) * (R / r0);
    const double x = log(R);
    if (x >= lr[K - 1]) return M[K - 1];
    const int i = bisect(lr, K, x);
    return (M[i + 1] - M[i]) / (lr[i + 1] - lr[i]) * (x - lr[i]) + M[i];
}

struct DiskRows {
    double *cdf, *vc2, *kap, *sR, *sphi, *sz, *vphi, *om2, *kap2;
};
__device__ __forceinline__ DiskRows disk_rows(double *disk) {
    return DiskRows{disk + (size_t)DCDF * KD, disk + (size_t)DVC2 * KD, disk + (size_t)DKAP * KD,
                    disk + (size_t)DSR * KD, disk + (size_t)DSPHI * KD, disk + (size_t)DSZ * KD,
                    disk + (size_t)DVPHI * KD, disk + (size_t)DOM2 * KD, disk + (size_t)DKAP2 * KD};
}

// 7a: cumulative surface mass on R_j = j h, v_c^2 and Omega^2 on (j + 1/2) h.
// The disk's part of v_c^2 in the midplane of the sech^2 exponential disk:
// 2 pi G Sigma0 R_d^2 R int_0^inf k J1(kR) I(k z0) (1 + k^2 R_d^2)^{-3/2} dk
// (the thin disk's Hankel form with e^{-k|z|} averaged over the layer),
// Simpson's rule on k in [0, 40 / R_d].
// A warp per radius, its lanes taking every 32nd term of the k integral.
__global__ void k_disk_rotation(bonsai_galaxy g, const double *rad, const double *iz,
                                double *disk) {
    const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= KD) return;
    const DiskRows D = disk_rows(disk);
    const double h = g.R_max / (KD - 1);
    const double s0 = g.M_disk / (2.0 * PI * g.R_d * g.R_d);
    const double R = (j + 0.5) * h;
    const double hk = VC_KMAX / g.R_d / VC_NK;
    double acc = 0.0;
    for (int i = lane; i <= VC_NK; i += 32) {
        const double k = hk * i;
        const double q = 1.0 + (k * g.R_d) * (k * g.R_d);
        acc += simpson_w(i, VC_NK) * (j1(R * k) * (k * iz[i] * (1.0 / (q * sqrt(q)))));
    }
    acc = warp_sum(acc);
    if (lane != 0) return;
    D.cdf[j] = j == KD - 1 ? 1.0 : disk_fraction(j * h / g.R_d) / disk_fraction(g.R_max / g.R_d);
    const double ms = sph_mass_at(rad, RMH, R) + sph_mass_at(rad, RMB, R);
    const double vd2 = 2.0 * PI * g.G * s0 * g.R_d * g.R_d * R * (hk / 3.0 * acc);
    const double v2 = g.G * ms / R + vd2;
    D.vc2[j] = v2;
    D.om2[j] = v2 / (R * R);
}

// 7b: kappa from central differences of Omega^2
__global__ void k_disk_kappa(bonsai_galaxy g, double *disk) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= KD) return;
    const DiskRows D = disk_rows(disk);
    const double h = g.R_max / (KD - 1);
    const double R = (j + 0.5) * h;
    const double k2 = R * central(D.om2, j, h) + 4.0 * D.om2[j];
    D.kap2[j] = k2;
    D.kap[j] = sqrt(k2 > 1e-30 ? k2 : 1e-30);
}

// 7c: sigma_R^2 proportional to Sigma with Toomre's Q at R_Q, the epicyclic
// sigma_phi, the isothermal-sheet sigma_z and the asymmetric-drift mean
// rotation v_phi^2 = v_c^2 + sigma_R^2 (1 - kappa^2/(4 Omega^2) - 2R/R_d),
// held within [0, v_c^2]
__global__ void k_disk_kinematics(bonsai_galaxy g, double *disk) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= KD) return;
    const DiskRows D = disk_rows(disk);
    const double h = g.R_max / (KD - 1);
    const double s0 = g.M_disk / (2.0 * PI * g.R_d * g.R_d);
    double sq = g.R_Q / h - 0.5;
    sq = sq < 0.0 ? 0.0 : (sq > KD - 1.0 ? KD - 1.0 : sq);
    int iq = (int)sq;
    iq = iq > KD - 2 ? KD - 2 : iq;
    const double wq = sq - iq;
    const double kq = (1.0 - wq) * D.kap[iq] + wq * D.kap[iq + 1];
    const double sRq = g.Q * 3.36 * g.G * s0 * exp(-g.R_Q / g.R_d) / kq;
    const double R = (j + 0.5) * h;
    const double sr = sRq * exp(-(R - g.R_Q) / (2.0 * g.R_d));
    const double Sig = s0 * exp(-R / g.R_d);
    D.sR[j] = sr;
    D.sphi[j] = sr * D.kap[j] / (2.0 * sqrt(D.om2[j]));
    D.sz[j] = sqrt(PI * g.G * Sig * g.z0);
    const double vc2 = D.vc2[j];
    double v2 = vc2 + sr * sr * (1.0 - D.kap2[j] / (4.0 * D.om2[j]) - 2.0 * R / g.R_d);
    v2 = v2 < 0.0 ? 0.0 : (v2 > vc2 ? vc2 : v2);
    D.vphi[j] = sqrt(v2);
}

// ---------------------------------------------------------------- step 8
struct U2 {
    double a, b;
};

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC11): two uniforms
// (m + 1/2) 2^-52 from the 52-bit m = (w0 >> 6) 2^26 + (w1 >> 6) (words 0, 1
// and 2, 3).
__device__ __forceinline__ U2 draws(uint32_t i, uint32_t comp, uint32_t call, uint32_t k0,
                                    uint32_t k1) {
    uint32_t c0 = i, c1 = comp, c2 = call, c3 = 0;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    const uint64_t ma = ((uint64_t)(c0 >> 6) << 26) | (c1 >> 6);
    const uint64_t mb = ((uint64_t)(c2 >> 6) << 26) | (c3 >> 6);
    const double s = 0x1p-52;
    return U2{((double)ma + 0.5) * s, ((double)mb + 0.5) * s};
}

__device__ __forceinline__ void isotropic(double uc, double up, double &x, double &y, double &z) {
    const double c = 2.0 * uc - 1.0;
    const double s = sqrt((1.0 - c) * (1.0 + c));
    double sp, cp;
    sincos(2.0 * PI * up, &sp, &cp);
    x = s * cp;
    y = s * sp;
    z = c;
}

// q with C_row(q) = u
__device__ __forceinline__ double invert_row(const double *C, double u) {
    const int m = bisect(C, V, u);
    const double c0 = C[m], c1 = C[m + 1];
    return (m + (u - c0) / (c1 - c0)) / (V - 1.0);
}

struct SampleArgs {
    bonsai_galaxy g;
    const double *rad, *vcdf, *disk;
    double *pos, *vel, *mass;
    int64_t n;
};

__global__ void __launch_bounds__(256) k_sample(const SampleArgs A) {
    const bonsai_galaxy &g = A.g;
    const int64_t n = A.n;
    const uint32_t k0 = (uint32_t)(g.seed & 0xFFFFFFFFu), k1 = (uint32_t)(g.seed >> 32);
    const double dl = log(R_MAX / R_MIN) / (K - 1);
    const double *r_n = row(A.rad, RR), *Psi = row(A.rad, RPSI);
    const int64_t hd = g.n_halo + g.n_disk;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double px, py, pz, vx, vy, vz, m;
        if (i < g.n_halo || i >= hd) {
            const bool halo = i < g.n_halo;
            const uint32_t comp = halo ? 0u : 2u;
            const double *P = row(A.rad, halo ? RPH : RPB);
            const double *C = A.vcdf + (halo ? 0 : (size_t)K * V);
            const U2 a = draws((uint32_t)i, comp, 0, k0, k1);
            const U2 b = draws((uint32_t)i, comp, 1, k0, k1);
            const U2 c = draws((uint32_t)i, comp, 2, k0, k1);
            const double ur = a.a;
            int k;
            double t, r;
            if (ur < P[0]) {
                k = 0;
                t = 0.0;
                r = r_n[0] * sqrt(ur / P[0]);
            } else {
                k = bisect(P, K, ur);
                t = (ur - P[k]) / (P[k + 1] - P[k]);
                r = r_n[k] * exp(t * dl);
            }
            const double q = (1.0 - t) * invert_row(C + (size_t)k * V, b.b) +
                             t * invert_row(C + (size_t)(k + 1) * V, b.b);
            const double psi = (1.0 - t) * Psi[k] + t * Psi[k + 1];
            const double v = q * sqrt(2.0 * (psi - Psi[K - 1]));
            double dx, dy, dz;
            isotropic(a.b, b.a, dx, dy, dz);
            px = dx * r;
            py = dy * r;
            pz = dz * r;
            isotropic(c.a, c.b, dx, dy, dz);
            vx = dx * v;
            vy = dy * v;
            vz = dz * v;
            m = halo ? g.M_halo / (double)g.n_halo : g.M_bulge / (double)g.n_bulge;
        } else {
            const double *cdf = A.disk + (size_t)DCDF * KD;
            const double h = g.R_max / (KD - 1);
            const U2 a = draws((uint32_t)i, 1u, 0, k0, k1);
            const U2 b = draws((uint32_t)i, 1u, 1, k0, k1);
            const U2 c = draws((uint32_t)i, 1u, 2, k0, k1);
            const U2 d = draws((uint32_t)i, 1u, 3, k0, k1);
            const int j = bisect(cdf, KD, a.a);
            const double R = (j + (a.a - cdf[j]) / (cdf[j + 1] - cdf[j])) * h;
            const double z = g.z0 * atanh(2.0 * a.b - 1.0);
            double s = R / h - 0.5;
            s = s < 0.0 ? 0.0 : (s > KD - 1.0 ? KD - 1.0 : s);
            int i0 = (int)s;
            i0 = i0 > KD - 2 ? KD - 2 : i0;
            const double w = s - i0;
            auto at = [&](int rw) {
                const double *y = A.disk + (size_t)rw * KD;
                return (1.0 - w) * y[i0] + w * y[i0 + 1];
            };
            const double rho1 = sqrt(-2.0 * log(b.b));
            const double rho2 = sqrt(-2.0 * log(c.b));
            double sb, cb, sd, cd, sp, cp;
            sincos(2.0 * PI * c.a, &sb, &cb);
            sincos(2.0 * PI * d.a, &sd, &cd);
            sincos(2.0 * PI * b.a, &sp, &cp);
            const double n1 = rho1 * cb, n2 = rho1 * sb, n3 = rho2 * cd;
            const double vR = at(DSR) * n1;
            const double vp = at(DVPHI) + at(DSPHI) * n2;
            vz = at(DSZ) * n3;
            px = R * cp;
            py = R * sp;
            pz = z;
            vx = vR * cp - vp * sp;
            vy = vR * sp + vp * cp;
            m = g.M_disk / (double)g.n_disk;
        }
        A.pos[i] = px;
        A.pos[n + i] = py;
        A.pos[2 * n + i] = pz;
        A.vel[i] = vx;
        A.vel[n + i] = vy;
        A.vel[2 * n + i] = vz;
        A.mass[i] = m;
    }
}

// ---------------------------------------------------------------- step 9
constexpr int MOM_T = 256;
__global__ void __launch_bounds__(MOM_T) k_moments(const double *pos, const double *vel,
                                                   const double *mass, int64_t n, double *part) {
    __shared__ double sh[7][MOM_T / 32];
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)MOM_T + threadIdx.x; i < n; i += (int64_t)gridDim.x * MOM_T) {
        const double m = mass[i];
        s[0] += m * pos[i];
        s[1] += m * pos[n + i];
        s[2] += m * pos[2 * n + i];
        s[3] += m * vel[i];
        s[4] += m * vel[n + i];
        s[5] += m * vel[2 * n + i];
        s[6] += m;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        double v = s[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[q][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double v = 0.0;
        for (int k = 0; k < MOM_T / 32; ++k) v += sh[threadIdx.x][k];
        part[(size_t)blockIdx.x * 7 + threadIdx.x] = v;
    }
}

__global__ void __launch_bounds__(256) k_shift(double *pos, double *vel, int64_t n,
                                               const double *part, int nparts) {
    __shared__ double tot[7];
    if (threadIdx.x < 7) {
        double v = 0.0;
        for (int b = 0; b < nparts; ++b) v += part[(size_t)b * 7 + threadIdx.x];
        tot[threadIdx.x] = v;
    }
    __syncthreads();
    const double mt = tot[6];
    const double cx = tot[0] / mt, cy = tot[1] / mt, cz = tot[2] / mt;
    const double ux = tot[3] / mt, uy = tot[4] / mt, uz = tot[5] / mt;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        pos[i] -= cx;
        pos[n + i] -= cy;
        pos[2 * n + i] -= cz;
        vel[i] -= ux;
        vel[n + i] -= uy;
        vel[2 * n + i] -= uz;
    }
}

bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

int check(const bonsai_galaxy *g) {
    if (!g) return BONSAI_EINVAL;
    if (g->n_halo < 0 || g->n_disk < 0 || g->n_bulge < 0) return BONSAI_EINVAL;
    const int64_t n = g->n_halo + g->n_disk + g->n_bulge;
    if (n > (int64_t)0xFFFFFFFFll) return BONSAI_EINVAL;  // one Philox counter word
    if (!finite_pos(g->G) || !finite_pos(g->a_halo) || !finite_pos(g->a_bulge) ||
        !finite_pos(g->dr_t) || !finite_pos(g->R_d) || !finite_pos(g->z0) ||
        !finite_pos(g->R_max) || !finite_pos(g->Q) || !finite_pos(g->R_Q) || !isfinite(g->r_t))
        return BONSAI_EINVAL;
    const double Ms[3] = {g->M_halo, g->M_disk, g->M_bulge};
    const int64_t Ns[3] = {g->n_halo, g->n_disk, g->n_bulge};
    for (int c = 0; c < 3; ++c) {
        if (!isfinite(Ms[c]) || Ms[c] < 0.0) return BONSAI_EINVAL;
        if (Ns[c] > 0 && !(Ms[c] > 0.0)) return BONSAI_EINVAL;
    }
    if (!(g->M_halo + g->M_disk + g->M_bulge > 0.0)) return BONSAI_EINVAL;
    if (g->R_max > 200.0 * g->R_d) return BONSAI_EINVAL;  // the disk tables' range
    return BONSAI_OK;
}

int build_tables(const bonsai_galaxy &g, IcsTables &t, cudaStream_t s) {
    k_shapes<<<(K + 255) / 256, 256, 0, s>>>(g, t.rad);
    k_disk_shell<<<(K * 32 + 255) / 256, 256, 0, s>>>(g, t.rad);
    k_cumulative<<<3, SCAN_T, 0, s>>>(g, t.rad);
    k_profiles<<<(K + 255) / 256, 256, 0, s>>>(g, t.rad);
    k_potential<<<1, SCAN_T, 0, s>>>(g, t.rad);
    k_eddington<<<(2 * K + EDD_WARPS - 1) / EDD_WARPS, EDD_WARPS * 32, 0, s>>>(t.rad);
    k_speed_cdf<<<(2 * K + EDD_WARPS - 1) / EDD_WARPS, EDD_WARPS * 32, 0, s>>>(t.rad, t.vcdf);
    k_disk_vertical<<<((VC_NK + 1) * 32 + 255) / 256, 256, 0, s>>>(g, t.iz);
    k_disk_rotation<<<(KD * 32 + 255) / 256, 256, 0, s>>>(g, t.rad, t.iz, t.disk);
    k_disk_kappa<<<KD / 256, 256, 0, s>>>(g, t.disk);
    k_disk_kinematics<<<KD / 256, 256, 0, s>>>(g, t.disk);
    return cudaGetLastError() == cudaSuccess ? BONSAI_OK : BONSAI_ECUDA;
}

constexpr size_t RAD_BYTES = sizeof(double) * (size_t)NRAD * K;
constexpr size_t VCDF_BYTES = sizeof(double) * (size_t)2 * K * V;
constexpr size_t DISK_BYTES = sizeof(double) * (size_t)NDISK * KD;
constexpr size_t IZ_BYTES = sizeof(double) * (size_t)(VC_NK + 2);

struct Scratch {
    unsigned char *p = nullptr;
    cudaStream_t s;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() {
        if (p) cudaFreeAsync(p, s);
    }
};

}  // namespace

extern "C" int bonsai_galaxy_sec4(bonsai_galaxy *g, int64_t n, uint64_t seed) {
    if (!g || n < 1 || n > (int64_t)0xFFFFFFFFll) return BONSAI_EINVAL;
    // counts in the ratio of the 51 G-particle realisation of Sec. IV
    const int64_t b = 994689024ll, d = 2945105920ll, h = 47260172288ll, tot = b + d + h;
    const unsigned __int128 nn = (unsigned __int128)n;
    g->n_bulge = (int64_t)(nn * b / tot);
    g->n_disk = (int64_t)(nn * d / tot);
    g->n_halo = n - g->n_disk - g->n_bulge;
    g->seed = seed;
    g->G = 4.30091727e-6 * (1.0227121650537077e-3 * 1.0227121650537077e-3);
    g->M_halo = 6.0e11;
    g->a_halo = 15.0;
    g->M_bulge = 4.6e9;
    g->a_bulge = 0.5;
    g->r_t = 200.0;
    g->dr_t = 20.0;
    g->M_disk = 5.0e10;
    g->R_d = 2.5;
    g->z0 = 0.3;
    g->R_max = 30.0;
    g->Q = 1.5;
    g->R_Q = 2.43 * 2.5;
    return BONSAI_OK;
}

extern "C" int bonsai_galaxy_tables(const bonsai_galaxy *g, double *radial, double *vcdf,
                                    double *disk, void *stream) {
    int rc = check(g);
    if (rc != BONSAI_OK) return rc;
    if (!radial || !disk) return BONSAI_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch sc(s);
    if (cudaMallocAsync((void **)&sc.p, RAD_BYTES + VCDF_BYTES + DISK_BYTES + IZ_BYTES, s) !=
        cudaSuccess) {
        cudaGetLastError();
        return BONSAI_ENOMEM;
    }
    IcsTables t{reinterpret_cast<double *>(sc.p), reinterpret_cast<double *>(sc.p + RAD_BYTES),
                reinterpret_cast<double *>(sc.p + RAD_BYTES + VCDF_BYTES),
                reinterpret_cast<double *>(sc.p + RAD_BYTES + VCDF_BYTES + DISK_BYTES)};
    rc = build_tables(*g, t, s);
    if (rc != BONSAI_OK) return rc;
    if (cudaMemcpyAsync(radial, t.rad, sizeof(double) * (size_t)BONSAI_ICS_NRAD_OUT * K,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        (vcdf && cudaMemcpyAsync(vcdf, t.vcdf, VCDF_BYTES, cudaMemcpyDeviceToDevice, s) !=
                     cudaSuccess) ||
        cudaMemcpyAsync(disk, t.disk, sizeof(double) * (size_t)BONSAI_ICS_NDISK_OUT * KD,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return BONSAI_ECUDA;
    return bgb::wait_stream(s);
}

extern "C" int bonsai_galaxy_generate(const bonsai_galaxy *g, double *pos, double *vel,
                                      double *mass, void *stream) {
    int rc = check(g);
    if (rc != BONSAI_OK) return rc;
    const int64_t n = g->n_halo + g->n_disk + g->n_bulge;
    if (n == 0) return BONSAI_OK;
    if (!pos || !vel || !mass) return BONSAI_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return BONSAI_ECUDA;
    const int nparts = sms * 4;
    Scratch sc(s);
    const size_t part_bytes = sizeof(double) * 7 * (size_t)nparts;
    if (cudaMallocAsync((void **)&sc.p, RAD_BYTES + VCDF_BYTES + DISK_BYTES + IZ_BYTES + part_bytes,
                        s) != cudaSuccess) {
        cudaGetLastError();
        return BONSAI_ENOMEM;
    }
    IcsTables t{reinterpret_cast<double *>(sc.p), reinterpret_cast<double *>(sc.p + RAD_BYTES),
                reinterpret_cast<double *>(sc.p + RAD_BYTES + VCDF_BYTES),
                reinterpret_cast<double *>(sc.p + RAD_BYTES + VCDF_BYTES + DISK_BYTES)};
    double *part =
        reinterpret_cast<double *>(sc.p + RAD_BYTES + VCDF_BYTES + DISK_BYTES + IZ_BYTES);
    rc = build_tables(*g, t, s);
    if (rc != BONSAI_OK) return rc;
    SampleArgs A{*g, t.rad, t.vcdf, t.disk, pos, vel, mass, n};
    const int64_t want = (n + 255) / 256;
    const int blocks = (int)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
    k_sample<<<blocks, 256, 0, s>>>(A);
    k_moments<<<nparts, MOM_T, 0, s>>>(pos, vel, mass, n, part);
    k_shift<<<blocks, 256, 0, s>>>(pos, vel, n, part, nparts);
    if (cudaGetLastError() != cudaSuccess) return BONSAI_ECUDA;
    return bgb::wait_stream(s);
}
