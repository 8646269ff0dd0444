"""FP64 CPU oracle of the on-the-fly galaxy initial conditions (test
infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the CUDA library never does).

Sec. IV builds its Milky Way model on the fly instead of reading an initial
condition file: an NFW dark-matter halo (6.0e11 Msun), an exponential
stellar disk (5.0e10 Msun) and a Hernquist bulge (4.6e9 Msun), realised with
GalacticICS (smooth exponential disk, spherical bulge and halo).  This
module states, step by step in plain numpy, what the GPU generator computes:

1. A logarithmic radial grid r_k (K nodes), the tapered spheroid densities
   rho_c = rho0_c / (x (1 + x)^beta_c) * C(r), x = r / a_c, beta = 2 (NFW)
   or 3 (Hernquist), C(r) = erfc((r - r_t) / (sqrt(2) dr_t)) / 2, with
   their first and second radial derivatives in closed form; cumulative
   masses by the trapezoid rule in ln r; rho0_c sets each total mass.
2. The spherically averaged potential of all three components,
   Psi(r) = G M(<r) / r + G int_r (dM/dr') d ln r', where the disk enters
   through its mass inside the sphere of radius r (the sech^2 layer's
   density averaged over each sphere, Simpson in the polar angle).
3. Each spheroid's isotropic distribution function by Eddington's formula,
   f(E) = 1/(sqrt(8) pi^2) int_Psimin^E d2rho/dPsi2 dPsi / sqrt(E - Psi),
   with d2rho/dPsi2 = (rho'' Psi' - rho' Psi'') / Psi'^3 from the radial
   derivatives and the integral taken exactly for a piecewise-linear
   integrand between grid nodes.  The surface term vanishes: the taper
   makes rho and its derivative zero (to FP64) at the edge of the grid.
4. Per grid radius, the cumulative distribution of the speed fraction
   q = v / v_esc, p(q) ~ q^2 f(Psimin + (1 - q^2)(Psi - Psimin)), on V nodes.
5. The disk: R from the truncated exponential surface density (cumulative
   in closed form on a linear grid), z = z0 atanh(2u - 1) (sech^2),
   Gaussian velocities: sigma_R^2 proportional to Sigma, scaled so that
   Toomre's sigma_R kappa / (3.36 G Sigma) equals Q at R_Q = 2.43 R_d
   (Hernquist 1993: Q set at the solar radius, 2.43 scale lengths); the
   epicyclic sigma_phi = sigma_R kappa / (2 Omega); the isothermal-sheet
   sigma_z^2 = pi G Sigma z0; and the mean rotation from the asymmetric
   drift, v_phi^2 = v_c^2 + sigma_R^2 (1 - kappa^2 / (4 Omega^2) - 2 R /
   R_d), held within [0, v_c^2] (the epicyclic closure fails where sigma_R
   approaches v_c, near the centre, and would make the disk rotate faster
   than circular), in the potential of the spheroids (their enclosed mass)
   plus the disk's own midplane force (the Hankel integral of the
   exponential disk with e^{-k|z|} averaged over its sech^2 layer).
6. Sampling: every particle draws its uniforms from Philox4x32-10 (Salmon,
   Moraes, Dror & Shaw, SC11) with counter (particle index, component,
   call, 0) and key (seed low, seed high); each uniform takes two 32-bit
   words.  Radii and speed fractions are inverted from the tables by binary
   search and linear interpolation; directions are isotropic.
7. Equal masses within each component; the centre of mass and the mean
   velocity are moved to zero.

The disk's kinematics are the epicyclic (Jeans) approximation, not a disk
distribution function: the spheroids are in equilibrium in the spherically
averaged potential, the disk approximately so.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

K = 4096       # radial grid nodes of the spheroid tables
V = 256        # speed-fraction nodes of a velocity table row
KD = 4096      # radial grid nodes of the disk tables
R_MIN = 1.0e-4  # kpc: inner edge of the spheroid grid
R_MAX = 600.0   # kpc: outer edge of the spheroid grid

# Particle counts of the 51 G-particle model of Sec. IV: bulge, disk, halo.
PAPER_COUNTS = (994_689_024, 2_945_105_920, 47_260_172_288)
G_KPC_MSUN_MYR = 4.30091727e-6 * (1.0227121650537077e-3) ** 2


@dataclass
class Galaxy:
    """Model parameters (kpc, Msun, Myr).  Masses are the components' total
    masses; the spheroids carry the outer taper C(r)."""
    n_halo: int
    n_disk: int
    n_bulge: int
    seed: int = 1006
    G: float = G_KPC_MSUN_MYR
    M_halo: float = 6.0e11
    a_halo: float = 15.0
    M_bulge: float = 4.6e9
    a_bulge: float = 0.5
    r_t: float = 200.0
    dr_t: float = 20.0
    M_disk: float = 5.0e10
    R_d: float = 2.5
    z0: float = 0.3
    R_max: float = 30.0
    Q: float = 1.5
    R_Q: float = 6.075

    @property
    def n(self) -> int:
        return self.n_halo + self.n_disk + self.n_bulge


def counts(n: int):
    """Halo, disk and bulge counts for n particles in the ratio of the
    paper's realisation (floor for bulge and disk, the rest to the halo)."""
    tot = sum(PAPER_COUNTS)
    n_b = n * PAPER_COUNTS[0] // tot
    n_d = n * PAPER_COUNTS[1] // tot
    return n - n_d - n_b, n_d, n_b


def milky_way_sec4(n: int, seed: int = 1006) -> Galaxy:
    h, d, b = counts(n)
    return Galaxy(h, d, b, seed=seed)


# ---------------------------------------------------------------------------
# Philox4x32-10
# ---------------------------------------------------------------------------

_PM0, _PM1 = 0xD2511F53, 0xCD9E8D57
_PW0, _PW1 = 0x9E3779B9, 0xBB67AE85
_M32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten rounds of Philox4x32: each round multiplies words 0 and 2 by the
    two round constants (64-bit products), swaps and xors the high halves
    with words 1 and 3 and the key; the key advances by the Weyl constants
    between rounds.  Inputs broadcast; returns four uint32 arrays."""
    c = [np.asarray(x, dtype=np.uint64) & _M32 for x in (c0, c1, c2, c3)]
    k0 = np.asarray(k0, dtype=np.uint64) & _M32
    k1 = np.asarray(k1, dtype=np.uint64) & _M32
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(_PW0)) & _M32
            k1 = (k1 + np.uint64(_PW1)) & _M32
        p0 = c[0] * np.uint64(_PM0)
        p1 = c[2] * np.uint64(_PM1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & _M32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _M32
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return [x.astype(np.uint32) for x in c]


def uniform52(wa, wb):
    """(m + 1/2) / 2^52 with the 52-bit m = (wa >> 6) 2^26 + (wb >> 6):
    exact in FP64, inside (0, 1)."""
    m = (np.asarray(wa, np.uint64) >> np.uint64(6)) * np.uint64(1 << 26) + (
        np.asarray(wb, np.uint64) >> np.uint64(6))
    return (m.astype(np.float64) + 0.5) * 2.0 ** -52


def draws(idx, comp, call, seed):
    """Two uniforms from Philox call ``call`` of particles idx."""
    w = philox4x32_10(idx, comp, call, 0, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return uniform52(w[0], w[1]), uniform52(w[2], w[3])


# ---------------------------------------------------------------------------
# Step 1-2: spheroid profiles and the spherical potential
# ---------------------------------------------------------------------------

def radial_grid():
    dl = math.log(R_MAX / R_MIN) / (K - 1)
    return R_MIN * np.exp(dl * np.arange(K)), dl


def taper(r, rt, drt):
    """C(r) and its first two radial derivatives."""
    from scipy.special import erfc
    y = (r - rt) / (math.sqrt(2.0) * drt)
    C = 0.5 * erfc(y)
    C1 = -np.exp(-y * y) / (math.sqrt(2.0 * math.pi) * drt)
    C2 = -C1 * (r - rt) / (drt * drt)
    return C, C1, C2


def spheroid_shape(r, a, beta, rt, drt):
    """rho/rho0 = C(r) / (x (1 + x)^beta), x = r/a, with d/dr and d2/dr2."""
    x = r / a
    h = 1.0 / (x * (1.0 + x) ** beta)
    L1 = -1.0 / r - beta / (a + r)
    L1p = 1.0 / (r * r) + beta / ((a + r) * (a + r))
    h1 = h * L1
    h2 = h * (L1 * L1 + L1p)
    C, C1, C2 = taper(r, rt, drt)
    return h * C, h1 * C + h * C1, h2 * C + 2.0 * h1 * C1 + h * C2


def inner_mass_shape(r0, a, beta, C0):
    """int_0^r0 4 pi r^2 C0 / (x (1 + x)^beta) dr in closed form (the taper
    taken constant, C0 = C(r0)): 4 pi a^3 C0 times ln(1+x) - x/(1+x) for
    beta = 2 and x^2 / (2 (1+x)^2) for beta = 3, x = r0 / a."""
    x = r0 / a
    if beta == 2.0:
        I = math.log1p(x) - x / (1.0 + x)
    elif beta == 3.0:
        I = x * x / (2.0 * (1.0 + x) * (1.0 + x))
    else:
        raise ValueError(beta)
    return 4.0 * math.pi * a ** 3 * C0 * I


def cumulative_mass_shape(r, dl, a, beta, shape, C0):
    """int_0^r 4 pi r'^2 shape dr': the closed-form inner part below the
    first node, then the trapezoid rule in ln r."""
    F = 4.0 * math.pi * r ** 3 * shape
    S = np.empty_like(r)
    S[0] = inner_mass_shape(r[0], a, beta, C0)
    S[1:] = S[0] + np.cumsum(0.5 * (F[1:] + F[:-1]) * dl)
    return S


def disk_fraction(x):
    """1 - (1 + x) e^-x: the alternating series sum_{k>=2} (-1)^k (k-1) x^k / k!
    (22 terms) below x = 1/2, where the closed form cancels; the closed form
    above."""
    x = np.asarray(x, dtype=np.float64)
    s = np.zeros_like(x)
    t = x * x / 2.0            # x^k / k! at k = 2
    for k in range(2, 24):
        s = s + (1.0 if k % 2 == 0 else -1.0) * (k - 1) * t
        t = t * x / (k + 1)
    return np.where(x < 0.5, s, 1.0 - (1.0 + x) * np.exp(-x))


SHELL_N = 2048   # Simpson intervals of the disk's spherical shell average
VC_NK = 4000     # Simpson intervals of the disk's Hankel integral in k
VC_KMAX = 40.0   # k range, in units of 1 / R_d
IZ_NT = 4096     # Simpson intervals of the vertical factor in t = z / z0
IZ_TMAX = 40.0


def simpson(y, h, axis=-1):
    """Composite Simpson rule of samples y (an odd count) with step h."""
    y = np.moveaxis(np.asarray(y), axis, -1)
    return h / 3.0 * (y[..., 0] + y[..., -1] + 4.0 * y[..., 1:-1:2].sum(-1) + 2.0 * y[..., 2:-1:2].sum(-1))


def disk_sigma0(g: Galaxy):
    """Central surface density of the truncated disk (total mass M_disk)."""
    return g.M_disk / (2.0 * math.pi * g.R_d * g.R_d * float(disk_fraction(g.R_max / g.R_d)))


def disk_shell_rate(r, g: Galaxy):
    """dM/dr of the disk, rho = Sigma0 e^{-R/R_d} sech^2(z/z0) / (2 z0) for
    R <= R_max: 4 pi r^2 times the density averaged over the sphere of
    radius r, int_0^{pi/2} rho(r cos phi, r sin phi) cos phi dphi, by
    Simpson's rule on [phi_lo, phi_hi] with phi_hi = asin(min(1, 40 z0 / r))
    (sech^2 < 1e-34 beyond) and phi_lo = acos(min(1, R_max / r)) (the disk
    ends at R_max)."""
    sig0 = disk_sigma0(g)
    out = np.zeros_like(r)
    for k, rk in enumerate(r):
        hi = math.asin(min(1.0, IZ_TMAX * g.z0 / rk))
        lo = math.acos(min(1.0, g.R_max / rk))
        if hi <= lo:
            continue
        phi = lo + (hi - lo) * np.arange(SHELL_N + 1) / SHELL_N
        R, z = rk * np.cos(phi), rk * np.sin(phi)
        rho = sig0 * np.exp(-R / g.R_d) / (2.0 * g.z0) / np.cosh(z / g.z0) ** 2
        out[k] = 4.0 * math.pi * rk * rk * simpson(rho * np.cos(phi), (hi - lo) / SHELL_N)
    return out


def disk_sph_mass(r, dl, g: Galaxy):
    """Mass of the disk inside radius r and its r-derivative: the shell rate
    above, integrated by the trapezoid rule in ln r from the mass of the
    central density inside the first node."""
    dM = disk_shell_rate(r, g)
    F = r * dM
    M = np.empty_like(r)
    M[0] = 4.0 / 3.0 * math.pi * r[0] ** 3 * disk_sigma0(g) / (2.0 * g.z0)
    M[1:] = M[0] + np.cumsum(0.5 * (F[1:] + F[:-1]) * dl)
    return M, dM


def profiles(g: Galaxy):
    """Grid, component densities (with derivatives), masses and Psi."""
    r, dl = radial_grid()
    comp = {}
    for name, M, a, beta in (("halo", g.M_halo, g.a_halo, 2.0), ("bulge", g.M_bulge, g.a_bulge, 3.0)):
        s0, s1, s2 = spheroid_shape(r, a, beta, g.r_t, g.dr_t)
        S = cumulative_mass_shape(r, dl, a, beta, s0, float(taper(r[:1], g.r_t, g.dr_t)[0][0]))
        rho0 = M / S[-1]
        comp[name] = {"rho": rho0 * s0, "rho1": rho0 * s1, "rho2": rho0 * s2, "M": rho0 * S,
                      "P": S / S[-1]}
    Md, dMd = disk_sph_mass(r, dl, g)
    Mt = comp["halo"]["M"] + comp["bulge"]["M"] + Md
    dMt = 4.0 * math.pi * r * r * (comp["halo"]["rho"] + comp["bulge"]["rho"]) + dMd
    seg = 0.5 * (dMt[1:] + dMt[:-1]) * dl
    O = np.zeros(K)
    O[:-1] = np.cumsum(seg[::-1])[::-1]
    Psi = g.G * (Mt / r + O)
    d1 = -g.G * Mt / (r * r)
    d2 = 2.0 * g.G * Mt / r ** 3 - g.G * dMt / (r * r)
    return {"r": r, "dl": dl, "Mt": Mt, "dMt": dMt, "Psi": Psi, "Psi1": d1, "Psi2": d2, "comp": comp}


# ---------------------------------------------------------------------------
# Step 3-4: Eddington inversion and speed tables
# ---------------------------------------------------------------------------

def eddington(Psi, g2):
    """f(E_j) at E_j = Psi_j: 1/(sqrt(8) pi^2) times the integral of g2 /
    sqrt(E - Psi) from Psi_min = Psi[-1] to E, exact for g2 linear in Psi
    between nodes.  Negative values (rounding, at the lowest energies) are
    set to zero."""
    n = Psi.size
    f = np.zeros(n)
    pa, pb = Psi[1:], Psi[:-1]          # segment k spans [Psi_{k+1}, Psi_k]
    ga, gb = g2[1:], g2[:-1]
    slope = (gb - ga) / (pb - pa)
    for j in range(n - 1):
        E = Psi[j]
        sa = E - pa[j:]
        sb = E - pb[j:]
        rsa, rsb = np.sqrt(sa), np.sqrt(sb)
        D = (pb[j:] - pa[j:]) / (rsa + rsb)
        A = ga[j:] + slope[j:] * sa
        seg = 2.0 * A * D - (2.0 / 3.0) * slope[j:] * D * (sa + rsa * rsb + sb)
        f[j] = seg.sum()
    f *= 1.0 / (math.sqrt(8.0) * math.pi * math.pi)
    return np.maximum(f, 0.0)


def interp_desc(x, xs, ys):
    """Linear interpolation on a strictly decreasing abscissa xs, clamped."""
    return np.interp(-np.asarray(x), -xs, ys)


def speed_cdf(Psi, f):
    """Row k: normalised cumulative of q^2 f(Psi_min + (1 - q^2)(Psi_k - Psi_min))
    on q_m = m/(V-1) by the trapezoid rule; a row without mass is uniform."""
    q = np.arange(V) / (V - 1.0)
    w = Psi - Psi[-1]
    E = Psi[-1] + (1.0 - q[None, :] ** 2) * w[:, None]
    p = q[None, :] ** 2 * interp_desc(E, Psi, f)
    C = np.zeros((Psi.size, V))
    C[:, 1:] = np.cumsum(0.5 * (p[:, 1:] + p[:, :-1]) / (V - 1.0), axis=1)
    tot = C[:, -1].copy()
    ok = tot > 0.0
    C[ok] /= tot[ok, None]
    C[~ok] = q[None, :]
    return C, tot


# ---------------------------------------------------------------------------
# Step 5: disk tables
# ---------------------------------------------------------------------------

def freeman_vc2(R, G, Md, Rd):
    """Circular speed squared in the plane of a thin exponential disk
    (Freeman 1970), the thin limit of disk_vc2 (used by the tests)."""
    from scipy import special
    y = R / (2.0 * Rd)
    s0 = Md / (2.0 * math.pi * Rd * Rd)
    return 4.0 * math.pi * G * s0 * Rd * y * y * (
        special.i0(y) * special.k0(y) - special.i1(y) * special.k1(y))


def vertical_factor(kz):
    """I(k z0) = int_0^inf sech^2(t) e^{-k z0 t} dt (the sech^2 layer's
    weight of e^{-k|z|}; 1 for a thin disk), Simpson on t in [0, 40]."""
    t = IZ_TMAX * np.arange(IZ_NT + 1) / IZ_NT
    kz = np.asarray(kz, dtype=np.float64)
    y = np.exp(-kz[..., None] * t) / np.cosh(t) ** 2
    return simpson(y, IZ_TMAX / IZ_NT)


def disk_vc2(R, g: Galaxy):
    """Circular speed squared in the midplane of the sech^2 exponential disk
    (surface density Sigma0 e^{-R/R_d}, Sigma0 = M_disk / (2 pi R_d^2)):
    v_c^2 = 2 pi G Sigma0 R_d^2 R int_0^inf k J1(kR) I(k z0) (1 + k^2 R_d^2)^{-3/2} dk
    (the thin disk's Hankel form with e^{-k|z|} averaged over the layer), by
    Simpson's rule on k in [0, 40 / R_d]."""
    from scipy import special
    s0 = g.M_disk / (2.0 * math.pi * g.R_d * g.R_d)
    hk = VC_KMAX / g.R_d / VC_NK
    k = hk * np.arange(VC_NK + 1)
    w = k * vertical_factor(k * g.z0) * (1.0 + (k * g.R_d) ** 2) ** -1.5
    R = np.asarray(R, dtype=np.float64)
    out = np.empty_like(R)
    for a in range(0, R.size, 256):
        Rb = R[a:a + 256]
        out[a:a + 256] = simpson(special.j1(Rb[:, None] * k[None, :]) * w[None, :], hk)
    return 2.0 * math.pi * g.G * s0 * g.R_d * g.R_d * R * out


def central_diff(y, h):
    d = np.empty_like(y)
    d[1:-1] = (y[2:] - y[:-2]) / (2.0 * h)
    d[0] = (y[1] - y[0]) / h
    d[-1] = (y[-1] - y[-2]) / h
    return d


def sph_mass_at(pr, name, R):
    """Enclosed spheroid mass at radius R: linear in ln r between nodes,
    ~ r^2 below the first node."""
    r, M = pr["r"], pr["comp"][name]["M"]
    lr = np.log(np.maximum(R, r[0]))
    out = np.interp(lr, np.log(r), M)
    return np.where(R < r[0], M[0] * (R / r[0]) ** 2, out)


def disk_tables(g: Galaxy, pr):
    h = g.R_max / (KD - 1)
    Rc = np.arange(KD) * h                    # cumulative-mass grid
    x = Rc / g.R_d
    xm = g.R_max / g.R_d
    cdf = disk_fraction(x) / disk_fraction(xm)
    cdf[-1] = 1.0
    R = (np.arange(KD) + 0.5) * h            # kinematic grid
    msph = sph_mass_at(pr, "halo", R) + sph_mass_at(pr, "bulge", R)
    vc2 = g.G * msph / R + disk_vc2(R, g)
    om2 = vc2 / (R * R)
    kap2 = R * central_diff(om2, h) + 4.0 * om2
    kap = np.sqrt(np.maximum(kap2, 1e-30))
    s0 = g.M_disk / (2.0 * math.pi * g.R_d * g.R_d)
    Sig = s0 * np.exp(-R / g.R_d)
    # kappa at R_Q: linear between the kinematic nodes, clamped
    sq = min(max(g.R_Q / h - 0.5, 0.0), KD - 1.0)
    iq = min(int(sq), KD - 2)
    kq = (1.0 - (sq - iq)) * kap[iq] + (sq - iq) * kap[iq + 1]
    sRq = g.Q * 3.36 * g.G * s0 * math.exp(-g.R_Q / g.R_d) / kq
    sR = sRq * np.exp(-(R - g.R_Q) / (2.0 * g.R_d))
    sphi = sR * kap / (2.0 * np.sqrt(om2))
    sz = np.sqrt(math.pi * g.G * Sig * g.z0)
    vphi = np.sqrt(np.clip(vc2 + sR * sR * (1.0 - kap2 / (4.0 * om2) - 2.0 * R / g.R_d), 0.0, vc2))
    return {"h": h, "cdf": cdf, "R": R, "vc2": vc2, "kappa": kap, "sR": sR, "sphi": sphi,
            "sz": sz, "vphi": vphi, "kappa_Q": kq}


def tables(g: Galaxy):
    pr = profiles(g)
    out = {"prof": pr}
    for name in ("halo", "bulge"):
        c = pr["comp"][name]
        g2 = (c["rho2"] * pr["Psi1"] - c["rho1"] * pr["Psi2"]) / pr["Psi1"] ** 3
        f = eddington(pr["Psi"], g2)
        C, tot = speed_cdf(pr["Psi"], f)
        out[name] = {"g2": g2, "f": f, "vcdf": C, "vnorm": tot}
    out["disk"] = disk_tables(g, pr)
    return out


# ---------------------------------------------------------------------------
# Step 6-7: sampling
# ---------------------------------------------------------------------------

def _search(table, u, rows=None):
    """Largest m in [0, n - 2] with table[m] <= u, by bisection (n = last axis;
    ``rows`` picks a row of a 2-D table per element)."""
    n = table.shape[-1]
    u = np.asarray(u)
    lo = np.zeros(u.shape, np.int64)
    hi = np.full(u.shape, n - 1, np.int64)
    while np.any(hi - lo > 1):
        mid = (lo + hi) // 2
        tv = table[mid] if rows is None else table[rows, mid]
        le = tv <= u
        lo = np.where(le, mid, lo)
        hi = np.where(le, hi, mid)
    return lo


def _invert_row(C, k, u):
    """q with C[k](q) = u (row-wise inverse of the speed cdf)."""
    m = _search(C, u, rows=k)
    c0 = C[k, m]
    c1 = C[k, m + 1]
    return (m + (u - c0) / (c1 - c0)) / (V - 1.0)


def _isotropic(uc, up):
    c = 2.0 * uc - 1.0
    s = np.sqrt((1.0 - c) * (1.0 + c))
    ph = 2.0 * math.pi * up
    return np.stack([s * np.cos(ph), s * np.sin(ph), c])


def sample_spheroid(g: Galaxy, tb, name, first, count, comp_id):
    pr = tb["prof"]
    r_nodes, dl, Psi = pr["r"], pr["dl"], pr["Psi"]
    P = pr["comp"][name]["P"]
    C = tb[name]["vcdf"]
    idx = np.arange(first, first + count, dtype=np.uint64)
    ur, uc = draws(idx, comp_id, 0, g.seed)
    up, uv = draws(idx, comp_id, 1, g.seed)
    uvc, uvp = draws(idx, comp_id, 2, g.seed)
    inner = ur < P[0]
    k = _search(P, ur)
    t = np.where(inner, 0.0, (ur - P[k]) / (P[k + 1] - P[k]))
    k = np.where(inner, 0, k)
    r = np.where(inner, r_nodes[0] * np.sqrt(ur / P[0]), r_nodes[k] * np.exp(t * dl))
    q = (1.0 - t) * _invert_row(C, k, uv) + t * _invert_row(C, k + 1, uv)
    psi = (1.0 - t) * Psi[k] + t * Psi[k + 1]
    v = q * np.sqrt(2.0 * (psi - Psi[-1]))
    return _isotropic(uc, up) * r, _isotropic(uvc, uvp) * v


def sample_disk(g: Galaxy, tb, first, count, comp_id=1):
    d = tb["disk"]
    idx = np.arange(first, first + count, dtype=np.uint64)
    uR, uz = draws(idx, comp_id, 0, g.seed)
    up, ua = draws(idx, comp_id, 1, g.seed)
    ub, uc = draws(idx, comp_id, 2, g.seed)
    ud, _ = draws(idx, comp_id, 3, g.seed)
    j = _search(d["cdf"], uR)
    R = (j + (uR - d["cdf"][j]) / (d["cdf"][j + 1] - d["cdf"][j])) * d["h"]
    z = g.z0 * np.arctanh(2.0 * uz - 1.0)
    ph = 2.0 * math.pi * up
    # kinematic tables at (j + 1/2) h: linear in R, clamped at the ends
    s = np.clip(R / d["h"] - 0.5, 0.0, KD - 1.0)
    i0 = np.minimum(s.astype(np.int64), KD - 2)
    w = s - i0

    def at(a):
        return (1.0 - w) * a[i0] + w * a[i0 + 1]
    rho1 = np.sqrt(-2.0 * np.log(ua))
    rho2 = np.sqrt(-2.0 * np.log(uc))
    n1 = rho1 * np.cos(2.0 * math.pi * ub)
    n2 = rho1 * np.sin(2.0 * math.pi * ub)
    n3 = rho2 * np.cos(2.0 * math.pi * ud)
    vR = at(d["sR"]) * n1
    vp = at(d["vphi"]) + at(d["sphi"]) * n2
    vz = at(d["sz"]) * n3
    c, sn = np.cos(ph), np.sin(ph)
    return np.stack([R * c, R * sn, z]), np.stack([vR * c - vp * sn, vR * sn + vp * c, vz])


def generate(g: Galaxy, tb=None):
    """Positions (3, N), velocities (3, N) and masses (N,): halo, disk, bulge
    in that order; centre of mass and mean velocity at zero."""
    tb = tables(g) if tb is None else tb
    hp, hv = sample_spheroid(g, tb, "halo", 0, g.n_halo, 0)
    dp, dv = sample_disk(g, tb, g.n_halo, g.n_disk, 1)
    bp, bv = sample_spheroid(g, tb, "bulge", g.n_halo + g.n_disk, g.n_bulge, 2)
    pos = np.concatenate([hp, dp, bp], axis=1)
    vel = np.concatenate([hv, dv, bv], axis=1)
    mass = np.concatenate([np.full(g.n_halo, g.M_halo / max(g.n_halo, 1)),
                           np.full(g.n_disk, g.M_disk / max(g.n_disk, 1)),
                           np.full(g.n_bulge, g.M_bulge / max(g.n_bulge, 1))])
    mt = mass.sum()
    pos -= (pos * mass).sum(axis=1, keepdims=True) / mt
    vel -= (vel * mass).sum(axis=1, keepdims=True) / mt
    return pos, vel, mass
