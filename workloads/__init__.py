"""Seeded synthetic initial conditions shared by the CUDA path and the oracle.

This module holds no arithmetic of the tree method: it only draws particle
positions, velocities and masses (numpy PCG64, host FP64) with the shapes of
the paper's workloads, which are not available here (the 51 G-particle Milky
Way realisation of Sec. IV was made with GalacticICS).  The same arrays feed
both implementations.

Units: ``plummer`` uses G = M = a = 1.  The galaxy models use kpc, Msun and
Myr, for which G = 4.4985e-12 kpc^3 Msun^-1 Myr^-2.

Arrays are SoA: positions and velocities ``(3, N)`` float64, masses ``(N,)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# G = 4.30091727e-6 kpc (km/s)^2 / Msun, and 1 km/s = 1.0227121650537077e-3 kpc/Myr
G_KPC_MSUN_MYR = 4.30091727e-6 * (1.0227121650537077e-3) ** 2


@dataclass
class Model:
    pos: np.ndarray   # (3, N) float64
    vel: np.ndarray   # (3, N) float64
    mass: np.ndarray  # (N,) float64
    G: float
    eps: float
    theta: float
    dt: float
    name: str
    components: dict  # name -> (start, count)

    @property
    def n(self) -> int:
        return int(self.mass.shape[0])


def _isotropic(rng, n):
    u = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    s = np.sqrt(1.0 - u * u)
    return np.stack([s * np.cos(ph), s * np.sin(ph), u])


def plummer(n: int, seed: int = 1001, rmax: float = 100.0, G: float = 1.0, M: float = 1.0,
            a: float = 1.0, eps: float = 0.01, theta: float = 0.4, dt: float = 1.0 / 64) -> Model:
    """Equal-mass Plummer sphere sampled from its isotropic distribution
    function (Aarseth, Henon & Wielen 1974): r from the cumulative mass,
    speeds by rejection from q^2 (1 - q^2)^{7/2}.  Radii beyond ``rmax`` are
    redrawn.  Centre of mass and mean velocity are shifted to zero."""
    rng = np.random.default_rng(seed)
    r = np.empty(n)
    k = 0
    while k < n:
        u = rng.uniform(0.0, 1.0, 2 * (n - k) + 16)
        u = u[u > 0.0]
        rr = 1.0 / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        rr = rr[rr <= rmax][: n - k]
        r[k:k + rr.size] = rr
        k += rr.size
    pos = _isotropic(rng, n) * r * a
    q = np.empty(n)
    k = 0
    while k < n:
        m = 2 * (n - k) + 64
        x = rng.uniform(0.0, 1.0, m)
        y = rng.uniform(0.0, 0.1, m)
        ok = x[y < x * x * (1.0 - x * x) ** 3.5][: n - k]
        q[k:k + ok.size] = ok
        k += ok.size
    v = q * math.sqrt(2.0) * (1.0 + r * r) ** (-0.25) * math.sqrt(G * M / a)
    vel = _isotropic(rng, n) * v
    mass = np.full(n, M / n)
    pos -= (pos * mass).sum(axis=1, keepdims=True) / mass.sum()
    vel -= (vel * mass).sum(axis=1, keepdims=True) / mass.sum()
    return Model(pos, vel, mass, G, eps, theta, dt, f"plummer-{n}", {"all": (0, n)})


# -------------------------------------------------------------------------
# Milky-Way-like model: Hernquist halo + Hernquist bulge + exponential disk
# -------------------------------------------------------------------------

def _hernquist_r(rng, n, a, rcut):
    xmax = (rcut / (rcut + a)) ** 2
    s = np.sqrt(rng.uniform(0.0, xmax, n))
    return a * s / (1.0 - s)


def _hernquist_menc(r, M, a, rcut):
    """Enclosed mass of a Hernquist sphere whose mass inside rcut is M."""
    Mtot = M * (rcut + a) ** 2 / rcut ** 2
    rr = np.minimum(r, rcut)
    return Mtot * rr * rr / (rr + a) ** 2


def _hernquist_rho(r, M, a, rcut):
    Mtot = M * (rcut + a) ** 2 / rcut ** 2
    rho = Mtot * a / (2.0 * math.pi * r * (r + a) ** 3)
    return np.where(r <= rcut, rho, 0.0)


def _exp_disk_menc_sph(r, Md, Rd):
    # mass of the disk within cylindrical radius r, used as a spherical proxy
    x = r / Rd
    return Md * (1.0 - (1.0 + x) * np.exp(-x))


def _jeans_sigma2(rgrid, rho, menc_tot, G):
    """Isotropic Jeans equation: sigma_r^2(r) = (1/rho) int_r^inf rho G M(r')/r'^2 dr'."""
    f = rho * G * menc_tot / rgrid ** 2
    # cumulative trapezoid from the outside in
    seg = 0.5 * (f[1:] + f[:-1]) * np.diff(rgrid)
    tail = np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]])
    with np.errstate(invalid="ignore", divide="ignore"):
        s2 = np.where(rho > 0, tail / rho, 0.0)
    return s2


def _exp_disk(rng, n_d, M_disk, R_d, z0, R_max, Q_toomre, G, menc_other):
    """Exponential disk: R from Gamma(2, R_d) truncated at R_max, z = z0
    atanh(U) (sech^2), Toomre-Q radial dispersion, epicyclic azimuthal
    dispersion, vertical dispersion from the isothermal sheet, and the
    asymmetric-drift corrected mean rotation in the potential of the disk
    (Freeman's thin-disk circular speed) plus the spherical mass
    menc_other(R) of the other components."""
    from scipy import special

    R = np.empty(n_d)
    k = 0
    while k < n_d:
        rr = rng.gamma(2.0, R_d, 2 * (n_d - k) + 16)
        rr = rr[rr <= R_max][: n_d - k]
        R[k:k + rr.size] = rr
        k += rr.size
    phi = rng.uniform(0.0, 2.0 * math.pi, n_d)
    u = rng.uniform(-1.0, 1.0, n_d)
    u = np.clip(u, -1.0 + 1e-15, 1.0 - 1e-15)
    z = z0 * np.arctanh(u)

    Rg = np.linspace(0.01, R_max * 1.2, 4000)
    sigma0 = M_disk / (2.0 * math.pi * R_d * R_d)
    y = Rg / (2.0 * R_d)
    vdisk2 = 4.0 * math.pi * G * sigma0 * R_d * y * y * (
        special.i0(y) * special.k0(y) - special.i1(y) * special.k1(y))
    vc2 = G * menc_other(Rg) / Rg + vdisk2
    om2 = vc2 / (Rg * Rg)
    kap2 = Rg * np.gradient(om2, Rg) + 4.0 * om2
    kap = np.sqrt(np.maximum(kap2, 1e-30))
    Sig = sigma0 * np.exp(-Rg / R_d)
    sR = Q_toomre * 3.36 * G * Sig / kap
    sphi = sR * kap / (2.0 * np.sqrt(om2))
    sz = np.sqrt(math.pi * G * Sig * z0)
    # asymmetric drift: vphi^2 = vc^2 + sR^2 (1 - sphi^2/sR^2 + dln(Sig sR^2)/dlnR)
    dln = np.gradient(np.log(Sig * sR * sR), np.log(Rg))
    vphi2 = np.maximum(vc2 + sR * sR * (1.0 - (sphi * sphi) / (sR * sR) + dln), 0.0)
    vbar = np.sqrt(vphi2)

    vR = rng.standard_normal(n_d) * np.interp(R, Rg, sR)
    vphi = np.interp(R, Rg, vbar) + rng.standard_normal(n_d) * np.interp(R, Rg, sphi)
    vz = rng.standard_normal(n_d) * np.interp(R, Rg, sz)
    c, s = np.cos(phi), np.sin(phi)
    return np.stack([R * c, R * s, z]), np.stack([vR * c - vphi * s, vR * s + vphi * c, vz])


def milky_way(n: int, seed: int = 1002, eps: float = 0.01, theta: float = 0.4, dt: float = 0.1,
              ratio=(5.0, 1.0, 0.2), M_halo=1.0e12, a_halo=30.0, rcut=200.0, M_bulge=1.0e10,
              a_bulge=0.5, M_disk=5.0e10, R_d=2.5, z0=0.3, R_max=30.0, Q_toomre=1.5,
              G: float = G_KPC_MSUN_MYR, name: str | None = None) -> Model:
    """Milky-Way-like galaxy in kpc / Msun / Myr.

    Particle counts follow halo:disk:bulge = 5:1:0.2 (N_d = floor(N/6.2),
    N_b = floor(0.2 N_d), the halo takes the rest); masses are equal within
    each component.  Halo and bulge are Hernquist spheres truncated at rcut
    whose mass inside the cut is the stated mass, with isotropic Gaussian
    velocities of the Jeans dispersion in the total enclosed mass.  The disk
    is exponential in R (Gamma(2, R_d), truncated at R_max) and sech^2 in z,
    with Toomre-Q epicyclic velocity dispersions and an asymmetric-drift
    corrected mean rotation."""
    rng = np.random.default_rng(seed)
    tot = sum(ratio)
    n_d = int(math.floor(n * ratio[1] / tot))
    n_b = int(math.floor(n_d * ratio[2] / ratio[1]))
    n_h = n - n_d - n_b

    rgrid = np.logspace(-4, math.log10(rcut * 1.5), 4000)

    def menc_sph(r):
        return (_hernquist_menc(r, M_halo, a_halo, rcut) + _hernquist_menc(r, M_bulge, a_bulge, rcut)
                + _exp_disk_menc_sph(r, M_disk, R_d))

    mgrid = menc_sph(rgrid)

    def spheroid(nc, M, a):
        r = _hernquist_r(rng, nc, a, rcut)
        pos = _isotropic(rng, nc) * r
        s2 = _jeans_sigma2(rgrid, _hernquist_rho(rgrid, M, a, rcut), mgrid, G)
        sig = np.sqrt(np.interp(r, rgrid, s2))
        vel = rng.standard_normal((3, nc)) * sig
        return pos, vel

    hp, hv = spheroid(n_h, M_halo, a_halo)
    bp, bv = spheroid(n_b, M_bulge, a_bulge)

    dp, dv = _exp_disk(rng, n_d, M_disk, R_d, z0, R_max, Q_toomre, G,
                       lambda R: _hernquist_menc(R, M_halo, a_halo, rcut)
                       + _hernquist_menc(R, M_bulge, a_bulge, rcut))

    pos = np.concatenate([hp, dp, bp], axis=1)
    vel = np.concatenate([hv, dv, bv], axis=1)
    mass = np.concatenate([np.full(n_h, M_halo / n_h), np.full(n_d, M_disk / max(n_d, 1)),
                           np.full(n_b, M_bulge / max(n_b, 1))])
    mass = mass[: n]
    pos -= (pos * mass).sum(axis=1, keepdims=True) / mass.sum()
    vel -= (vel * mass).sum(axis=1, keepdims=True) / mass.sum()
    comps = {"halo": (0, n_h), "disk": (n_h, n_d), "bulge": (n_h + n_d, n_b)}
    return Model(np.ascontiguousarray(pos), np.ascontiguousarray(vel), mass, G, eps, theta, dt,
                 name or f"milky-way-{n}", comps)


def halo_disk(n_halo: int, n_disk: int, seed: int = 1004, eps: float = 0.02, theta: float = 0.4,
              dt: float = 0.1, M_halo=1.0e11, a_halo=10.0, rmax_halo=300.0, M_disk=5.0e10, R_d=2.5,
              z0=0.3, R_max=30.0, Q_toomre=1.5, G: float = G_KPC_MSUN_MYR) -> Model:
    """Plummer halo plus exponential disk in kpc / Msun / Myr (the model of
    the differentiable run): the halo is sampled from its own isotropic
    distribution function (radii beyond rmax_halo redrawn), the disk as in
    the Milky-Way-like model with its rotation in the potential of the disk
    plus the Plummer halo.  Equal masses within each component; centre of
    mass and mean velocity at rest."""
    rng = np.random.default_rng(seed)
    h = plummer(n_halo, seed=int(rng.integers(1 << 31)), rmax=rmax_halo / a_halo, G=G, M=M_halo,
                a=a_halo)

    def menc_plummer(R):
        return M_halo * R ** 3 / (R * R + a_halo * a_halo) ** 1.5

    dp, dv = _exp_disk(rng, n_disk, M_disk, R_d, z0, R_max, Q_toomre, G, menc_plummer)
    pos = np.concatenate([h.pos, dp], axis=1)
    vel = np.concatenate([h.vel, dv], axis=1)
    mass = np.concatenate([h.mass, np.full(n_disk, M_disk / max(n_disk, 1))])
    pos -= (pos * mass).sum(axis=1, keepdims=True) / mass.sum()
    vel -= (vel * mass).sum(axis=1, keepdims=True) / mass.sum()
    return Model(np.ascontiguousarray(pos), np.ascontiguousarray(vel), mass, G, eps, theta, dt,
                 f"halo-disk-{n_halo}+{n_disk}", {"halo": (0, n_halo), "disk": (n_halo, n_disk)})


def config_model(index: int, n: int | None = None) -> Model:
    """The benchmark workloads by index: 0 = Plummer sphere N = 2^14 (G = M = a = 1,
    eps = 0.01, dt = 1/64); 1 = Milky-Way-like N = 2^23 (eps = 10 pc, dt = 0.1 Myr).
    Seeds are 1000 + index + 1."""
    if index == 0:
        return plummer(n or (1 << 14), seed=1001)
    if index == 1:
        return milky_way(n or (1 << 23), seed=1002, eps=0.01, theta=0.4, dt=0.1)
    raise ValueError(index)
