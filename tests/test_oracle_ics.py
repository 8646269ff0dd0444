"""Pins of the oracle's on-the-fly galaxy initial conditions (Sec. IV: NFW
halo, exponential disk, Hernquist bulge, generated on the fly).

The generator's pieces are checked against what mathematics and published
results fix, not against themselves: Philox4x32-10 against the known-answer
vectors published with the generator (Salmon et al., SC11); Eddington's
inversion against Hernquist's closed-form distribution function (Hernquist
1990, Eq. 17); the distribution function against its own density (Eddington's
defining integral) and against the isotropic Jeans equation; sampled radii,
heights and speeds against their distributions; the virial theorem for a
sampled halo (forces by direct summation); Freeman's disk rotation against
its Keplerian limit and the position of its maximum; the thick disk's
vertical factor against its closed forms, its spherical mass against an
independent cylindrical integral, and its midplane rotation against
Freeman's curve in the thin limit."""
import math

import numpy as np
import pytest

import oracle
from oracle import galaxy_ics as gi


@pytest.mark.parametrize("ctr,key,want", [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
])
def test_philox_known_answers(ctr, key, want):
    got = gi.philox4x32_10(*ctr, *key)
    assert tuple(int(x) for x in got) == want


def test_uniforms_are_exact_and_inside_the_unit_interval():
    lo = gi.uniform52(0, 0)
    hi = gi.uniform52(0xFFFFFFFF, 0xFFFFFFFF)
    assert lo == 2.0 ** -53 and hi == 1.0 - 2.0 ** -53
    u0, u1 = gi.draws(np.arange(100000, dtype=np.uint64), 0, 0, 12345)
    for u in (u0, u1):
        assert u.min() > 0.0 and u.max() < 1.0
        assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)
    assert abs(np.corrcoef(u0, u1)[0, 1]) < 0.02


def test_counts_follow_the_paper_realisation():
    assert gi.counts(sum(gi.PAPER_COUNTS)) == (gi.PAPER_COUNTS[2], gi.PAPER_COUNTS[1], gi.PAPER_COUNTS[0])
    for n in (1 << 14, 1 << 23, 1 << 28):
        h, d, b = gi.counts(n)
        assert h + d + b == n and b < d < h


def _hernquist_only(a=0.01):
    return gi.Galaxy(0, 0, 1000, G=1.0, M_halo=0.0, M_disk=0.0, M_bulge=1.0, a_bulge=a,
                     r_t=1e6, dr_t=1.0)


def test_hernquist_potential_and_df_closed_forms():
    """A lone Hernquist sphere (G = M = 1, a = 0.01; no taper on the grid):
    Psi = GM/(r + a), and f(E) of Hernquist (1990) Eq. 17."""
    a = 0.01
    tb = gi.tables(_hernquist_only(a))
    pr = tb["prof"]
    r, Psi = pr["r"], pr["Psi"]
    # the grid ends at 600: the sphere inside it carries all the mass (x 1.0000333)
    assert np.max(np.abs(Psi * (r + a) - 1.0)) < 5e-5
    q2 = Psi * a
    q = np.sqrt(q2)
    vg = math.sqrt(1.0 / a)
    fcf = (1.0 / (8 * math.sqrt(2) * math.pi ** 3 * a ** 3 * vg ** 3) / (1 - q2) ** 2.5
           * (3 * np.arcsin(q) + q * np.sqrt(1 - q2) * (1 - 2 * q2) * (8 * q2 * q2 - 8 * q2 - 3)))
    f = tb["bulge"]["f"]
    mid = (q2 > 0.02) & (q2 < 0.8)
    assert np.max(np.abs(f[mid] / fcf[mid] - 1)) < 5e-4
    deep = (q2 >= 0.8) & (q2 < 0.99)
    assert np.max(np.abs(f[deep] / fcf[deep] - 1)) < 1.5e-2


def test_nfw_enclosed_mass():
    """An untapered NFW halo: M(<r) proportional to ln(1 + x) - x/(1 + x)."""
    g = gi.Galaxy(1000, 0, 0, G=1.0, M_halo=1.0, a_halo=15.0, M_bulge=0.0, M_disk=0.0,
                  r_t=1e6, dr_t=1.0)
    pr = gi.profiles(g)
    r = pr["r"]
    x = r / 15.0
    m = np.log1p(x) - x / (1 + x)
    ref = np.searchsorted(r, 10.0)
    got = pr["comp"]["halo"]["M"] / pr["comp"]["halo"]["M"][ref]
    sel = r < 300
    # trapezoid rule in ln r, step 0.0038: error of order step^2 / 12
    assert np.max(np.abs(got[sel] / (m[sel] / m[ref]) - 1)) < 5e-6


@pytest.fixture(scope="module")
def sec4():
    g = gi.milky_way_sec4(1 << 17)
    return g, gi.tables(g)


def test_df_gives_back_the_density(sec4):
    """4 pi int v^2 f(Psi - v^2/2) dv = rho for both spheroids, inside the taper."""
    _, tb = sec4
    pr = tb["prof"]
    r, Psi = pr["r"], pr["Psi"]
    for name in ("halo", "bulge"):
        rho = pr["comp"][name]["rho"]
        rec = 4 * math.pi * (2 * (Psi - Psi[-1])) ** 1.5 * tb[name]["vnorm"]
        sel = (r > 1e-3) & (r < 200)
        assert np.max(np.abs(rec[sel] / rho[sel] - 1)) < 2e-4, name
        assert np.all(tb[name]["f"] >= 0)


def test_df_dispersion_solves_the_jeans_equation(sec4):
    """<v^2>/3 of the distribution function equals the isotropic Jeans
    dispersion (1/rho) int_r rho G M / r'^2 dr' of each spheroid."""
    g, tb = sec4
    pr = tb["prof"]
    r, Psi, Mt = pr["r"], pr["Psi"], pr["Mt"]
    q = np.linspace(0, 1, 4001)
    for name in ("halo", "bulge"):
        rho = pr["comp"][name]["rho"]
        integrand = rho * g.G * Mt / r ** 2 * r  # d ln r
        tail = np.concatenate([np.cumsum((0.5 * (integrand[1:] + integrand[:-1]) * pr["dl"])[::-1])[::-1], [0]])
        s2_jeans = tail / rho
        for k in np.searchsorted(r, [0.01, 0.1, 1.0, 10.0, 50.0, 150.0]):
            w = Psi[k] - Psi[-1]
            fv = gi.interp_desc(Psi[-1] + (1 - q * q) * w, Psi, tb[name]["f"])
            m2 = np.trapezoid(q ** 2 * fv, q)
            m4 = np.trapezoid(q ** 4 * fv, q)
            s2_df = 2 * w * m4 / m2 / 3
            assert abs(s2_df / s2_jeans[k] - 1) < 2e-3, (name, r[k], s2_df, s2_jeans[k])


def test_sampled_spheroids_follow_the_tables(sec4):
    g, tb = sec4
    pos, vel, _ = gi.generate(g, tb)
    pr = tb["prof"]
    Psi = pr["Psi"]
    for name, (s, n) in (("halo", (0, g.n_halo)), ("bulge", (g.n_halo + g.n_disk, g.n_bulge))):
        # sampled before the centre-of-mass shift: redo the draw for the raw radii
        comp_id = 0 if name == "halo" else 2
        p, v = gi.sample_spheroid(g, tb, name, s, n, comp_id)
        r = np.sqrt((p * p).sum(0))
        sp = np.sqrt((v * v).sum(0))
        rr = np.sort(r)
        P = pr["comp"][name]["P"]
        for x in np.quantile(r, [0.05, 0.25, 0.5, 0.75, 0.95]):
            emp = np.searchsorted(rr, x) / n
            assert abs(emp - np.interp(math.log(x), np.log(pr["r"]), P)) < 2.0 / math.sqrt(n)
        vesc = np.sqrt(2 * (np.interp(np.log(r), np.log(pr["r"]), Psi) - Psi[-1]))
        assert np.all(sp <= vesc * (1 + 1e-12))
        # isotropy: each axis carries a third of <v^2>; directions uniform
        m2 = (v * v).mean(1)
        assert np.max(np.abs(m2 / m2.mean() - 1)) < 6 / math.sqrt(n)
        assert np.max(np.abs(p.mean(1))) < 6 * r.std() / math.sqrt(n) + 1e-9


def test_generate_centres_and_is_deterministic(sec4):
    g, tb = sec4
    pos, vel, mass = gi.generate(g, tb)
    mt = mass.sum()
    assert np.max(np.abs((pos * mass).sum(1) / mt)) < 1e-12 * np.abs(pos).max()
    assert np.max(np.abs((vel * mass).sum(1) / mt)) < 1e-12 * np.abs(vel).max()
    assert math.isclose(mt, g.M_halo + g.M_disk + g.M_bulge, rel_tol=1e-12)
    p2, v2, _ = gi.generate(g, tb)
    assert np.array_equal(pos, p2) and np.array_equal(vel, v2)
    g3 = gi.milky_way_sec4(1 << 17, seed=g.seed + 1)
    p3, _, _ = gi.generate(g3, tb)
    assert not np.array_equal(pos, p3)


def test_sampled_halo_is_virialised():
    """A lone tapered NFW halo from its distribution function: 2K/|W| = 1
    within the sampling noise (W by direct summation)."""
    g = gi.Galaxy(6000, 0, 0, seed=7, M_bulge=0.0, M_disk=0.0)
    pos, vel, mass = gi.generate(g)
    _, pot = oracle.direct_forces(pos, mass, 0.05, g.G)
    W = 0.5 * float((mass * pot).sum())
    Kin = 0.5 * float((mass * (vel * vel).sum(0)).sum())
    assert abs(2 * Kin / abs(W) - 1) < 0.05


def test_disk_positions_follow_exponential_and_sech2(sec4):
    g, tb = sec4
    p, _ = gi.sample_disk(g, tb, g.n_halo, g.n_disk)
    n = g.n_disk
    R = np.sqrt(p[0] ** 2 + p[1] ** 2)
    assert R.max() <= g.R_max * (1 + 1e-12)
    norm = 1 - (1 + g.R_max / g.R_d) * math.exp(-g.R_max / g.R_d)
    for x in (1.0, 2.5, 5.0, 10.0):
        want = (1 - (1 + x / g.R_d) * math.exp(-x / g.R_d)) / norm
        assert abs((R < x).mean() - want) < 2.5 / math.sqrt(n)
    for x in (0.1, 0.3, 0.9):
        assert abs((np.abs(p[2]) < x).mean() - math.tanh(x / g.z0)) < 2.5 / math.sqrt(n)


def test_disk_fraction_series_and_closed_form_agree():
    """1 - (1 + x) e^-x: the series branch against the closed form where the
    latter is accurate, and against its first five Taylor terms for small x."""
    x = np.linspace(0.3, 0.5, 51)
    direct = 1.0 - (1.0 + x) * np.exp(-x)
    below = x < 0.5
    assert np.max(np.abs(gi.disk_fraction(x)[below] / direct[below] - 1)) < 1e-14
    t = np.array([1e-8, 1e-5, 1e-3])
    taylor = t * t / 2 - t ** 3 / 3 + t ** 4 / 8 - t ** 5 / 30 + t ** 6 / 144
    assert np.max(np.abs(gi.disk_fraction(t) / taylor - 1)) < 1e-14


def test_freeman_rotation_limits():
    """Thin exponential disk: Keplerian far out; maximum near 2.15 R_d."""
    G, M, Rd = 1.0, 1.0, 1.0
    R = np.array([200.0])
    assert abs(gi.freeman_vc2(R, G, M, Rd)[0] * R[0] / (G * M) - 1) < 2e-4
    Rg = np.linspace(0.5, 5, 9001)
    Rpk = Rg[np.argmax(gi.freeman_vc2(Rg, G, M, Rd))]
    assert abs(Rpk - 2.15) < 0.01


def test_vertical_factor_closed_forms():
    """I(kappa) = int_0^inf sech^2(t) e^{-kappa t} dt: 1, pi/2 - 1,
    2 ln 2 - 1 and 3 - 4 ln 2 at kappa = 0, 1, 2, 4 (from sech^2 t = 4
    sum_n (-1)^(n+1) n e^{-2nt}, summed in the Abel sense); kappa = 4 is
    near the top of the range the disk uses (40 z0 / R_d = 4.8)."""
    I = gi.vertical_factor(np.array([0.0, 1.0, 2.0, 4.0]))
    assert abs(I[0] - 1) < 1e-12
    assert abs(I[1] - (math.pi / 2 - 1)) < 1e-8
    assert abs(I[2] - (2 * math.log(2) - 1)) < 1e-8
    assert abs(I[3] - (3 - 4 * math.log(2))) < 1e-8


def test_disk_spherical_mass_against_cylindrical_integral(sec4):
    """M(<r) of the sech^2 disk from its shell rate (Simpson in the polar
    angle, trapezoid in ln r) equals the independent integral over
    cylinders, int_0^min(r, R_max) 2 pi R Sigma(R) tanh(sqrt(r^2 - R^2)/z0)
    dR (a sech^2 column holds tanh(h/z0) of its mass within |z| < h); the
    total is M_disk; far inside z0 it is the central density times the
    volume; in the thin limit it is the thin disk's 1 - (1 + x) e^-x."""
    from scipy import integrate
    g, _ = sec4
    r, dl = gi.radial_grid()
    M, dM = gi.disk_sph_mass(r, dl, g)
    sig0 = gi.disk_sigma0(g)
    for rr in (0.05, 0.3, 1.0, 3.0, 10.0, 29.0, 40.0):
        k = int(np.argmin(np.abs(r - rr)))
        rk = r[k]
        cyl = integrate.quad(lambda R: 2 * math.pi * R * sig0 * math.exp(-R / g.R_d)
                             * math.tanh(math.sqrt(max(rk * rk - R * R, 0.0)) / g.z0),
                             0.0, min(rk, g.R_max), limit=400, epsabs=0, epsrel=1e-11)[0]
        assert abs(M[k] / cyl - 1) < 2e-5, (rr, M[k], cyl)
    assert abs(M[-1] / g.M_disk - 1) < 1e-5
    k = int(np.argmin(np.abs(r - 1e-3)))
    # to first order in r / R_d (the radial fall-off of Sigma inside the sphere)
    assert abs(M[k] / (4 / 3 * math.pi * r[k] ** 3 * sig0 / (2 * g.z0)) - 1) < 2 * r[k] / g.R_d
    import dataclasses
    thin = dataclasses.replace(g, z0=1e-4)
    Mt, _ = gi.disk_sph_mass(r, dl, thin)
    sel = (r > 0.5) & (r < 25)
    want = g.M_disk * gi.disk_fraction(r[sel] / g.R_d) / gi.disk_fraction(g.R_max / g.R_d)
    assert np.max(np.abs(Mt[sel] / want - 1)) < 2e-3


def test_thick_disk_rotation_limits(sec4):
    """The sech^2 disk's midplane circular speed tends to Freeman's thin-disk
    curve as z0 -> 0 (within the k range's truncation), lies below it for
    z0 = 0.3 kpc by an amount that shrinks outwards, and is Keplerian far
    out."""
    import dataclasses
    g, _ = sec4
    R = np.array([1.0, 2.0, 4.0, 8.0, 16.0])
    fr = gi.freeman_vc2(R, g.G, g.M_disk, g.R_d)
    thin = dataclasses.replace(g, z0=1e-7)
    assert np.max(np.abs(gi.disk_vc2(R, thin) / fr - 1)) < 2e-3
    ratio = gi.disk_vc2(R, g) / fr
    assert np.all(ratio < 1) and np.all(np.diff(ratio) > 0) and ratio[-1] > 0.99
    far = np.array([60.0 * g.R_d])
    assert abs(gi.disk_vc2(far, g)[0] * far[0] / (g.G * g.M_disk) - 1) < 2e-3


def test_disk_kinematic_tables(sec4):
    """Toomre's Q equals the set value at R_Q; sigma_R^2 follows Sigma; the
    epicyclic ratio holds; the drift slope -2R/R_d used for the mean
    rotation equals the numerical d ln(Sigma sigma_R^2)/d ln R of the
    tables; the mean rotation never exceeds v_c and lags it where the
    drift term is negative."""
    g, tb = sec4
    d = tb["disk"]
    R = d["R"]
    s0 = g.M_disk / (2 * math.pi * g.R_d ** 2)
    Sig = s0 * np.exp(-R / g.R_d)
    Q = d["sR"] * d["kappa"] / (3.36 * g.G * Sig)
    iq = np.argmin(np.abs(R - g.R_Q))
    assert abs(Q[iq] / g.Q - 1) < 1e-3
    assert np.allclose(d["sR"] ** 2 / Sig, (d["sR"] ** 2 / Sig)[0], rtol=1e-12)
    om2 = d["vc2"] / R ** 2
    assert np.allclose(d["sphi"] / d["sR"], d["kappa"] / (2 * np.sqrt(om2)), rtol=1e-12)
    num = np.gradient(np.log(Sig * d["sR"] ** 2), np.log(R))
    sel = (R > 0.5) & (R < 25)
    assert np.max(np.abs(num[sel] + 2 * R[sel] / g.R_d)) < 5e-5  # 2nd-order differences
    assert np.all(d["vphi"] ** 2 <= d["vc2"] * (1 + 1e-15))
    drift = 1 - d["kappa"] ** 2 / (4 * om2) - 2 * R / g.R_d
    lag = drift < -1e-3
    assert lag[R > 2].all()
    assert np.all(d["vphi"][lag] ** 2 < d["vc2"][lag])
    # the sample's moments per radial bin follow the tables
    p, v = gi.sample_disk(g, tb, g.n_halo, g.n_disk)
    Rp = np.sqrt(p[0] ** 2 + p[1] ** 2)
    c, s = p[0] / Rp, p[1] / Rp
    vR = v[0] * c + v[1] * s
    vp = -v[0] * s + v[1] * c
    for lo, hi in ((2.0, 3.0), (4.0, 6.0)):
        m = (Rp > lo) & (Rp < hi)
        k = m.sum()
        mid = np.interp(Rp[m], R, d["vphi"]).mean()
        sRm = math.sqrt(np.mean(np.interp(Rp[m], R, d["sR"]) ** 2))
        assert abs(vp[m].mean() - mid) < 4 * d["sphi"].max() / math.sqrt(k)
        assert abs(vR[m].std() / sRm - 1) < 4 / math.sqrt(2 * k)
