"""Pins for the oracle's force evaluation: Eq. 1-2 (Sec. VI.A) for one
source, direct summation (Sec. I.A) against closed forms and Newton's third
law, and the tree method against direct summation."""
import math

import numpy as np
import pytest

import workloads


# ---------------------------------------------------------------- Eq. 1-2 ---

def test_point_mass_newton_by_hand(orc):
    # unit mass at r = (3, 4, 0) from the target: |r| = 5
    phi, a = orc.eval_source([3.0, 4.0, 0.0], 2.0, None, eps=0.0, G=1.5)
    assert phi == pytest.approx(-1.5 * 2.0 / 5.0, rel=1e-15)
    assert np.allclose(a, 1.5 * 2.0 * np.array([3.0, 4.0, 0.0]) / 125.0, rtol=1e-15)
    # Plummer softening replaces |r| by sqrt(r^2 + eps^2)
    phi, a = orc.eval_source([3.0, 4.0, 0.0], 1.0, None, eps=12.0)
    assert phi == pytest.approx(-1.0 / 13.0, rel=1e-15)
    assert np.allclose(a, np.array([3.0, 4.0, 0.0]) / 13.0 ** 3, rtol=1e-15)


@pytest.mark.parametrize("eps", [0.0, 0.3])
def test_cell_acceleration_is_gradient_of_potential(orc, eps):
    """Eq. 2 must be the gradient of Eq. 1 with respect to r (a = -grad_x_i phi
    and r = r_j - r_i); checked by central differences with a full Q."""
    Q = np.array([0.7, 0.2, 0.4, 0.15, -0.25, 0.05])
    r0 = np.array([1.3, -0.8, 2.1])
    _, a = orc.eval_source(r0, 1.7, Q, eps=eps)
    h = 1e-5
    g = np.zeros(3)
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        pp, _ = orc.eval_source(r0 + e, 1.7, Q, eps=eps)
        pm, _ = orc.eval_source(r0 - e, 1.7, Q, eps=eps)
        g[d] = (pp - pm) / (2 * h)
    assert np.allclose(a, g, rtol=1e-8, atol=1e-10)


def _cluster_error(orc, members, mvec, D, direction):
    """Relative acceleration error of the cell (M, com, Q) expansion of the
    members, seen from a target at distance D from the com."""
    t = orc.Tree(members, mvec)          # <= 16 particles: the root is a leaf
    mp = t.multipoles()
    M, com, Q = mp["M"][0], mp["com"][:, 0], mp["Q"][:, 0]
    target = com + D * direction
    _, a_cell = orc.eval_source(com - target, M, Q)
    acc, _ = orc.direct_forces(np.concatenate([members, target[:, None]], 1),
                               np.concatenate([mvec, [0.0]]), eps=0.0, targets=[members.shape[1]])
    return np.linalg.norm(a_cell - acc[:, 0]) / np.linalg.norm(acc[:, 0])


def test_quadrupole_error_falls_as_third_power(orc):
    """Monopole + non-traceless quadrupole about the com leaves an octupole
    error ~ (l/D)^3; a dropped or mis-signed quadrupole term leaves (l/D)^2."""
    rng = np.random.default_rng(2)
    members = rng.uniform(-0.5, 0.5, (3, 12))
    mvec = rng.uniform(0.5, 1.5, 12)
    u = np.array([0.48, -0.6, 0.64])
    Ds = np.array([8.0, 16.0, 32.0, 64.0])
    err = [_cluster_error(orc, members, mvec, D, u) for D in Ds]
    slope = np.polyfit(np.log(Ds), np.log(err), 1)[0]
    assert -3.3 < slope < -2.7, (slope, err)


def test_symmetric_cluster_error_falls_as_fourth_power(orc):
    """For +-d pairs of equal mass the octupole vanishes: error ~ (l/D)^4."""
    rng = np.random.default_rng(4)
    half = rng.uniform(-0.5, 0.5, (3, 6))
    members = np.concatenate([half, -half], 1)
    mvec = np.concatenate([np.full(6, 1.0), np.full(6, 1.0)])
    u = np.array([0.0, 0.6, 0.8])
    Ds = np.array([8.0, 16.0, 32.0, 64.0])
    err = [_cluster_error(orc, members, mvec, D, u) for D in Ds]
    slope = np.polyfit(np.log(Ds), np.log(err), 1)[0]
    assert -4.3 < slope < -3.7, (slope, err)


# ---------------------------------------------------------- O1: direct sum ---

def test_two_body_and_triangle_by_hand(orc):
    pos = np.array([[0.0, 2.0], [0.0, 0.0], [0.0, 0.0]])
    acc, pot = orc.direct_forces(pos, np.array([3.0, 5.0]), eps=0.0, G=2.0)
    assert np.allclose(acc[:, 0], [2.0 * 5.0 / 4.0, 0, 0], rtol=1e-15)
    assert np.allclose(acc[:, 1], [-2.0 * 3.0 / 4.0, 0, 0], rtol=1e-15)
    assert np.allclose(pot, [-2.0 * 5.0 / 2.0, -2.0 * 3.0 / 2.0], rtol=1e-15)
    # equilateral triangle of side s, unit masses: |a| = sqrt(3)/s^2 toward the centre
    s = 1.7
    ang = np.array([90.0, 210.0, 330.0]) * math.pi / 180
    R = s / math.sqrt(3)
    pos = np.stack([R * np.cos(ang), R * np.sin(ang), np.zeros(3)])
    acc, pot = orc.direct_forces(pos, np.ones(3), eps=0.0)
    for i in range(3):
        assert np.allclose(acc[:, i], -math.sqrt(3) / s ** 2 * pos[:, i] / R, rtol=1e-14, atol=1e-15)
    assert np.allclose(pot, -2.0 / s, rtol=1e-15)


def test_newton_third_law(orc):
    rng = np.random.default_rng(8)
    pos = rng.standard_normal((3, 800))
    m = rng.uniform(0.1, 2.0, 800)
    acc, _ = orc.direct_forces(pos, m, eps=0.05)
    net = np.linalg.norm((acc * m).sum(1))
    assert net <= 1e-13 * (m * np.linalg.norm(acc, axis=0)).sum()


def test_plummer_closed_forms(orc):
    """G = M = a = 1: phi(r) = -1/sqrt(r^2+1), |a|(r) = r/(r^2+1)^{3/2},
    W = -3 pi / 32; the sample is in virial equilibrium (2K/|W| = 1)."""
    n = 1 << 14
    mdl = workloads.plummer(n, seed=1001)
    acc, pot = orc.direct_forces(mdl.pos, mdl.mass, eps=0.01)
    r = np.linalg.norm(mdl.pos, axis=0)
    edges = np.quantile(r, np.linspace(0.02, 0.9, 12))
    for lo_, hi_ in zip(edges[:-1], edges[1:]):
        sel = (r >= lo_) & (r < hi_)
        rr = r[sel]
        phi_cf = -1.0 / np.sqrt(rr * rr + 1.0)
        a_cf = rr / (rr * rr + 1.0) ** 1.5
        tol = 4.0 / math.sqrt(sel.sum()) + 2e-3
        assert abs(pot[sel].mean() / phi_cf.mean() - 1) < tol
        assert abs(np.linalg.norm(acc[:, sel], axis=0).mean() / a_cf.mean() - 1) < 3 * tol
    W = 0.5 * (mdl.mass * pot).sum()
    assert abs(W / (-3 * math.pi / 32) - 1) < 4.0 / math.sqrt(n)
    K = 0.5 * (mdl.mass * (mdl.vel ** 2).sum(0)).sum()
    assert abs(2 * K / abs(W) - 1) < 4.0 / math.sqrt(n)


# ----------------------------------------------------- O2: tree vs direct ---

def test_tree_equals_direct_when_every_cell_opens(orc):
    mdl = workloads.plummer(3000, seed=21)
    acc_d, pot_d = orc.direct_forces(mdl.pos, mdl.mass, eps=0.01)
    t = orc.Tree(mdl.pos, mdl.mass)
    acc_t, pot_t, (npp, npc) = t.forces(1e-4, 0.01)
    assert npc == 0 and npp == 3000 * 3000          # every pair, self pair included
    scale = np.linalg.norm(acc_d, axis=0)
    assert np.all(np.linalg.norm(acc_t - acc_d, axis=0) <= 1e-13 * scale)
    assert np.all(np.abs(pot_t - pot_d) <= 1e-13 * np.abs(pot_d))


def test_tree_is_direct_for_a_single_leaf(orc):
    rng = np.random.default_rng(13)
    pos = rng.standard_normal((3, 16))
    m = rng.uniform(0.5, 1.5, 16)
    t = orc.Tree(pos, m)
    assert t.nnodes == 1
    acc_t, pot_t, (npp, npc) = t.forces(0.4, 0.02, G=3.0)
    acc_d, pot_d = orc.direct_forces(pos, m, eps=0.02, G=3.0)
    assert (npp, npc) == (256, 0)
    assert np.allclose(acc_t, acc_d, rtol=1e-14, atol=0)
    assert np.allclose(pot_t, pot_d, rtol=1e-14, atol=0)


def test_tree_error_shrinks_with_theta(orc):
    mdl = workloads.plummer(6000, seed=33)
    acc_d, _ = orc.direct_forces(mdl.pos, mdl.mass, eps=0.01)
    t = orc.Tree(mdl.pos, mdl.mass)
    med = []
    npc = []
    for th in (0.8, 0.4, 0.2):
        acc_t, _, counts = t.forces(th, 0.01)
        e = np.linalg.norm(acc_t - acc_d, axis=0) / np.linalg.norm(acc_d, axis=0)
        med.append(np.median(e))
        npc.append(counts[1])
    assert med[0] > med[1] > med[2]
    assert med[1] < 1e-3                     # theta = 0.4 with quadrupoles is well below 0.1 %


def test_interaction_counts_are_consistent(orc):
    mdl = workloads.plummer(5000, seed=44)
    t = orc.Tree(mdl.pos, mdl.mass)
    _, _, g_npp, g_npc, (npp, npc) = t.forces_sorted(0.4, 0.01)
    g = t.groups()
    assert npp == int((g["count"].astype(np.int64) * g_npp).sum())
    assert npc == int((g["count"].astype(np.int64) * g_npc).sum())
    assert np.all(g_npp >= g["count"])      # a group's own particles are p-p sources
    # the accepted cells and opened leaves of a group partition the particles:
    # every particle is covered exactly once (no cell dropped or doubled)
    nd = t.nodes()
    for gi in range(0, t.ngroups, max(1, t.ngroups // 25)):
        pc, leaves = t.group_lists(0.4, gi)
        assert len(pc) == g_npc[gi] and nd["count"][leaves].sum() == g_npp[gi]
        cover = np.zeros(5000, np.int64)
        for c in np.concatenate([pc, leaves]):
            cover[nd["first"][c]:nd["first"][c] + nd["count"][c]] += 1
        assert np.all(cover == 1)
        # the group's own particles sit in opened leaves
        own = slice(int(g["first"][gi]), int(g["first"][gi] + g["count"][gi]))
        in_leaf = np.zeros(5000, bool)
        for c in leaves:
            in_leaf[nd["first"][c]:nd["first"][c] + nd["count"][c]] = True
        assert in_leaf[own].all()


def test_all_particles_at_one_point(orc):
    """Degenerate input: n coincident particles.  The cube falls back to
    L = 1, all keys are equal, the one max-depth leaf is cut into groups of
    64; every pair has r = 0, so a = 0 exactly and phi = -G (n - 1) m / eps."""
    n, m, eps, G = 200, 0.5, 0.02, 2.0
    pos = np.tile(np.array([[0.3], [-1.2], [4.0]]), (1, n))
    t = orc.Tree(pos, np.full(n, m))
    assert t.cube()[1] == 1.0
    acc, pot, (npp, npc) = t.forces(0.4, eps, G)
    assert np.all(acc == 0.0)
    assert np.allclose(pot, -G * (n - 1) * m / eps, rtol=1e-14)
    assert (npp, npc) == (n * n, 0)


def test_group_lists_follow_the_opening_test(orc):
    """Each group's lists, recomputed from the definition in plain Python: a
    breadth-first walk from the root that accepts a cell when the FP32
    opening test (each operation rounded) fails and otherwise opens it,
    descending into an internal cell and taking an opened leaf's particles;
    the oracle's accepted cells and opened leaves are exactly these sets."""
    mdl = workloads.milky_way(12000, seed=45)
    t = orc.Tree(mdl.pos, mdl.mass)
    com_f, r2 = t.cell_mac(0.4)
    gc, gh = t.group_box_f32()
    nd = t.nodes()
    zero = np.float32(0.0)
    for gi in range(0, t.ngroups, max(1, t.ngroups // 40)):
        acc, opened_leaves, frontier = [], [], [0]
        while frontier:
            nxt = []
            for c in frontier:
                a = [max(np.abs(com_f[d, c] - gc[d, gi]) - gh[d, gi], zero) for d in range(3)]
                if (a[0] * a[0] + a[1] * a[1]) + a[2] * a[2] < r2[c]:
                    if nd["nchild"][c] == 0:
                        opened_leaves.append(c)
                    else:
                        nxt.extend(range(int(nd["child"][c]), int(nd["child"][c] + nd["nchild"][c])))
                else:
                    acc.append(c)
            frontier = nxt
        pc, leaves = t.group_lists(0.4, gi)
        assert sorted(pc.tolist()) == sorted(acc)
        assert sorted(leaves.tolist()) == sorted(opened_leaves)
