"""Pins for the oracle's opening test (Sec. I.A: a cell is used whole when it
is far enough from the group, by a criterion parameterised by the opening
angle theta).  The reading is r_open = l / theta + |com - geometric centre|
with l the cell's side; the cell is opened when the squared FP32 distance
from its com to the group's box is below r_open^2 (rounded to FP32 once),
and a tie is accepted.

Nothing here reads the oracle's own r_open: the tests build configurations
whose geometry is known exactly (dyadic coordinates, so that every mean,
midpoint and half-width is exact), compute r_open by hand from the cube,
the cell's level and its particles, and check the oracle's accept/open
decision through the interaction lists it produces.  The boundary cases
are placed so that each plausible misreading (no com offset, the parent's
side, a strict inequality at a tie) flips a decision."""
import math

import numpy as np
import pytest

import workloads

F32 = np.float32


def _two_octant_model():
    """65 unit masses in [0, 1]^3: a group B of 49 particles in the low octant
    (a 4 x 4 x 3 grid of spacing 1/32 from the corner (0, 0, 0), and (1/8, 0,
    0)) and a cell C
    of 16 particles in the high octant (the corner (1, 1, 1) and 15 particles
    at (11/16, 11/16, 11/16)).  The root (65 > 64) splits into the two
    octants: B is a group, C a leaf and a group."""
    b = [(i / 32.0, j / 32.0, k / 32.0) for i in range(4) for j in range(4) for k in range(3)]
    b.append((4 / 32.0, 0.0, 0.0))
    assert len(b) == 49
    c = [(1.0, 1.0, 1.0)] + [(11 / 16.0,) * 3] * 15
    pos = np.array(b + c, dtype=np.float64).T.copy()
    return pos, np.ones(pos.shape[1])


def _by_hand(pos):
    """Cube, group box and cell geometry of the two-octant model, from the
    definitions (each value exact in FP64)."""
    ext = 1.0
    L = ext * (1.0 + 2.0 ** -20)
    lo = 0.0 - (L - ext) * 0.5
    side_c = L / 2.0                                  # level 1
    centre_c = lo + 1.5 * side_c                      # high octant, every axis
    com_c = (15 * (11 / 16.0) + 1.0) / 16.0           # every axis
    s_c = math.sqrt(3.0) * abs(com_c - centre_c)
    bmin = pos[:, :49].min(axis=1)
    bmax = pos[:, :49].max(axis=1)
    gc = ((bmin + bmax) * 0.5).astype(F32)
    gh = ((bmax - bmin) * 0.5).astype(F32)           # exact: no rounding up needed
    cf = F32(com_c)
    a = [max(abs(cf - gc[d]) - gh[d], F32(0)) for d in range(3)]
    d2 = (a[0] * a[0] + a[1] * a[1]) + a[2] * a[2]
    assert isinstance(d2, np.float32)
    return side_c, s_c, d2


def _decision(orc, pos, mass, theta):
    """'accept' or 'open' for cell C in group B's walk, from the oracle's lists."""
    t = orc.Tree(pos, mass)
    nd = t.nodes()
    gr = t.groups()
    c_node = [i for i in range(t.nnodes) if nd["level"][i] == 1 and nd["count"][i] == 16]
    b_grp = [g for g in range(t.ngroups) if gr["count"][g] == 49]
    assert len(c_node) == 1 and len(b_grp) == 1
    pc, leaves = t.group_lists(theta, b_grp[0])
    if c_node[0] in pc.tolist():
        assert c_node[0] not in leaves.tolist()
        return "accept"
    assert c_node[0] in leaves.tolist()
    return "open"


def test_the_com_offset_is_part_of_the_opening_radius(orc):
    pos, mass = _two_octant_model()
    side, s, d2 = _by_hand(pos)
    d = math.sqrt(float(d2))
    assert s > 0.07                                   # a large offset by construction
    # d halfway between side/theta and side/theta + s: opened only if s counts
    theta = F32(side / (d - 0.5 * s))
    r_true = side / float(theta) + s
    assert F32(r_true * r_true) > d2 > F32((side / float(theta)) ** 2)
    assert _decision(orc, pos, mass, float(theta)) == "open"


def test_the_cell_side_is_its_own_not_its_parents(orc):
    pos, mass = _two_octant_model()
    side, s, d2 = _by_hand(pos)
    d = math.sqrt(float(d2))
    # d 5 % beyond the cell's radius but inside the parent's (side 2 l)
    theta = F32(side / (d / 1.05 - s))
    r_true = side / float(theta) + s
    r_parent = 2.0 * side / float(theta) + s
    assert F32(r_true * r_true) < d2 < F32(r_parent * r_parent)
    assert _decision(orc, pos, mass, float(theta)) == "accept"


def test_a_tie_is_accepted_and_one_ulp_more_radius_opens(orc):
    """Find the FP32 theta whose r_open^2, rounded to FP32 once, equals the
    FP32 squared distance exactly: that cell is accepted; the next smaller
    theta (a larger radius) opens it."""
    pos, mass = _two_octant_model()
    side, s, d2 = _by_hand(pos)
    theta = F32(side / (math.sqrt(float(d2)) - s))
    tie = None
    for _ in range(4096):
        r = side / float(theta) + s
        r2 = F32(r * r)
        if r2 == d2:
            tie = theta
            break
        theta = np.nextafter(theta, F32(np.inf)) if r2 > d2 else np.nextafter(theta, F32(0))
    assert tie is not None, "no FP32 theta gives an exact tie"
    assert _decision(orc, pos, mass, float(tie)) == "accept"
    below = tie
    while True:                                      # the next theta whose radius exceeds d
        below = np.nextafter(below, F32(0))
        r = side / float(below) + s
        if F32(r * r) > d2:
            break
    assert _decision(orc, pos, mass, float(below)) == "open"


def _hand_mac(t, theta):
    """Every cell's FP32 com and r_open^2, and every group's FP32 box, from
    the particles and the cube alone: com = sum m x / sum m over the cell's
    particles; the cell's cube from its level and the quantised coordinates
    of one of its particles; r_open = l / theta + |com - centre|."""
    lo, L = t.cube()
    x, m = t.sorted_state()
    nd = t.nodes()
    first = nd["first"].astype(np.int64)
    count = nd["count"].astype(np.int64)
    level = nd["level"].astype(np.int64)
    scale = 2.0 ** 21 / L
    q = np.clip(np.floor((x - lo[:, None]) * scale), 0, 2 ** 21 - 1).astype(np.int64)
    cm = np.concatenate([np.zeros(1), np.cumsum(m)])
    cmx = np.concatenate([np.zeros((3, 1)), np.cumsum(m * x, axis=1)], axis=1)
    M = cm[first + count] - cm[first]
    com = (cmx[:, first + count] - cmx[:, first]) / M
    # the prefix sums lose a few ulps against a plain per-cell sum; redo
    # small cells exactly, the rest only matter through one FP32 rounding
    for i in np.nonzero(count <= 64)[0]:
        sl = slice(first[i], first[i] + count[i])
        com[:, i] = (m[sl] * x[:, sl]).sum(axis=1) / m[sl].sum()
    side = L / 2.0 ** level
    cell = q[:, first] >> (21 - level)
    centre = lo[:, None] + (cell + 0.5) * side
    s = np.sqrt(((com - centre) ** 2).sum(axis=0))
    r_open = side / float(theta) + s
    r2 = (r_open * r_open).astype(F32)
    gr = t.groups()
    gf = gr["first"].astype(np.int64)
    gn = gr["count"].astype(np.int64)
    gc = np.zeros((3, t.ngroups), F32)
    gh = np.zeros((3, t.ngroups), F32)
    for g in range(t.ngroups):
        sl = slice(gf[g], gf[g] + gn[g])
        mn, mx = x[:, sl].min(axis=1), x[:, sl].max(axis=1)
        gc[:, g] = ((mn + mx) * 0.5).astype(F32)
        h = (mx - mn) * 0.5
        hf = h.astype(F32)
        gh[:, g] = np.where(hf.astype(np.float64) < h, np.nextafter(hf, F32(np.inf)), hf)
    return com.astype(F32), r2, gc, gh, nd


@pytest.mark.parametrize("theta", [0.4, 0.75, 1.0])
def test_lists_follow_the_hand_computed_opening_radius(orc, theta):
    """On a Milky-Way-like model, each sampled group's accepted cells and
    opened leaves equal a plain-Python breadth-first walk driven by the
    opening radii computed above from the particles alone."""
    mdl = workloads.milky_way(12000, seed=46)
    t = orc.Tree(mdl.pos, mdl.mass)
    com_f, r2, gc, gh, nd = _hand_mac(t, theta)
    zero = F32(0.0)
    for gi in range(0, t.ngroups, max(1, t.ngroups // 30)):
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
        pc, leaves = t.group_lists(theta, gi)
        assert sorted(pc.tolist()) == sorted(acc)
        assert sorted(leaves.tolist()) == sorted(opened_leaves)


def test_accepted_cells_keep_every_target_outside_the_cell(orc):
    """What the criterion is for: with theta <= 1 an accepted cell's com is
    at least r_open >= l + s from every target of the group, while every
    particle of the cell lies within s + sqrt(3) l / 2 < r_open of the com,
    so each target sees the cell's particles from outside their sphere.
    Checked per target with the true FP64 distances."""
    mdl = workloads.plummer(6000, seed=47)
    t = orc.Tree(mdl.pos, mdl.mass)
    x, _ = t.sorted_state()
    com_f, r2, _, _, nd = _hand_mac(t, 1.0)
    lo, L = t.cube()
    gr = t.groups()
    for gi in range(0, t.ngroups, max(1, t.ngroups // 25)):
        pc, _ = t.group_lists(1.0, gi)
        tg = x[:, gr["first"][gi]: gr["first"][gi] + gr["count"][gi]]
        for c in pc:
            cf = com_f[:, c].astype(np.float64)
            r_open = math.sqrt(float(r2[c]))
            dmin = np.sqrt(((tg - cf[:, None]) ** 2).sum(axis=0)).min()
            assert dmin >= r_open * (1 - 1e-6)
            sl = slice(nd["first"][c], nd["first"][c] + nd["count"][c])
            ext = np.sqrt(((x[:, sl] - cf[:, None]) ** 2).sum(axis=0)).max()
            assert ext < r_open
