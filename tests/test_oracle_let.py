"""Pins of the oracle's domain decomposition and local essential trees
(Sec. III.B): domains are equal pieces of the global Peano-Hilbert order
whose trees, built in the global cube, carry exactly the global keys; the
cells marked for a remote domain are closed under parents and include every
child of an opened cell; and the force assembled from the own tree plus the
other domains' trees equals direct summation as theta -> 0 and follows the
single global tree at theta = 0.4; and the marks equal, cell for cell, the
union of the cells reached by every destination group's walk, recomputed
here in plain Python from the definition."""
import numpy as np
import pytest

import oracle
import workloads


def _domains(m, R):
    g = oracle.Tree(m.pos, m.mass)
    key, perm = g.keys()
    cube = g.cube()
    cuts = [m.n * r // R for r in range(R + 1)]
    idx = [perm[cuts[r]:cuts[r + 1]] for r in range(R)]
    trees = [oracle.Tree(m.pos[:, i], m.mass[i], cube=cube) for i in idx]
    return g, key, idx, trees


def test_domain_trees_are_branches_of_the_global_octree():
    m = workloads.plummer(6000, seed=21)
    g, key, idx, trees = _domains(m, 5)
    n0 = 0
    for t, i in zip(trees, idx):
        k, p = t.keys()
        assert t.cube()[1] == g.cube()[1] and np.array_equal(t.cube()[0], g.cube()[0])
        # the domain's keys are the global keys of its particles, in the same order
        assert np.array_equal(k, key[n0:n0 + t.n])
        assert np.array_equal(i[p], i)  # the piece is already in key order
        n0 += t.n


def test_let_marks_are_closed_under_parents_and_children():
    m = workloads.milky_way(8000, seed=5)
    _, _, _, trees = _domains(m, 4)
    src, dst = trees[1], trees[2]
    v, o = src.let_mark(dst, 0.4)
    nd = src.nodes()
    assert v[0] and o[0]          # the root is always opened by a remote domain
    assert np.all(v[o])           # opened cells were visited
    parent = np.zeros(src.nnodes, np.int64)
    for c in range(src.nnodes):
        for k in range(nd["nchild"][c]):
            parent[nd["child"][c] + k] = c
    vis = np.nonzero(v)[0]
    assert np.all(o[parent[vis[vis > 0]]])  # a visited cell's parent was opened
    for c in np.nonzero(o)[0]:
        ch = nd["child"][c] + np.arange(nd["nchild"][c])
        assert np.all(v[ch])                # every child of an opened cell is visited
    # fewer cells than the whole tree: a remote domain needs only part of it
    assert v.sum() < src.nnodes


def _assembled(m, trees, idx, theta, eps, G=1.0):
    acc = np.zeros((3, m.n))
    pot = np.zeros(m.n)
    for i, ti in enumerate(trees):
        a, p, _ = ti.forces(theta, eps, G)
        for j, tj in enumerate(trees):
            if j != i:
                a2, p2, _, _, _ = tj.cross_forces(ti, theta, eps, G)
                a, p = a + a2, p + p2
        acc[:, idx[i]] = a
        pot[idx[i]] = p
    return acc, pot


def test_assembled_forces_tend_to_direct_summation():
    m = workloads.plummer(3000, seed=8)
    _, _, idx, trees = _domains(m, 3)
    acc, pot = _assembled(m, trees, idx, 1e-4, 0.01)
    ad, pdir = oracle.direct_forces(m.pos, m.mass, 0.01, 1.0)
    e = np.linalg.norm(acc - ad, axis=0) / np.linalg.norm(ad, axis=0)
    assert e.max() < 1e-12 and np.max(np.abs(pot - pdir) / np.abs(pdir)) < 1e-12


@pytest.mark.parametrize("R", [2, 7])
def test_assembled_forces_follow_the_global_tree(R):
    m = workloads.milky_way(20000, seed=12)
    g, _, idx, trees = _domains(m, R)
    acc, _ = _assembled(m, trees, idx, 0.4, 0.01, m.G)
    ag, _, _ = g.forces(0.4, 0.01, m.G)
    ad, _ = oracle.direct_forces(m.pos, m.mass, 0.01, m.G, targets=np.arange(0, m.n, 7))
    e_dom = np.linalg.norm(acc[:, ::7] - ad, axis=0) / np.linalg.norm(ad, axis=0)
    e_glob = np.linalg.norm(ag[:, ::7] - ad, axis=0) / np.linalg.norm(ad, axis=0)
    # the decomposition approximates direct summation as well as one tree does
    assert np.median(e_dom) < 2.0 * np.median(e_glob) and np.median(e_dom) < 1e-3


def _walk_visits(src, dst, theta):
    """The definition of a local essential tree, walked in plain Python: the
    cells of src reached by the breadth-first walk of each of dst's groups
    (the opening test in FP32, each operation rounded, on the FP32 cell and
    group-box inputs), and those among them that the test opens."""
    com_f, r2 = src.cell_mac(theta)
    gc, gh = dst.group_box_f32()
    nd = src.nodes()
    zero = np.float32(0.0)
    v = np.zeros(src.nnodes, bool)
    o = np.zeros(src.nnodes, bool)
    for g in range(dst.ngroups):
        frontier = [0]
        while frontier:
            nxt = []
            for c in frontier:
                v[c] = True
                a = [max(np.abs(com_f[d, c] - gc[d, g]) - gh[d, g], zero) for d in range(3)]
                d2 = (a[0] * a[0] + a[1] * a[1]) + a[2] * a[2]
                if d2 < r2[c]:
                    o[c] = True
                    first, k = int(nd["child"][c]), int(nd["nchild"][c])
                    nxt.extend(range(first, first + k))
            frontier = nxt
    return v, o


@pytest.mark.parametrize("pair", [(3, 0), (0, 1)])
def test_let_marks_equal_the_union_of_the_group_walks(pair):
    m = workloads.milky_way(20000, seed=41)
    _, _, _, trees = _domains(m, 4)
    src, dst = trees[pair[0]], trees[pair[1]]
    v, o = src.let_mark(dst, 0.4)
    vw, ow = _walk_visits(src, dst, 0.4)
    assert np.array_equal(v, vw) and np.array_equal(o, ow)
    if pair == (3, 0):  # distant domains: only part of the tree is sent
        assert v.sum() < 0.8 * src.nnodes
