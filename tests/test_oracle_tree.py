"""Pins for the oracle's octree, groups and multipoles (Sec. I.A: octants
split until a node holds at most 16 particles; Sec. VI.A: mass, position and
3x3 symmetric quadrupole of each cell).  The octree is compared with an
independent recursive geometric octree; multipoles with direct per-node
sums."""
import numpy as np
import pytest

import workloads


def _quantise(pos, lo, L):
    scale = 2.0 ** 21 / L
    q = np.floor((pos - lo[:, None]) * scale)
    return np.clip(q, 0, 2 ** 21 - 1).astype(np.int64)


def _brute_octree(q, nleaf):
    """Recursive geometric octree on integer coordinates: a cube with more
    than nleaf particles (and above the 21st level) is cut into its 8
    octants; empty octants are dropped."""
    out = set()

    def rec(idx, level):
        out.add((level, frozenset(idx.tolist())))
        if idx.size <= nleaf or level >= 21:
            return
        s = 20 - level
        octant = (((q[0, idx] >> s) & 1) << 2) | (((q[1, idx] >> s) & 1) << 1) | ((q[2, idx] >> s) & 1)
        for o in range(8):
            sub = idx[octant == o]
            if sub.size:
                rec(sub, level + 1)

    rec(np.arange(q.shape[1]), 0)
    return out


def _cases():
    rng = np.random.default_rng(5)
    uni = rng.uniform(-1, 1, (3, 700))
    plum = workloads.plummer(1500, seed=9).pos
    clump = np.concatenate([rng.normal(0, 1e-3, (3, 200)), rng.normal(5, 1.0, (3, 300))], axis=1)
    dup = rng.uniform(-1, 1, (3, 400))
    dup[:, 200:300] = dup[:, 3:4]     # 101 coincident particles -> max-depth leaf
    tiny = rng.uniform(-1, 1, (3, 40))
    return {"uniform": uni, "plummer": plum, "clump": clump, "coincident": dup, "tiny": tiny}


@pytest.fixture(scope="module", params=list(_cases().keys()))
def case(request, orc):
    pos = _cases()[request.param]
    n = pos.shape[1]
    mass = np.random.default_rng(1).uniform(0.5, 2.0, n)
    return request.param, pos, mass, orc.Tree(pos, mass)


def test_octree_matches_recursive_brute_force(case):
    name, pos, mass, t = case
    key, perm = t.keys()
    nd = t.nodes()
    lo, L = t.cube()
    got = {(int(nd["level"][i]), frozenset(perm[nd["first"][i]:nd["first"][i] + nd["count"][i]].tolist()))
           for i in range(t.nnodes)}
    assert len(got) == t.nnodes
    assert got == _brute_octree(_quantise(pos, lo, L), 16)


def test_octree_invariants(case):
    name, pos, mass, t = case
    nd = t.nodes()
    key, perm = t.keys()
    n = pos.shape[1]
    assert nd["first"][0] == 0 and nd["count"][0] == n and nd["level"][0] == 0
    assert np.all(np.diff(nd["level"].astype(np.int64)) >= 0)          # breadth-first
    nxt = 1
    for i in range(t.nnodes):
        f, c, ch, nc, lv = (int(nd[k][i]) for k in ("first", "count", "child", "nchild", "level"))
        if nc == 0:
            assert c <= 16 or lv == 21
            if lv == 21:
                assert np.all(key[f:f + c] == key[f])
            continue
        assert c > 16 and lv < 21
        assert ch == nxt                                                  # children numbered in order
        nxt += nc
        kids = range(ch, ch + nc)
        assert int(nd["first"][ch]) == f
        cover = 0
        for k in kids:
            assert nd["level"][k] == lv + 1
            assert nd["first"][k] == f + cover                            # contiguous, key order
            cover += int(nd["count"][k])
            # all members share the level-(lv+1) key prefix
            s = 3 * (21 - (lv + 1))
            seg = key[nd["first"][k]:nd["first"][k] + nd["count"][k]] >> np.uint64(s)
            assert np.all(seg == seg[0])
        assert cover == c
    assert nxt == t.nnodes


def test_groups_tile_and_follow_the_rule(case):
    name, pos, mass, t = case
    g = t.groups()
    nd = t.nodes()
    n = pos.shape[1]
    assert g["first"][0] == 0
    assert np.array_equal(g["first"][1:], (g["first"] + g["count"])[:-1])
    assert int(g["first"][-1] + g["count"][-1]) == n
    assert np.all((g["count"] >= 1) & (g["count"] <= 64))
    # each group is the root (n <= 64), a run of 64 inside a max-depth leaf,
    # or a run of consecutive children of one node with > 64 particles, each
    # child holding <= 64 and the run <= 64 in all; runs are greedy: a run
    # ends at a big child, at the last child, or where the next child would
    # push it past 64
    first, count = nd["first"].astype(np.int64), nd["count"].astype(np.int64)
    child, nchild = nd["child"].astype(np.int64), nd["nchild"].astype(np.int64)
    owner = {}                               # first particle of a small child of a big node
    for i in range(t.nnodes):              # -> (that node, the child's index)
        if count[i] > 64:
            for k in range(nchild[i]):
                if count[child[i] + k] <= 64:
                    owner[int(first[child[i] + k])] = (i, k)
    for f, c in zip(g["first"].tolist(), g["count"].tolist()):
        if c == n and f == 0 and n <= 64:
            continue                          # the root is the one group
        if f in owner:
            p, k0 = owner[f]
            ks, tot, k = [], 0, k0
            while tot < c:                    # the children that make up the run
                ck = count[child[p] + k]
                assert ck <= 64 and first[child[p] + k] == f + tot
                tot += ck
                ks.append(k)
                k += 1
            assert tot == c <= 64
            # greedy: it could not have joined the previous run, and the next
            # child could not join it
            if k0 > 0:
                prev = child[p] + k0 - 1
                if count[prev] <= 64:
                    j = g["first"].tolist().index(f) - 1
                    assert g["count"][j] + count[child[p] + k0] > 64
            if k < nchild[p]:
                assert count[child[p] + k] > 64 or tot + count[child[p] + k] > 64
        else:
            host = [i for i in range(t.nnodes) if nchild[i] == 0 and first[i] <= f
                    and f + c <= first[i] + count[i]]
            assert host and nd["level"][host[0]] == 21 and count[host[0]] > 64
            assert (f - first[host[0]]) % 64 == 0
    # the FP64 box contains every member
    spos, _ = t.sorted_state()
    for k in range(t.ngroups):
        f, c = int(g["first"][k]), int(g["count"][k])
        for d in range(3):
            seg = spos[d, f:f + c]
            tol = 4 * np.spacing(np.abs(seg).max())      # centre/half are rounded once each
            assert g["centre"][d, k] - g["half"][d, k] <= seg.min() + tol
            assert seg.max() <= g["centre"][d, k] + g["half"][d, k] + tol
            assert g["half"][d, k] == 0.5 * (seg.max() - seg.min())


def test_multipoles_match_direct_sums(case):
    name, pos, mass, t = case
    key, perm = t.keys()
    nd = t.nodes()
    mp = t.multipoles()
    lo, L = t.cube()
    for i in range(t.nnodes):
        idx = perm[nd["first"][i]:nd["first"][i] + nd["count"][i]]
        m = mass[idx]
        x = pos[:, idx]
        M = m.sum()
        com = (x * m).sum(1) / M
        d = x - com[:, None]
        Q = np.array([(m * d[0] * d[0]).sum(), (m * d[1] * d[1]).sum(), (m * d[2] * d[2]).sum(),
                      (m * d[0] * d[1]).sum(), (m * d[0] * d[2]).sum(), (m * d[1] * d[2]).sum()])
        side = L / 2 ** int(nd["level"][i])
        assert abs(mp["M"][i] - M) <= 1e-13 * M
        assert np.all(np.abs(mp["com"][:, i] - com) <= 1e-12 * L)
        assert np.all(np.abs(mp["Q"][:, i] - Q) <= 1e-11 * M * side * side + 1e-300)
        # geometric cube of side L/2^level holds every member
        assert mp["side"][i] == side
        assert np.all(np.abs(x - mp["centre"][:, i][:, None]) <= 0.5 * side * (1 + 1e-12))
