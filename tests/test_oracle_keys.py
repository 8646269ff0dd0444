"""Pins for the oracle's bounding cube, Peano-Hilbert keys and sort
(Sec. III.B.1 and Fig. 2: PH keys from the bounding box; Table 2 "Sorting
SFC").  The pins are properties any Hilbert curve must have, checked
exhaustively on small grids, so that a wrong bit, axis or rotation in the
key code fails one of them."""
import itertools

import numpy as np
import pytest


def _all_keys(orc, bits):
    side = 1 << bits
    cells = np.array(list(itertools.product(range(side), repeat=3)), dtype=np.int64)
    keys = np.array([orc.hilbert_key(int(a), int(b), int(c), bits) for a, b, c in cells], dtype=np.int64)
    return cells, keys


@pytest.mark.parametrize("bits", [1, 2, 3, 4])
def test_hilbert_bijection_and_adjacency(orc, bits):
    cells, keys = _all_keys(orc, bits)
    # bijection onto 0 .. 8^bits - 1
    assert np.array_equal(np.sort(keys), np.arange(8 ** bits))
    # consecutive keys are face-adjacent cells (a Hilbert curve has unit steps)
    order = cells[np.argsort(keys)]
    steps = np.abs(np.diff(order, axis=0)).sum(axis=1)
    assert np.all(steps == 1)
    # the curve starts at the origin corner
    assert keys[0] == 0 and np.all(order[0] == 0)


@pytest.mark.parametrize("bits", [2, 3, 4])
def test_hilbert_prefix_property(orc, bits):
    """Each level-l octant is one aligned contiguous key range: the top 3l key
    bits are a function of the top l bits of each coordinate, and distinct
    octants get distinct prefixes."""
    cells, keys = _all_keys(orc, bits)
    for lvl in range(1, bits + 1):
        coarse = cells >> (bits - lvl)
        cid = (coarse[:, 0] << (2 * lvl)) | (coarse[:, 1] << lvl) | coarse[:, 2]
        pref = keys >> (3 * (bits - lvl))
        m = {}
        for c, p in zip(cid.tolist(), pref.tolist()):
            assert m.setdefault(c, p) == p
        assert len(set(m.values())) == len(m) == 8 ** lvl


def test_hilbert_21bit_coarsens_to_small_grids(orc):
    """The 21-bit key's top 3b bits equal the b-bit key of the coarse cell, so
    the exhaustive small-grid pins above carry over to the 21-bit curve."""
    rng = np.random.default_rng(7)
    for _ in range(400):
        q = [int(v) for v in rng.integers(0, 1 << 21, 3)]
        k21 = orc.hilbert_key(*q)
        assert k21 < (1 << 63)
        for b in (1, 2, 3, 4, 7, 11, 20):
            kb = orc.hilbert_key(*[v >> (21 - b) for v in q], bits=b)
            assert kb == k21 >> (3 * (21 - b))


def test_bounding_cube(orc):
    rng = np.random.default_rng(3)
    pos = rng.standard_normal((3, 1000)) * np.array([[1.0], [3.0], [0.5]]) + 10.0
    lo, L = orc.bounding_cube(pos)
    ext = (pos.max(1) - pos.min(1)).max()
    assert L == ext * (1.0 + 2.0 ** -20)
    # the cube is centred on the box and contains every point strictly
    for d in range(3):
        assert lo[d] < pos[d].min() and pos[d].max() < lo[d] + L
        assert abs((lo[d] + 0.5 * L) - 0.5 * (pos[d].min() + pos[d].max())) < 1e-12 * L
    # degenerate: all points coincide -> unit cube around them
    lo1, L1 = orc.bounding_cube(np.ones((3, 5)))
    assert L1 == 1.0 and np.allclose(lo1, 0.5)


def test_sort_is_stable_by_caller_index(orc):
    rng = np.random.default_rng(11)
    pos = rng.uniform(-1, 1, (3, 300))
    pos[:, 100:150] = pos[:, 7:8]          # 51 coincident particles: equal keys
    t = orc.Tree(pos, np.ones(300))
    key, perm = t.keys()
    assert np.array_equal(np.sort(perm), np.arange(300))
    assert np.all(np.diff(key.astype(np.float64)) >= 0)
    # equal keys appear in increasing caller index
    same = key[1:] == key[:-1]
    assert same.sum() >= 50
    assert np.all(perm[1:][same] > perm[:-1][same])
    # keys agree with the per-particle key function on the same quantisation
    lo, L = t.cube()
    scale = 2.0 ** 21 / L
    for s in range(0, 300, 37):
        i = perm[s]
        q = [int(np.clip(np.floor((pos[d, i] - lo[d]) * scale), 0, 2 ** 21 - 1)) for d in range(3)]
        assert orc.hilbert_key(*q) == int(key[s])
