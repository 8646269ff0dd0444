"""Domains and local essential trees on the GPU against the oracle: domain
trees carry the global keys; the cells of a LET (and what is done with each)
equal the oracle's marks bit for bit; a LET walk gives the oracle's cross
lists per group; forces assembled from own trees and LETs match the
oracle's assembly within the force tolerance and follow direct summation
as well as one global tree; also one pair at the 2^23 size."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _world(m):
    from gpu_helpers import DEV
    from paper_1412_0659_gb300 import TreeGravity
    g = TreeGravity(G=m.G, theta=m.theta, eps=m.eps)
    g.build(torch.from_numpy(m.pos).to(DEV), torch.from_numpy(m.mass).to(DEV))
    g.set_velocities(torch.from_numpy(m.vel).to(DEV))
    return g


def _oracle_domains(m, R):
    t = oracle.Tree(m.pos, m.mass)
    _, perm = t.keys()
    cube = t.cube()
    cuts = [m.n * r // R for r in range(R + 1)]
    idx = [perm[cuts[r]:cuts[r + 1]] for r in range(R)]
    return [oracle.Tree(m.pos[:, i], m.mass[i], cube=cube) for i in idx], idx


def test_domain_trees_carry_the_global_keys():
    from paper_1412_0659_gb300 import domains
    m = workloads.plummer(6000, seed=21)
    w = _world(m)
    doms = domains.split(w, 5)
    gkeys = w.debug()["keys"].cpu().numpy().view(np.uint64)
    n0 = 0
    ots, _ = _oracle_domains(m, 5)
    for (g, ids), ot in zip(doms, ots):
        d = g.debug()
        k = d["keys"].cpu().numpy().view(np.uint64)
        assert np.array_equal(k, gkeys[n0:n0 + g.n])
        nd = ot.nodes()
        for key in ("first", "count", "child", "nchild", "level"):
            assert np.array_equal(d["nodes"][key].cpu().numpy().view(np.uint32), nd[key]), key
        n0 += g.n
        g.close()
    w.close()


@pytest.mark.parametrize("pair", [(1, 2), (0, 3), (3, 0)])
def test_let_cells_and_lists_match_the_oracle(pair):
    from gpu_helpers import DEV  # noqa: F401
    from paper_1412_0659_gb300 import domains
    m = workloads.milky_way(30000, seed=77)
    w = _world(m)
    doms = domains.split(w, 4)
    ots, _ = _oracle_domains(m, 4)
    j, i = pair
    (gj, _), (gi, _) = doms[j], doms[i]
    let = domains.Let().build(gj, gi, 0.4)
    src, kind = [x.cpu().numpy() for x in let.cells()]
    v, o = ots[j].let_mark(ots[i], 0.4)
    assert np.array_equal(src, np.nonzero(v)[0])
    leaf = ots[j].nodes()["nchild"] == 0
    want_kind = np.where(~o, 0, np.where(leaf, 2, 1))[v]
    assert np.array_equal(kind, want_kind)
    info = let.info()
    assert info["particles"] == int(ots[j].nodes()["count"][o & leaf].sum())
    gi.forces(0.4, m.eps)
    let.add_forces(gi, m.eps)
    npp, npc = [x.cpu().numpy() for x in gi.group_lists()]
    _, _, o_npp, o_npc, counts = ots[j].cross_forces(ots[i], 0.4, m.eps, m.G)
    assert np.array_equal(npp, o_npp) and np.array_equal(npc, o_npc)
    st = gi.stats()
    assert (st["n_pp"], st["n_pc"]) == counts
    let.close()
    for g, _ in doms:
        g.close()
    w.close()


def _oracle_assembled(m, ots, idx, theta, eps):
    acc = np.zeros((3, m.n))
    pot = np.zeros(m.n)
    for i, ti in enumerate(ots):
        a, p, _ = ti.forces(theta, eps, m.G)
        for j, tj in enumerate(ots):
            if j != i:
                a2, p2, _, _, _ = tj.cross_forces(ti, theta, eps, m.G)
                a, p = a + a2, p + p2
        acc[:, idx[i]] = a
        pot[idx[i]] = p
    return acc, pot


@pytest.mark.parametrize("R", [3, 8])
def test_assembled_forces_match_the_oracle(R):
    from gpu_helpers import assert_force_tolerance
    from paper_1412_0659_gb300 import domains
    m = workloads.milky_way(40000, seed=31)
    w = _world(m)
    doms = domains.split(w, R)
    acc, pot, sizes = domains.domain_forces(doms, 0.4, m.eps)
    ots, idx = _oracle_domains(m, R)
    ao, po = _oracle_assembled(m, ots, idx, 0.4, m.eps)
    assert_force_tolerance(acc.double().cpu().numpy(), pot.double().cpu().numpy(), ao, po)
    assert len(sizes) == R * (R - 1)
    # a remote domain needs only part of a tree
    assert all(s["cells"] < s["source_cells"] for s in sizes.values())
    # the decomposition follows direct summation as well as one tree does
    ag, _ = w.forces(0.4, m.eps)
    sel = np.arange(0, m.n, 11)
    ad, _ = oracle.direct_forces(m.pos, m.mass, m.eps, m.G, targets=sel)

    def med(a):
        return np.median(np.linalg.norm(a[:, sel] - ad, axis=0) / np.linalg.norm(ad, axis=0))
    assert med(acc.double().cpu().numpy()) < 2.0 * med(ag.double().cpu().numpy())
    for g, _ in doms:
        g.close()
    w.close()


def test_let_errors():
    from paper_1412_0659_gb300 import TreeGravity, capi, domains
    m = workloads.plummer(3000, seed=2)
    w = _world(m)
    (ga, _), (gb, _) = domains.split(w, 2)
    let = domains.Let()
    with pytest.raises(capi.BonsaiError) as e:  # no forces yet on the receiver
        let.build(ga, gb, 0.4).add_forces(gb, 0.01)
    assert e.value.code == capi.BONSAI_ESTATE
    other = TreeGravity()
    other.build(torch.from_numpy(2.0 * m.pos).cuda(), torch.from_numpy(m.mass).cuda())  # another cube
    with pytest.raises(capi.BonsaiError) as e:
        let.build(ga, other, 0.4)
    assert e.value.code == capi.BONSAI_EINVAL
    let.close()
    for g in (ga, gb, other, w):
        g.close()


def test_fullsize_let_pair():
    """The 2^23 benchmark model in 8 domains: the LET from domain 3 to
    domain 4 (neighbours on the curve) cell for cell, and its lists."""
    from paper_1412_0659_gb300 import domains
    m = workloads.config_model(1)
    w = _world(m)
    doms = domains.split(w, 8)
    t = oracle.Tree(m.pos, m.mass)
    _, perm = t.keys()
    cube = t.cube()
    del t
    cut = [m.n * r // 8 for r in range(9)]
    o3 = oracle.Tree(m.pos[:, perm[cut[3]:cut[4]]], m.mass[perm[cut[3]:cut[4]]], cube=cube)
    o4 = oracle.Tree(m.pos[:, perm[cut[4]:cut[5]]], m.mass[perm[cut[4]:cut[5]]], cube=cube)
    let = domains.Let().build(doms[3][0], doms[4][0], 0.4)
    src, _ = [x.cpu().numpy() for x in let.cells()]
    v, _ = o3.let_mark(o4, 0.4)
    assert np.array_equal(src, np.nonzero(v)[0])
    g4 = doms[4][0]
    g4.forces(0.4, m.eps)
    let.add_forces(g4, m.eps)
    npp, npc = [x.cpu().numpy() for x in g4.group_lists()]
    _, _, o_npp, o_npc, _ = o3.cross_forces(o4, 0.4, m.eps, m.G)
    assert np.array_equal(npp, o_npp) and np.array_equal(npc, o_npc)
    let.close()
    for g, _ in doms:
        g.close()
    w.close()
