"""Direct summation on the GPU (the O(N^2) definition that the tree
approximates) against the FP64 oracle's direct sum O1: all targets on small
inputs (incl. eps = 0 and coincident clumps), target subsets, bad indices,
and sampled targets at the full 2^23 benchmark size.  The bounds follow from
the arithmetic: FP32 pair terms on head/remainder coordinates (~1e-7
relative each), FP32 sums over tiles of 256 sources and FP64 beyond, so the
potential (a sum of same-sign terms) is within 1e-6 and the acceleration
within 1e-6 of the sum of the magnitudes of its terms, which the median and
99th-percentile bounds below express."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

G_MW = 4.498502151469554e-12


def _cases():
    rng = np.random.default_rng(31)
    out = {}
    m = workloads.plummer(3000, seed=5)
    out["plummer3000"] = (m.pos, m.mass, 0.01, 1.0)
    out["uniform2049_eps0"] = (rng.uniform(-1, 1, (3, 2049)), rng.uniform(0.5, 1.5, 2049), 0.0, 1.0)
    clump = np.concatenate([rng.normal(0, 1e-3, (3, 700)), rng.normal(3, 0.5, (3, 1300))], 1)
    out["clumps2000"] = (clump, rng.uniform(0.5, 1.5, 2000), 1e-4, 1.0)
    mw = workloads.milky_way(5000, seed=8)
    out["milkyway5000"] = (mw.pos, mw.mass, 0.01, G_MW)
    return out


CASES = _cases()


def _errs(acc, pot, acc_o, pot_o):
    e = np.linalg.norm(acc - acc_o, axis=0) / np.linalg.norm(acc_o, axis=0)
    pe = np.abs(pot - pot_o) / np.abs(pot_o)
    return e, pe


def _gravity(pos, mass, eps, G):
    import torch

    from gpu_helpers import DEV
    from paper_1412_0659_gb300 import TreeGravity
    g = TreeGravity(G=G, theta=0.4, eps=eps)
    g.build(torch.from_numpy(np.ascontiguousarray(pos)).to(DEV),
            torch.from_numpy(np.ascontiguousarray(mass)).to(DEV))
    return g


@pytest.mark.parametrize("name", list(CASES))
def test_all_targets_match_oracle_direct_sum(name):
    pos, mass, eps, G = CASES[name]
    g = _gravity(pos, mass, eps, G)
    acc, pot = g.direct_forces()
    g.close()
    acc_o, pot_o = oracle.direct_forces(pos, mass, eps, G)
    e, pe = _errs(acc.cpu().numpy(), pot.cpu().numpy(), acc_o, pot_o)
    assert np.median(e) <= 1e-6 and np.quantile(e, 0.99) <= 1e-5, (np.median(e), np.quantile(e, 0.99))
    assert pe.max() <= 1e-6, pe.max()


def test_target_subset_in_the_given_order_and_bad_index():
    import torch

    from paper_1412_0659_gb300 import capi
    pos, mass, eps, G = CASES["plummer3000"]
    idx = np.random.default_rng(4).permutation(3000)[:777]
    g = _gravity(pos, mass, eps, G)
    acc, pot = g.direct_forces(torch.from_numpy(idx))
    acc_o, pot_o = oracle.direct_forces(pos, mass, eps, G, targets=idx)
    e, pe = _errs(acc.cpu().numpy(), pot.cpu().numpy(), acc_o, pot_o)
    assert np.median(e) <= 1e-6 and pe.max() <= 1e-6
    for bad in (-1, 3000):
        with pytest.raises(capi.BonsaiError) as ex:
            g.direct_forces(torch.tensor([0, bad, 5]))
        assert ex.value.code == capi.BONSAI_EINVAL
    acc2, _ = g.direct_forces(torch.from_numpy(idx))  # usable afterwards, deterministic
    assert torch.equal(acc2, acc)
    g.close()


def test_fullsize_sampled_targets_match_oracle_direct_sum():
    """The 2^23 Milky-Way-like benchmark model: 48 seeded targets against
    the FP64 direct sum over all 2^23 sources."""
    import torch
    m = workloads.milky_way(1 << 23, seed=1002, eps=0.01, theta=0.4, dt=0.1)
    idx = np.sort(np.random.default_rng(11).choice(m.n, 48, replace=False))
    g = _gravity(m.pos, m.mass, m.eps, m.G)
    acc, pot = g.direct_forces(torch.from_numpy(idx))
    g.close()
    acc_o, pot_o = oracle.direct_forces(m.pos, m.mass, m.eps, m.G, targets=idx)
    e, pe = _errs(acc.cpu().numpy(), pot.cpu().numpy(), acc_o, pot_o)
    assert np.median(e) <= 1e-6 and e.max() <= 1e-4, (np.median(e), e.max())
    assert pe.max() <= 1e-6, pe.max()


def test_tree_error_against_direct_sum_shrinks_with_theta():
    """The tree approximates the direct sum: its error, measured against
    the GPU direct sum, decreases as the opening angle decreases."""
    import torch
    m = workloads.milky_way(1 << 18, seed=21)
    idx = torch.from_numpy(np.random.default_rng(2).choice(m.n, 4096, replace=False))
    g = _gravity(m.pos, m.mass, m.eps, m.G)
    ad, _ = g.direct_forces(idx)
    ad = ad.cpu().numpy()
    med = []
    for theta in (0.8, 0.6, 0.4, 0.2):
        acc, _ = g.forces(theta, m.eps)
        a = acc.double().cpu().numpy()[:, idx.numpy()]
        med.append(float(np.median(np.linalg.norm(a - ad, axis=0) / np.linalg.norm(ad, axis=0))))
    g.close()
    assert all(x > y for x, y in zip(med, med[1:])), med
    assert med[2] < 1e-3, med
