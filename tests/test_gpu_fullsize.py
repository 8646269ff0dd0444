"""Parity at the full benchmark size: the Milky-Way-like model with N = 2^23
(Hernquist halo : exponential disk : Hernquist bulge = 5 : 1 : 0.2, theta =
0.4, eps = 10 pc), in the launch configuration the benchmark times.  Keys,
order, topology and groups are compared whole; forces and list lengths on a
seeded sample of groups that the oracle evaluates one by one."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    from gpu_helpers import gpu_run, oracle_tree
    m = workloads.config_model(1)
    gpu = gpu_run(m.pos, m.mass, theta=m.theta, eps=m.eps, G=m.G)
    t = oracle_tree(m.pos, m.mass)
    yield m, gpu, t
    gpu["g"].close()


def test_fullsize_keys_topology_groups(full):
    m, gpu, t = full
    key, perm = t.keys()
    assert np.array_equal(gpu["keys"], key)
    assert np.array_equal(gpu["perm"], perm)
    nd = t.nodes()
    for k in ("first", "count", "child", "nchild", "level"):
        assert np.array_equal(gpu["nodes"][k], nd[k]), k
    g = t.groups()
    assert np.array_equal(gpu["group_first"], g["first"])
    assert np.array_equal(gpu["group_count"], g["count"])


def test_fullsize_sampled_groups(full):
    from gpu_helpers import assert_force_tolerance
    m, gpu, t = full
    rng = np.random.default_rng(1004)
    starts = np.sort(rng.choice(t.ngroups - 40, 12, replace=False))
    g = t.groups()
    _, perm = t.keys()
    idx, a_o, p_o = [], [], []
    for s in starts:
        acc, pot, g_npp, g_npc, _ = t.forces_sorted(m.theta, m.eps, m.G, int(s), int(s) + 40)
        assert np.array_equal(gpu["g_npp"][s:s + 40], g_npp[s:s + 40])
        assert np.array_equal(gpu["g_npc"][s:s + 40], g_npc[s:s + 40])
        lo = int(g["first"][s])
        hi = int(g["first"][s + 39] + g["count"][s + 39])
        idx.append(perm[lo:hi])
        a_o.append(acc[:, lo:hi])
        p_o.append(pot[lo:hi])
    idx = np.concatenate(idx)
    a_o = np.concatenate(a_o, axis=1)
    p_o = np.concatenate(p_o)
    assert_force_tolerance(gpu["acc"][:, idx], gpu["pot"][idx], a_o, p_o)
    # interaction counts per particle are of the paper's order (Table 2:
    # 1745 p-p and 4529 p-c at 13 M particles, a different model)
    st = gpu["stats"]
    assert 200 < st["n_pp"] / m.n < 20000 and 500 < st["n_pc"] / m.n < 50000
