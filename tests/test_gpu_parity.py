"""GPU path vs the FP64 oracle, element by element, on seeded inputs that
span several tiles and ragged tails: bit-exact keys, order, topology and
groups; FP64 multipoles; equal interaction lists per group; forces within
the stated tolerance."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _cases():
    rng = np.random.default_rng(123)
    out = {}
    m = workloads.plummer(20011, seed=1001)           # several sort tiles, ragged tail
    out["plummer20011"] = (m.pos, m.mass, 0.01)
    out["uniform4099"] = (rng.uniform(-1, 1, (3, 4099)), rng.uniform(0.5, 1.5, 4099), 0.01)
    clump = np.concatenate([rng.normal(0, 1e-3, (3, 700)), rng.normal(3, 0.5, (3, 1300))], 1)
    out["clumps2000"] = (clump, rng.uniform(0.5, 1.5, 2000), 1e-4)
    dup = rng.uniform(-1, 1, (3, 1500))
    dup[:, 500:650] = dup[:, 11:12]                   # 151 coincident: max-depth leaf, > 64
    out["coincident1500"] = (dup, np.full(1500, 1.0 / 1500), 0.01)
    mw = workloads.milky_way(30000, seed=77)
    out["milkyway30000"] = (mw.pos, mw.mass, 0.01)
    # 118 clumps of 17 particles, 1e-5 across: each clump is a chain of
    # single-child nodes down to the level that separates its particles,
    # more nodes in all than the octree's first launch has room for.  The
    # softening (0.5) keeps the pair forces inside a clump negligible: FP32
    # coordinates relative to a group that spans several clumps resolve
    # separations of 1e-5 only to about 1e-3.
    centres = rng.uniform(-1, 1, (3, 118))
    chains = (centres[:, :, None] + rng.normal(0, 1e-5, (3, 118, 17))).reshape(3, -1)
    out["chains2006"] = (chains, rng.uniform(0.5, 1.5, chains.shape[1]), 0.5)
    return out


CASES = _cases()


@pytest.fixture(scope="module", params=list(CASES))
def run(request):
    from gpu_helpers import gpu_run, oracle_tree
    pos, mass, eps = CASES[request.param]
    G = 4.498502151469554e-12 if request.param.startswith("milky") else 1.0
    gpu = gpu_run(pos, mass, theta=0.4, eps=eps, G=G)
    t = oracle_tree(pos, mass)
    yield request.param, pos, mass, eps, G, gpu, t
    gpu["g"].close()


def test_cube_keys_and_order_bit_exact(run):
    name, pos, mass, eps, G, gpu, t = run
    lo, L = t.cube()
    assert np.array_equal(gpu["lo"], lo) and gpu["L"] == L
    key, perm = t.keys()
    assert np.array_equal(gpu["keys"], key)
    assert np.array_equal(gpu["perm"], perm)


def test_topology_bit_exact(run):
    name, pos, mass, eps, G, gpu, t = run
    nd = t.nodes()
    assert gpu["stats"]["n_nodes"] == t.nnodes
    for k in ("first", "count", "child", "nchild", "level"):
        assert np.array_equal(gpu["nodes"][k], nd[k]), k
    g = t.groups()
    assert gpu["stats"]["n_groups"] == t.ngroups
    assert np.array_equal(gpu["group_first"], g["first"])
    assert np.array_equal(gpu["group_count"], g["count"])


def test_multipoles_fp64(run):
    name, pos, mass, eps, G, gpu, t = run
    mp = t.multipoles()
    M = mp["M"]
    assert np.all(np.abs(gpu["M"] - M) <= 1e-14 * M)
    _, L = t.cube()
    assert np.all(np.abs(gpu["com"] - mp["com"]) <= 1e-14 * L)
    side = mp["side"]
    assert np.all(np.abs(gpu["Q"] - mp["Q"]) <= 1e-13 * M * side * side + 1e-300)


def test_node_storage_grows_for_deep_chains():
    """The octree's first launch holds n/2 + 64 nodes; the clump chains need
    more, so the build must report the overflow, grow its node arrays and
    build again (the topology test checks the result against the oracle)."""
    from gpu_helpers import gpu_run
    pos, mass, eps = CASES["chains2006"]
    gpu = gpu_run(pos, mass, theta=0.4, eps=eps)
    assert gpu["stats"]["n_nodes"] > pos.shape[1] // 2 + 64
    assert gpu["stats"]["depth"] >= 15
    gpu["g"].close()


def test_interaction_lists_match(run):
    name, pos, mass, eps, G, gpu, t = run
    _, _, g_npp, g_npc, (npp, npc) = t.forces_sorted(0.4, eps, G)
    assert np.array_equal(gpu["g_npp"], g_npp)
    assert np.array_equal(gpu["g_npc"], g_npc)
    assert (gpu["stats"]["n_pp"], gpu["stats"]["n_pc"]) == (npp, npc)


def test_interaction_list_membership(run):
    """Every group's accepted cells and p-p sources are the oracle's, as sets
    (the GPU walks breadth-first, the oracle depth-first): a list that traded
    one cell for another of the same count would fail here."""
    name, pos, mass, eps, G, gpu, t = run
    pc_off, pc, pp_off, pp = (a.cpu().numpy() for a in gpu["g"].group_list_members())
    nd = t.nodes()
    for g in range(t.ngroups):
        cells, leaves = t.group_lists(0.4, g)
        got = np.sort(pc[pc_off[g]:pc_off[g + 1]].astype(np.int64))
        assert np.array_equal(got, np.sort(cells.astype(np.int64))), (name, g)
        src = np.concatenate([np.arange(nd["first"][c], nd["first"][c] + nd["count"][c], dtype=np.int64)
                              for c in leaves]) if len(leaves) else np.zeros(0, np.int64)
        got = np.sort(pp[pp_off[g]:pp_off[g + 1]].astype(np.int64))
        assert np.array_equal(got, np.sort(src)), (name, g)


def test_forces_within_tolerance(run):
    from gpu_helpers import assert_force_tolerance
    name, pos, mass, eps, G, gpu, t = run
    acc_o, pot_o, _ = t.forces(0.4, eps, G)
    assert_force_tolerance(gpu["acc"], gpu["pot"], acc_o, pot_o)


@pytest.mark.parametrize("theta", [0.3, 0.6, 1.0])
def test_other_opening_angles(theta):
    from gpu_helpers import assert_force_tolerance, gpu_run, oracle_tree
    m = workloads.plummer(9000, seed=5)
    gpu = gpu_run(m.pos, m.mass, theta=theta, eps=0.01, debug=False)
    t = oracle_tree(m.pos, m.mass)
    acc_o, pot_o, (npp, npc) = t.forces(theta, 0.01)
    assert (gpu["stats"]["n_pp"], gpu["stats"]["n_pc"]) == (npp, npc)
    assert_force_tolerance(gpu["acc"], gpu["pot"], acc_o, pot_o)
    gpu["g"].close()


def test_tiny_and_degenerate_inputs():
    """n = 1 (no interaction), n = 2 (the root is a leaf: direct), n = 16 and
    17 (one leaf / first split), 65 (first group split)."""
    import oracle
    from gpu_helpers import gpu_run
    rng = np.random.default_rng(9)
    gpu = gpu_run(np.array([[0.5], [1.0], [-2.0]]), np.array([3.0]), eps=0.1)
    assert np.all(gpu["acc"] == 0) and np.all(gpu["pot"] == 0)
    assert (gpu["stats"]["n_pp"], gpu["stats"]["n_pc"]) == (1, 0)
    gpu["g"].close()
    for n in (2, 16, 17, 64, 65, 200):
        pos = rng.standard_normal((3, n))
        mass = rng.uniform(0.5, 1.5, n)
        gpu = gpu_run(pos, mass, eps=0.05)
        t = oracle.Tree(pos, mass)
        acc_o, pot_o, counts = t.forces(0.4, 0.05)
        assert (gpu["stats"]["n_pp"], gpu["stats"]["n_pc"]) == counts
        assert np.array_equal(gpu["keys"], t.keys()[0])
        e = np.linalg.norm(gpu["acc"] - acc_o, axis=0) / np.linalg.norm(acc_o, axis=0)
        assert e.max() < 1e-5, (n, e.max())
        gpu["g"].close()


def test_all_particles_at_one_point():
    """Degenerate input: 200 coincident particles (L = 1, equal keys, one
    max-depth leaf cut into groups of 64): a = 0 exactly and
    phi = -G (n - 1) m / eps, the oracle's closed form."""
    from gpu_helpers import gpu_run
    n, m, eps, G = 200, 0.5, 0.02, 2.0
    pos = np.tile(np.array([[0.3], [-1.2], [4.0]]), (1, n))
    gpu = gpu_run(pos, np.full(n, m), eps=eps, G=G)
    assert gpu["L"] == 1.0
    assert np.all(gpu["acc"] == 0.0)
    assert np.allclose(gpu["pot"], -G * (n - 1) * m / eps, rtol=1e-6)
    assert (gpu["stats"]["n_pp"], gpu["stats"]["n_pc"]) == (n * n, 0)
    assert np.array_equal(gpu["group_count"], [64, 64, 64, 8])
    gpu["g"].close()


def test_empty_input_is_rejected():
    import torch

    from gpu_helpers import DEV
    from paper_1412_0659_gb300 import TreeGravity, capi
    g = TreeGravity()
    with pytest.raises(capi.BonsaiError) as e:
        g.build(torch.zeros((3, 0), dtype=torch.float64, device=DEV),
                torch.zeros(0, dtype=torch.float64, device=DEV))
    assert e.value.code == capi.BONSAI_EINVAL
    g.close()


def test_zero_softening_distinct_particles():
    from gpu_helpers import assert_force_tolerance, gpu_run, oracle_tree
    m = workloads.plummer(5000, seed=12)
    gpu = gpu_run(m.pos, m.mass, eps=0.0, debug=False)
    acc_o, pot_o, _ = oracle_tree(m.pos, m.mass).forces(0.4, 0.0)
    assert np.all(np.isfinite(gpu["acc"])) and np.all(np.isfinite(gpu["pot"]))
    assert_force_tolerance(gpu["acc"], gpu["pot"], acc_o, pot_o)
    gpu["g"].close()


def test_invalid_inputs_are_reported():
    import torch

    from gpu_helpers import DEV
    from paper_1412_0659_gb300 import TreeGravity, capi
    g = TreeGravity()
    with pytest.raises(capi.BonsaiError) as e:
        g.forces()
    assert e.value.code == capi.BONSAI_ESTATE
    pos = torch.randn(3, 100, dtype=torch.float64, device=DEV)
    mass = torch.ones(100, dtype=torch.float64, device=DEV)
    bad = pos.clone()
    bad[1, 37] = float("nan")
    with pytest.raises(capi.BonsaiError) as e:
        g.build(bad, mass)
    assert e.value.code == capi.BONSAI_EINVAL
    m0 = mass.clone()
    m0[5] = 0.0
    with pytest.raises(capi.BonsaiError) as e:
        g.build(pos, m0)
    assert e.value.code == capi.BONSAI_EINVAL
    g.build(pos, mass)
    with pytest.raises(capi.BonsaiError) as e:
        g.forces(theta=0.0)
    assert e.value.code == capi.BONSAI_EINVAL
    acc, pot = g.forces()
    assert torch.isfinite(acc).all()
    g.close()


def test_host_buffer_entry_matches_device_path():
    import torch

    from gpu_helpers import gpu_run
    from paper_1412_0659_gb300 import TreeGravity
    m = workloads.plummer(12345, seed=3)
    ref = gpu_run(m.pos, m.mass, debug=False)
    g = TreeGravity(theta=0.4, eps=0.01)
    pos = torch.from_numpy(m.pos).pin_memory()
    mass = torch.from_numpy(m.mass).pin_memory()
    acc = torch.empty((3, m.n), dtype=torch.float32).pin_memory()
    pot = torch.empty(m.n, dtype=torch.float32).pin_memory()
    g.solve_host(pos, mass, acc, pot)
    assert np.array_equal(acc.numpy(), ref["acc"].astype(np.float32))
    assert np.array_equal(pot.numpy(), ref["pot"].astype(np.float32))
    g.close()
    ref["g"].close()


def test_frontier_overflow_is_reported_and_recoverable():
    """A walk whose frontier exceeds the (test-reduced) capacity stops adding
    cells, sets the device status word and returns BONSAI_EOVERFLOW from the
    forward and the adjoint; the context is usable afterwards."""
    import torch

    from gpu_helpers import DEV, assert_force_tolerance, oracle_tree
    from paper_1412_0659_gb300 import TreeGravity, capi
    m = workloads.plummer(6000, seed=91)
    g = TreeGravity(theta=0.4, eps=0.01)
    g.build(torch.from_numpy(m.pos).to(DEV), torch.from_numpy(m.mass).to(DEV))
    capi.tree_debug_set_frontier_capacity(g.ctx, 8)
    with pytest.raises(capi.BonsaiError) as e:
        g.forces()
    assert e.value.code == capi.BONSAI_EOVERFLOW
    capi.tree_debug_set_frontier_capacity(g.ctx, 0)
    acc, pot = g.forces()
    acc_o, pot_o, _ = oracle_tree(m.pos, m.mass).forces(0.4, 0.01)
    assert_force_tolerance(acc.double().cpu().numpy(), pot.double().cpu().numpy(), acc_o, pot_o)
    capi.tree_debug_set_frontier_capacity(g.ctx, 8)
    with pytest.raises(capi.BonsaiError) as e:
        g.forces_vjp(torch.ones((3, m.n), dtype=torch.float32, device=DEV))
    assert e.value.code == capi.BONSAI_EOVERFLOW
    g.close()


@pytest.mark.parametrize("name", ["plummer20011", "milkyway30000", "coincident1500"])
def test_fp64_variant_matches_oracle_to_round_off(name):
    """The all-FP64 evaluation of the same lists equals the FP64 oracle tree
    to summation-order round-off (1e-12 relative), with identical counts."""
    import torch

    from gpu_helpers import DEV, oracle_tree
    from paper_1412_0659_gb300 import TreeGravity
    pos, mass, eps = CASES[name]
    G = 4.498502151469554e-12 if name.startswith("milky") else 1.0
    g = TreeGravity(G=G, theta=0.4, eps=eps)
    g.build(torch.from_numpy(pos).to(DEV), torch.from_numpy(mass).to(DEV))
    acc, pot = g.forces_fp64(0.4, eps)
    st = g.stats()
    g.close()
    # the C ABI takes eps as float: give the oracle the same FP32-rounded value
    acc_o, pot_o, counts = oracle_tree(pos, mass).forces(0.4, float(np.float32(eps)), G)
    assert (st["n_pp"], st["n_pc"]) == counts
    e = np.linalg.norm(acc.cpu().numpy() - acc_o, axis=0) / np.linalg.norm(acc_o, axis=0)
    pe = np.abs(pot.cpu().numpy() - pot_o) / np.abs(pot_o)
    assert e.max() <= 1e-12 and pe.max() <= 1e-12, (e.max(), pe.max())
