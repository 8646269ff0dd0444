"""Leap-frog and diagnostics on the GPU against the oracle (Sec. III.B.2:
second-order leap-frog; FP64 state on the device)."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


def test_plummer_eight_kdk_steps_follow_the_oracle():
    """Plummer sphere, N = 2^14, G = M = a = 1, eps = 0.01, theta = 0.4,
    one force evaluation + 8 steps of dt = 1/64.  FP32 forces differ from the
    FP64 oracle by ~1e-6 (median) per evaluation, so after 8 steps positions
    agree to ~ 8^2 dt^2 * 1e-4 |a| and velocities to ~ 8 dt * 1e-4 |a|."""
    from gpu_helpers import DEV
    from paper_1412_0659_gb300 import TreeGravity
    m = workloads.plummer(1 << 14, seed=1001)
    g = TreeGravity(G=1.0, theta=0.4, eps=0.01)
    g.build(torch.from_numpy(m.pos).to(DEV), torch.from_numpy(m.mass).to(DEV))
    g.set_velocities(torch.from_numpy(m.vel).to(DEV))
    for _ in range(8):
        g.step(m.dt)
    pos, vel, mass = (t.cpu().numpy() for t in g.state())
    acc, pot = (t.cpu().numpy().astype(np.float64) for t in g.last_forces())
    d = g.diagnostics()
    g.close()
    op, ov, oa, opot = oracle.kdk(m.pos, m.vel, m.mass, 8, m.dt, theta=0.4, eps=0.01)
    assert np.array_equal(mass, m.mass)
    dx = np.linalg.norm(pos - op, axis=0)
    dv = np.linalg.norm(vel - ov, axis=0)
    amag = np.linalg.norm(oa, axis=0)
    assert np.median(dx / amag) < 1e-8 and np.max(dx / amag) < 1e-5
    assert np.median(dv / amag) < 1e-7 and np.max(dv / amag) < 1e-4
    e = np.linalg.norm(acc - oa, axis=0) / amag
    assert np.median(e) < 2e-6 and np.quantile(e, 0.999) < 1e-4
    od = oracle.diagnostics(op, ov, m.mass, opot)
    assert d["E_kin"] == pytest.approx(od[0], rel=1e-6)
    assert d["E_pot"] == pytest.approx(od[1], rel=1e-6)
    assert d["M"] == pytest.approx(od[9], rel=1e-14)
    for k, i in (("Px", 3), ("Py", 4), ("Pz", 5)):
        assert abs(d[k] - od[i]) < 1e-6 * np.abs(m.mass * np.linalg.norm(m.vel, axis=0)).sum()


def test_diagnostics_match_oracle_on_the_same_state():
    from gpu_helpers import DEV
    from paper_1412_0659_gb300 import TreeGravity
    m = workloads.milky_way(50000, seed=4)
    g = TreeGravity(G=m.G, theta=0.4, eps=m.eps)
    g.build(torch.from_numpy(m.pos).to(DEV), torch.from_numpy(m.mass).to(DEV))
    g.set_velocities(torch.from_numpy(m.vel).to(DEV))
    acc, pot = g.forces()
    d = g.diagnostics()
    g.close()
    od = oracle.diagnostics(m.pos, m.vel, m.mass, pot.cpu().numpy().astype(np.float64))
    keys = ("E_kin", "E_pot", "E_tot", "Px", "Py", "Pz", "Lx", "Ly", "Lz", "M")
    scale_p = (m.mass * np.linalg.norm(m.vel, axis=0)).sum()
    scale_l = (m.mass * np.linalg.norm(np.cross(m.pos.T, m.vel.T), axis=1)).sum()
    for i, k in enumerate(keys):
        tol = {3: scale_p, 4: scale_p, 5: scale_p, 6: scale_l, 7: scale_l, 8: scale_l}.get(i, abs(od[i]))
        assert abs(d[k] - od[i]) <= 1e-12 * tol, (k, d[k], od[i])


def test_free_drift_and_single_particle():
    from gpu_helpers import DEV
    from paper_1412_0659_gb300 import TreeGravity
    g = TreeGravity(G=1.0, theta=0.4, eps=0.1)
    g.build(torch.tensor([[1.0], [2.0], [3.0]], dtype=torch.float64, device=DEV),
            torch.tensor([1.0], dtype=torch.float64, device=DEV))
    v0 = torch.tensor([[0.5], [-0.25], [0.125]], dtype=torch.float64, device=DEV)
    g.set_velocities(v0)
    for _ in range(8):
        g.step(0.25)
    pos, vel, _ = g.state()
    g.close()
    assert torch.equal(pos.cpu(), torch.tensor([[1.0], [2.0], [3.0]], dtype=torch.float64) + 2.0 * v0.cpu())
    assert torch.equal(vel.cpu(), v0.cpu())


@pytest.mark.parametrize("copies", [3, 40])
def test_a_step_orders_equal_keys_by_caller_index_like_a_fresh_build(copies):
    """Coincident copies share a key.  After a step (which sorts the
    key-ordered state: runs of at most 32 equal keys are put in caller
    order after the sort, longer runs take the path that writes each key at
    its caller index), the order must be the (key, caller index) order that
    a fresh build of the same state gives, and every later tree with it.
    Copies of one particle get the same velocity and feel the same force,
    so they stay coincident."""
    from gpu_helpers import DEV
    from paper_1412_0659_gb300 import TreeGravity
    m = workloads.plummer(4096, seed=31)
    rng = np.random.default_rng(32)
    src = rng.choice(m.n, 12, replace=False)
    pos = np.concatenate([m.pos] + [m.pos[:, src]] * copies, axis=1)
    vel = np.concatenate([m.vel] + [m.vel[:, src]] * copies, axis=1)
    mass = np.concatenate([m.mass] + [m.mass[src]] * copies)
    shuffle = rng.permutation(pos.shape[1])  # copies spread over the caller indices
    pos, vel, mass = pos[:, shuffle], vel[:, shuffle], mass[shuffle]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    with TreeGravity(G=1.0, theta=0.4, eps=0.01) as g:
        g.build(t(pos), t(mass))
        g.set_velocities(t(vel))
        g.step(1.0 / 64)
        g.step(1.0 / 64)
        d_step = g.debug()
        p1, v1, m1 = g.state()
        keys = d_step["keys"].cpu().numpy().view(np.uint64)
        perm = d_step["perm"].cpu().numpy()
        edges = np.concatenate([[0], np.flatnonzero(np.diff(keys)) + 1, [keys.size]])
        assert np.diff(edges).max() >= copies + 1  # the copies did tie
        with TreeGravity(G=1.0, theta=0.4, eps=0.01) as f:
            f.build(p1, m1)
            d_build = f.debug()
    assert np.array_equal(keys, d_build["keys"].cpu().numpy().view(np.uint64))
    assert np.array_equal(perm, d_build["perm"].cpu().numpy())
    for k in ("first", "count", "child", "nchild"):
        assert torch.equal(d_step["nodes"][k], d_build["nodes"][k]), k
