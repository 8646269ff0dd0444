"""The remaining benchmark configurations at their full sizes, in the launch
configuration of the benchmark (one context, default launch shapes):

- precision study: Milky-Way-like N = 2^25 at theta = 0.3, 0.4, 0.6 --
  tree error against the GPU direct sum on a seeded 2^16 subset, FP32 path
  against the all-FP64 variant, sampled groups against the oracle tree,
  200 leap-frog steps (energy drift, net momentum);
- differentiable run: Plummer halo 2^19 + exponential disk 2^19, the
  surface-density loss after 64 steps, gradients through the adjoint with
  checkpoints every 8 steps, against the oracle's reverse chain at 4096
  particles and against the exact translation and boost identities at full
  size;
- largest single-GPU model: Milky-Way-like N = 2^28, eps = 5 pc -- tree
  against direct sum on sampled targets, the GPU direct sum against the
  oracle's on a few targets, 20 steps, and one adjoint over 4 steps with
  checkpoints (translation identity)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from surface_density import density_map, density_map_torch, loss_grad

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


def _gravity(m, theta=None, eps=None):
    from gpu_helpers import DEV
    from paper_1412_0659_gb300 import TreeGravity
    g = TreeGravity(G=m.G, theta=m.theta if theta is None else theta, eps=m.eps if eps is None else eps)
    g.build(torch.from_numpy(m.pos).to(DEV), torch.from_numpy(m.mass).to(DEV))
    g.set_velocities(torch.from_numpy(m.vel).to(DEV))
    return g


def _energy(d):
    return d["E_tot"], np.array([d["Px"], d["Py"], d["Pz"]])


def test_precision_study_milky_way_2e25():
    from gpu_helpers import assert_force_tolerance
    m = workloads.milky_way(1 << 25, seed=1003, eps=0.01, theta=0.4, dt=0.1)
    g = _gravity(m)
    idx = np.sort(np.random.default_rng(1006).choice(m.n, 1 << 16, replace=False))
    ad, pd = g.direct_forces(torch.from_numpy(idx))
    dev = ad.device
    ad, pd = ad.cpu().numpy(), pd.cpu().numpy()
    med = {}
    idx_d = torch.from_numpy(idx).to(dev)
    for theta in (0.3, 0.4, 0.6):
        acc, pot = g.forces(theta, m.eps)
        e = _rel(acc[:, idx_d].double().cpu().numpy(), ad)
        med[theta] = float(np.median(e))
        print(f"theta {theta}: tree vs direct, median {med[theta]:.3g}, p99 {np.quantile(e, 0.99):.3g}")
    assert med[0.3] < med[0.4] < med[0.6] < 1e-3, med
    # the FP32 path against the all-FP64 evaluation of the same lists
    acc, pot = g.forces(0.4, m.eps)
    a64, p64 = g.forces_fp64(0.4, m.eps)
    assert_force_tolerance(acc.double().cpu().numpy(), pot.double().cpu().numpy(), a64.cpu().numpy(),
                           p64.cpu().numpy())
    # sampled groups against the oracle tree: lists and forces
    t = oracle.Tree(m.pos, m.mass)
    npp_g, npc_g = [x.cpu().numpy() for x in g.group_lists()]
    gr = t.groups()
    _, perm = t.keys()
    starts = np.sort(np.random.default_rng(1007).choice(t.ngroups - 24, 8, replace=False))
    ii, ao, po = [], [], []
    for s in starts:
        a_s, p_s, g_npp, g_npc, _ = t.forces_sorted(0.4, m.eps, m.G, int(s), int(s) + 24)
        assert np.array_equal(npp_g[s:s + 24], g_npp[s:s + 24])
        assert np.array_equal(npc_g[s:s + 24], g_npc[s:s + 24])
        lo, hi = int(gr["first"][s]), int(gr["first"][s + 23] + gr["count"][s + 23])
        ii.append(perm[lo:hi])
        ao.append(a_s[:, lo:hi])
        po.append(p_s[lo:hi])
    ii = np.concatenate(ii)
    assert_force_tolerance(acc.double().cpu().numpy()[:, ii], pot.double().cpu().numpy()[ii],
                           np.concatenate(ao, axis=1), np.concatenate(po))
    del t
    # 200 steps with FP32 forces and FP64 state
    e0, p0 = _energy(g.diagnostics())
    mv = float((m.mass * np.linalg.norm(m.vel, axis=0)).sum())
    for _ in range(200):
        g.step(m.dt)
    e1, p1 = _energy(g.diagnostics())
    drift = abs((e1 - e0) / e0)
    pnet = float(np.linalg.norm(p1)) / mv
    print(f"200 steps: |dE/E| = {drift:.3g}, |sum m v| / sum m|v| = {pnet:.3g}")
    assert drift < 1e-5 and pnet < 2e-5, (drift, pnet)
    g.close()


def _halo_disk_case(n_half, seed=1004):
    m = workloads.halo_disk(n_half, n_half, seed=seed, eps=0.02, dt=0.1)
    target = density_map(workloads.halo_disk(n_half, n_half, seed=seed + 1).pos, m.mass)
    return m, target


def test_differentiable_run_matches_oracle_chain_4096():
    """64 steps, checkpoints every 8; the same cotangent (the loss gradient
    at the oracle's final state) through the GPU and the oracle chains."""
    from gpu_helpers import DEV
    m, target = _halo_disk_case(2048)
    plan = oracle.KdkPlan(m.pos, m.vel, m.mass, 64, m.dt, theta=0.4, eps=m.eps, G=m.G)
    xk, _ = plan.run(m.pos, m.vel)
    cx, cm = loss_grad(xk, m.mass, target)
    oxb, ovb, omb = plan.vjp(cx, np.zeros_like(cx), cm)
    g = _gravity(m)
    g.run(64, m.dt, 8)
    pos, _, _ = g.state()
    assert np.max(np.abs(pos.cpu().numpy() - xk)) < 1e-5 * np.abs(xk).max()
    xb, vb, mb = g.run_vjp(torch.from_numpy(cx).to(DEV), torch.zeros((3, m.n), dtype=torch.float64, device=DEV),
                           torch.from_numpy(cm).to(DEV))
    g.close()
    for got, ref in ((xb, oxb), (vb, ovb)):
        e = np.linalg.norm(got.cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0).max()
        assert np.median(e) <= 1e-5 and e.max() <= 1e-3, (np.median(e), e.max())
    e = np.abs(mb.cpu().numpy() - omb) / np.abs(omb).max()
    assert np.median(e) <= 1e-5 and e.max() <= 1e-3, (np.median(e), e.max())


def test_differentiable_run_full_size_identities():
    """2^19 + 2^19 particles, 64 steps, checkpoints every 8, gradients of the
    loss through autograd.  With each step's lists held fixed the chain is
    exactly invariant under a uniform translation of x0 (the final positions
    translate) and covariant under a uniform boost of v0 (the final
    positions move by K dt times it), so sum_i dL/dx0_i = sum_i dL/dx_K,i
    and sum_i dL/dv0_i = K dt sum_i dL/dx_K,i."""
    from gpu_helpers import DEV
    from paper_1412_0659_gb300.autograd import LeapfrogRun
    m, target = _halo_disk_case(1 << 19)
    g = _gravity(m)
    pos0 = torch.from_numpy(m.pos).to(DEV).requires_grad_(True)
    vel0 = torch.from_numpy(m.vel).to(DEV).requires_grad_(True)
    mass = torch.from_numpy(m.mass).to(DEV).requires_grad_(True)
    p, v = LeapfrogRun.apply(pos0, vel0, mass, g, 64, m.dt, 8)
    pk = p.detach().requires_grad_(True)
    tgt = torch.from_numpy(target).to(DEV)
    lk = ((density_map_torch(pk, mass.detach()) - tgt) ** 2).sum()
    (gxk,) = torch.autograd.grad(lk, pk)
    loss = ((density_map_torch(p, mass) - tgt) ** 2).sum()
    loss.backward()
    g.close()
    for t in (pos0.grad, vel0.grad, mass.grad):
        assert torch.isfinite(t).all()
    sx = pos0.grad.sum(dim=1).cpu().numpy()
    sk = gxk.sum(dim=1).cpu().numpy()
    scale = float(pos0.grad.abs().sum())
    assert np.abs(sx - sk).max() <= 1e-6 * scale, (sx, sk, scale)
    sv = vel0.grad.sum(dim=1).cpu().numpy()
    assert np.abs(sv - 64 * m.dt * sk).max() <= 1e-6 * float(vel0.grad.abs().sum()), (sv, sk)


def test_largest_model_milky_way_2e28():
    from gpu_helpers import DEV
    m = workloads.milky_way(1 << 28, seed=1005, eps=0.005, theta=0.4, dt=0.1)
    g = _gravity(m)
    acc, _ = g.forces(0.4, m.eps)
    st = g.stats()
    assert 200 < st["n_pp"] / m.n < 20000 and 500 < st["n_pc"] / m.n < 50000
    rng = np.random.default_rng(1008)
    idx = np.sort(rng.choice(m.n, 4096, replace=False))
    ad, pd = g.direct_forces(torch.from_numpy(idx))
    e = _rel(acc[:, torch.from_numpy(idx).to(DEV)].double().cpu().numpy(), ad.cpu().numpy())
    print(f"2^28 tree vs direct: median {np.median(e):.3g}, p99 {np.quantile(e, 0.99):.3g}")
    assert np.median(e) < 1e-3
    few = idx[:6]
    ao, po = oracle.direct_forces(m.pos, m.mass, m.eps, m.G, targets=few)
    eo = _rel(ad.cpu().numpy()[:, :6], ao)
    assert eo.max() <= 1e-5, eo
    assert np.max(np.abs(pd.cpu().numpy()[:6] - po) / np.abs(po)) <= 1e-6
    del acc
    e0, _ = _energy(g.diagnostics())
    for _ in range(20):
        g.step(m.dt)
    e1, _ = _energy(g.diagnostics())
    print(f"2^28, 20 steps: |dE/E| = {abs((e1 - e0) / e0):.3g}")
    assert abs((e1 - e0) / e0) < 1e-5
    # one adjoint over 4 steps with checkpoints every 2 steps
    g.run(4, m.dt, 2)
    cx = torch.randn((3, m.n), dtype=torch.float64, device=DEV)
    xb, vb, mb = g.run_vjp(cx, torch.zeros_like(cx))
    g.close()
    assert torch.isfinite(xb).all() and torch.isfinite(vb).all() and torch.isfinite(mb).all()
    d = (xb.sum(dim=1) - cx.sum(dim=1)).abs().max().item()
    assert d <= 1e-6 * xb.abs().sum().item(), d
