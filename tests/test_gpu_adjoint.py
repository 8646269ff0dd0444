"""The CUDA adjoint against the FP64 oracle adjoint (same frozen lists):
force VJP per particle, the theta -> 0 limit against the direct-summation
adjoint, the reverse leap-frog chain with checkpoints, and the autograd
wrappers."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _rel(a, b):
    """Per-particle relative error of 3-vectors (columns) or scalars.  With
    random cotangents a particle's gradient is a sum of thousands of FP32
    terms of both signs that can nearly cancel; its rounding error is about
    eps_32 sqrt(n_terms) |term|, i.e. ~1e-6 of the RMS gradient.  The
    denominator is therefore floored at 1e-2 of the RMS gradient, so that
    near-zero sums do not count as relative errors of order one."""
    if a.ndim == 2:
        nb = np.linalg.norm(b, axis=0)
        return np.linalg.norm(a - b, axis=0) / np.maximum(nb, 1e-2 * np.sqrt((nb ** 2).mean()))
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-2 * np.sqrt((b ** 2).mean()))


def _gpu_vjp(m, theta, eps, G, lam, mu):
    from gpu_helpers import DEV
    from paper_1412_0659_gb300 import TreeGravity
    g = TreeGravity(G=G, theta=theta, eps=eps)
    g.build(torch.from_numpy(m.pos).to(DEV), torch.from_numpy(m.mass).to(DEV))
    g.forces(theta, eps)
    gx, gm = g.forces_vjp(torch.from_numpy(lam).float().to(DEV),
                          None if mu is None else torch.from_numpy(mu).float().to(DEV))
    out = gx.cpu().numpy(), gm.cpu().numpy()
    g.close()
    return out


def _oracle_vjp(m, theta, eps, G, lam, mu):
    t = oracle.Tree(m.pos, m.mass)
    t.freeze_lists(theta)
    x, ms = t.sorted_state()
    # the GPU sees the cotangents rounded to FP32
    lam32 = lam.astype(np.float32).astype(np.float64)
    mu32 = None if mu is None else mu.astype(np.float32).astype(np.float64)
    gx, gm = t.frozen_vjp(eps, G, x, ms, t.to_sorted(lam32), None if mu32 is None else t.to_sorted(mu32))
    return t.to_caller(gx), t.to_caller(gm)


CASES = {
    "plummer20011": (lambda: workloads.plummer(20011, seed=1001), 0.01, 1.0),
    "milkyway30000": (lambda: workloads.milky_way(30000, seed=77), 0.01, workloads.G_KPC_MSUN_MYR),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("with_mu", [False, True])
def test_force_vjp_matches_oracle(name, with_mu):
    make, eps, G = CASES[name]
    m = make()
    rng = np.random.default_rng(2024)
    lam = rng.normal(size=(3, m.n))
    mu = rng.normal(size=m.n) if with_mu else None
    gx, gm = _gpu_vjp(m, 0.4, eps, G, lam, mu)
    ox, om = _oracle_vjp(m, 0.4, eps, G, lam, mu)
    ex, em = _rel(gx, ox), _rel(gm, om)
    assert np.median(ex) <= 2e-6 and np.quantile(ex, 0.999) <= 1e-4, (np.median(ex), np.quantile(ex, 0.999))
    assert np.median(em) <= 2e-6 and np.quantile(em, 0.999) <= 1e-4, (np.median(em), np.quantile(em, 0.999))


@pytest.mark.parametrize("n", [1, 2, 3, 9, 17, 33, 65, 130])
def test_force_vjp_small_groups(n):
    """Few-particle models whose groups have 1 to 65 members: every ragged
    chunk length (1 to 4 target pairs, with and without a full chunk of 8
    before it) and single-group trees, against the oracle."""
    m = workloads.plummer(n, seed=300 + n) if n > 1 else workloads.plummer(2, seed=301)
    if n == 1:
        m.pos, m.vel, m.mass = m.pos[:, :1].copy(), m.vel[:, :1].copy(), m.mass[:1].copy()
    rng = np.random.default_rng(n)
    lam = rng.normal(size=(3, m.n))
    mu = rng.normal(size=m.n)
    gx, gm = _gpu_vjp(m, 0.4, 0.01, 1.0, lam, mu)
    ox, om = _oracle_vjp(m, 0.4, 0.01, 1.0, lam, mu)
    if n == 1:  # a lone particle: no force, no gradient
        assert np.all(gx == 0) and np.all(ox == 0)
        assert np.allclose(gm, om, atol=1e-12)
        return
    ex, em = _rel(gx, ox), _rel(gm, om)
    assert np.max(ex) <= 1e-4 and np.max(em) <= 1e-4, (np.max(ex), np.max(em))


def test_force_vjp_tends_to_direct_adjoint():
    m = workloads.plummer(3000, seed=61)
    rng = np.random.default_rng(62)
    lam = rng.normal(size=(3, m.n))
    mu = rng.normal(size=m.n)
    gx, gm = _gpu_vjp(m, 1e-4, 0.01, 1.0, lam, mu)
    dx, dm = oracle.direct_vjp(m.pos, m.mass, 0.01, 1.0, lam.astype(np.float32).astype(np.float64),
                               mu.astype(np.float32).astype(np.float64))
    ex, em = _rel(gx, dx), _rel(gm, dm)
    assert np.median(ex) <= 2e-6 and np.quantile(ex, 0.999) <= 1e-4
    assert np.median(em) <= 2e-6 and np.quantile(em, 0.999) <= 1e-4


def test_leapfrog_chain_vjp_matches_oracle():
    """4 KDK steps, checkpoints every 3 steps (two segments), against the
    oracle's reverse chain with frozen per-step trees."""
    from gpu_helpers import DEV
    from paper_1412_0659_gb300 import TreeGravity
    m = workloads.plummer(4096, seed=71)
    dt = 1.0 / 64
    rng = np.random.default_rng(72)
    cx = rng.normal(size=(3, m.n))
    cv = rng.normal(size=(3, m.n))
    g = TreeGravity(G=1.0, theta=0.4, eps=0.01)
    g.build(torch.from_numpy(m.pos).to(DEV), torch.from_numpy(m.mass).to(DEV))
    g.set_velocities(torch.from_numpy(m.vel).to(DEV))
    g.run(4, dt, 3)
    pos, vel, _ = g.state()
    xb, vb, mb = g.run_vjp(torch.from_numpy(cx).to(DEV), torch.from_numpy(cv).to(DEV))
    xb, vb, mb = xb.cpu().numpy(), vb.cpu().numpy(), mb.cpu().numpy()
    g.close()
    plan = oracle.KdkPlan(m.pos, m.vel, m.mass, 4, dt, theta=0.4, eps=0.01)
    p_o, v_o = plan.run(m.pos, m.vel)
    assert np.max(np.abs(pos.cpu().numpy() - p_o)) < 1e-6
    oxb, ovb, omb = plan.vjp(cx, cv)
    for got, ref in ((xb, oxb), (vb, ovb)):
        e = _rel(got, ref)
        assert np.median(e) <= 1e-5 and np.quantile(e, 0.999) <= 1e-3, (np.median(e), np.quantile(e, 0.999))
    e = _rel(mb, omb)
    assert np.median(e) <= 1e-5 and np.quantile(e, 0.999) <= 1e-3, (np.median(e), np.quantile(e, 0.999))


def test_autograd_wrappers():
    from gpu_helpers import DEV
    from paper_1412_0659_gb300 import TreeGravity
    from paper_1412_0659_gb300.autograd import LeapfrogRun, TreeForces
    m = workloads.plummer(5000, seed=81)
    pos = torch.from_numpy(m.pos).to(DEV).requires_grad_(True)
    mass = torch.from_numpy(m.mass).to(DEV).requires_grad_(True)
    g = TreeGravity(G=1.0, theta=0.4, eps=0.01)
    acc, pot = TreeForces.apply(pos, mass, g, 0.4, 0.01)
    w = torch.randn_like(acc)
    loss = (w * acc).sum() + pot.sum()
    loss.backward()
    gx, gm = g.forces_vjp(w, torch.ones_like(pot))
    # FP32 atomics make the summation order differ from call to call
    assert torch.allclose(pos.grad, gx, rtol=1e-5, atol=1e-6 * gx.abs().max().item())
    assert torch.allclose(mass.grad, gm, rtol=1e-5, atol=1e-6 * gm.abs().max().item())
    # a leap-frog run: gradient of a linear functional of the final state
    pos0 = torch.from_numpy(m.pos).to(DEV).requires_grad_(True)
    vel0 = torch.from_numpy(m.vel).to(DEV).requires_grad_(True)
    p, v = LeapfrogRun.apply(pos0, vel0, mass.detach(), g, 3, 1.0 / 64, 2)
    (p.sum() + 2.0 * v.sum()).backward()
    assert torch.isfinite(pos0.grad).all() and torch.isfinite(vel0.grad).all()
    # d(sum v_K)/d v_0 is the identity up to O(dt^2) force terms
    assert abs(vel0.grad.mean().item() - (2.0 + 3 / 64)) < 1e-2
    g.close()
