"""The oracle on the shapes of the differentiable run: the gradient of the
surface-density loss after 64 leap-frog steps (reverse KDK chain with each
step's lists frozen) against central finite differences of the same frozen
chain, in FP64, on 32 seeded coordinates of a 2048 + 2048 halo + disk
model; and the loss gradient itself against finite differences."""
import numpy as np

import oracle
import workloads
from surface_density import density_map, loss, loss_grad

K, DT, EPS, THETA = 64, 0.1, 0.02, 0.4


def _model():
    m = workloads.halo_disk(2048, 2048, seed=1004, eps=EPS, dt=DT)
    target = density_map(workloads.halo_disk(2048, 2048, seed=1005).pos, m.mass)
    return m, target


def test_loss_gradient_matches_finite_differences():
    m, target = _model()
    gx, gm = loss_grad(m.pos, m.mass, target)
    rng = np.random.default_rng(3)
    for i in rng.choice(m.n, 8, replace=False):
        for d in (0, 1):
            h = 1e-6
            p = m.pos.copy()
            p[d, i] += h
            lp = loss(p, m.mass, target)
            p[d, i] -= 2 * h
            fd = (lp - loss(p, m.mass, target)) / (2 * h)
            assert abs(fd - gx[d, i]) <= 1e-5 * max(abs(gx[d, i]), np.abs(gx).max() * 1e-3), (i, d)
        h = 1e-6 * m.mass[i]
        mm = m.mass.copy()
        mm[i] += h
        lp = loss(m.pos, mm, target)
        mm[i] -= 2 * h
        fd = (lp - loss(m.pos, mm, target)) / (2 * h)
        assert abs(fd - gm[i]) <= 1e-5 * max(abs(gm[i]), np.abs(gm).max() * 1e-3)


def test_differentiable_run_gradient_matches_finite_differences():
    m, target = _model()
    plan = oracle.KdkPlan(m.pos, m.vel, m.mass, K, DT, theta=THETA, eps=EPS, G=m.G)
    xk, _ = plan.run(m.pos, m.vel)
    cx, cm = loss_grad(xk, m.mass, target)
    xb, vb, mb = plan.vjp(cx, np.zeros_like(cx), cm)

    def L(p0, v0, mass):
        p, _ = plan.run(p0, v0, mass)
        return loss(p, mass, target)

    rng = np.random.default_rng(5)
    idx = rng.choice(m.n, 32, replace=False)
    kinds = ["x"] * 12 + ["v"] * 12 + ["m"] * 8
    for i, kind in zip(idx, kinds):
        d = int(rng.integers(0, 3))
        p0, v0, ms = m.pos.copy(), m.vel.copy(), m.mass.copy()
        if kind == "x":
            arr, h, adj = p0, 1e-5, xb[d, i]
        elif kind == "v":
            arr, h, adj = v0, 1e-7, vb[d, i]
        else:
            arr, h, adj = ms, 1e-6 * m.mass[i], mb[i]
        ref = arr[d, i] if arr.ndim == 2 else arr[i]
        if arr.ndim == 2:
            arr[d, i] = ref + h
        else:
            arr[i] = ref + h
        lp = L(p0, v0, ms)
        if arr.ndim == 2:
            arr[d, i] = ref - h
        else:
            arr[i] = ref - h
        fd = (lp - L(p0, v0, ms)) / (2 * h)
        scale = {"x": np.abs(xb).max(), "v": np.abs(vb).max(), "m": np.abs(mb).max()}[kind]
        assert abs(fd - adj) <= 1e-4 * max(abs(adj), 1e-2 * scale), (kind, i, d, fd, adj)
