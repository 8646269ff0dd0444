"""Pins for the oracle's adjoint: the vector-Jacobian products of the tree
forces (lists frozen) and of the kick-drift-kick chain are checked against
central finite differences in FP64, against the direct-summation adjoint,
and against translation invariance.  The paper has no adjoint; these pins
only use the forward functions already pinned in test_oracle_forces.py."""
import numpy as np
import pytest

import workloads


def _fd_source(orc, r, m, Q, eps, lam, mu, h=1e-6):
    def L(r_, m_, Q_):
        phi, a = orc.eval_source(r_, m_, Q_, eps)
        return lam @ a + mu * phi
    g_r = np.array([(L(r + h * e, m, Q) - L(r - h * e, m, Q)) / (2 * h) for e in np.eye(3)])
    g_m = (L(r, m + h, Q) - L(r, m - h, Q)) / (2 * h)
    g_q = None
    if Q is not None:
        g_q = []
        for k in range(6):
            e = np.zeros(6)
            e[k] = h
            g_q.append((L(r, m, Q + e) - L(r, m, Q - e)) / (2 * h))
        g_q = np.array(g_q)
    return g_r, g_m, g_q


@pytest.mark.parametrize("eps", [0.0, 0.25])
@pytest.mark.parametrize("with_q", [False, True])
def test_single_source_vjp_matches_finite_differences(orc, eps, with_q):
    rng = np.random.default_rng(5)
    for _ in range(5):
        r = rng.normal(size=3) * 2
        m = rng.uniform(0.5, 2.0)
        Q = rng.normal(size=6) * 0.3 if with_q else None
        lam = rng.normal(size=3)
        mu = rng.normal()
        g_r, g_m, g_q = orc.eval_source_vjp(r, m, Q, eps, 1.0, lam, mu)
        f_r, f_m, f_q = _fd_source(orc, r, m, Q, eps, lam, mu)
        assert np.allclose(g_r, f_r, rtol=1e-6, atol=1e-9)
        assert g_m == pytest.approx(f_m, rel=1e-6, abs=1e-9)
        if with_q:
            # the VJP returns the gradient with respect to the symmetric matrix:
            # an off-diagonal stored component appears twice in it
            assert np.allclose(g_q * np.array([1, 1, 1, 2, 2, 2]), f_q, rtol=1e-6, atol=1e-9)


@pytest.fixture(scope="module")
def frozen(orc):
    mdl = workloads.plummer(4096, seed=1005)
    t = orc.Tree(mdl.pos, mdl.mass)
    t.freeze_lists(0.4)
    x, m = t.sorted_state()
    rng = np.random.default_rng(1006)
    lam = rng.normal(size=(3, t.n))
    mu = rng.normal(size=t.n)
    return t, x, m, lam, mu


def test_frozen_forces_reproduce_the_tree_forces(frozen):
    t, x, m, lam, mu = frozen
    acc, pot = t.frozen_forces(0.01, 1.0, x, m)
    acc_s, pot_s, _, _, _ = t.forces_sorted(0.4, 0.01, 1.0)
    assert np.array_equal(acc, acc_s) and np.array_equal(pot, pot_s)


def test_frozen_tree_vjp_matches_finite_differences(frozen):
    """N = 4096, FP64, 32 random coordinates (positions and masses)."""
    t, x, m, lam, mu = frozen
    gx, gm = t.frozen_vjp(0.01, 1.0, x, m, lam, mu)

    def L(x_, m_):
        a, p = t.frozen_forces(0.01, 1.0, x_, m_)
        return (lam * a).sum() + (mu * p).sum()

    # central differences with h = 1e-5 (positions are O(1)); an error is
    # measured against max(|fd|, rms gradient) so that FD round-off on tiny
    # components does not count
    rng = np.random.default_rng(1007)
    sx = np.sqrt((gx ** 2).mean())
    sm = np.sqrt((gm ** 2).mean())
    for k in range(24):
        d, i = int(rng.integers(3)), int(rng.integers(t.n))
        h = 1e-5
        xp, xm = x.copy(), x.copy()
        xp[d, i] += h
        xm[d, i] -= h
        fd = (L(xp, m) - L(xm, m)) / (2 * h)
        assert abs(gx[d, i] - fd) <= 1e-6 * max(abs(fd), sx), (d, i, gx[d, i], fd)
    for k in range(8):
        i = int(rng.integers(t.n))
        h = 1e-5 * m[i]
        mp, mm = m.copy(), m.copy()
        mp[i] += h
        mm[i] -= h
        fd = (L(x, mp) - L(x, mm)) / (2 * h)
        assert abs(gm[i] - fd) <= 1e-6 * max(abs(fd), sm), (i, gm[i], fd)


def test_frozen_tree_vjp_is_translation_invariant(frozen):
    """The forces depend on differences only (cells move with their
    particles), so the position gradients sum to zero."""
    t, x, m, lam, mu = frozen
    gx, _ = t.frozen_vjp(0.01, 1.0, x, m, lam, mu)
    assert np.all(np.abs(gx.sum(axis=1)) <= 1e-11 * np.abs(gx).sum(axis=1))


def test_direct_vjp_matches_finite_differences(orc):
    rng = np.random.default_rng(8)
    n = 300
    pos = rng.normal(size=(3, n))
    m = rng.uniform(0.5, 1.5, n) / n
    lam = rng.normal(size=(3, n))
    mu = rng.normal(size=n)
    gx, gm = orc.direct_vjp(pos, m, 0.05, 2.0, lam, mu)

    def L(p_, m_):
        a, ph = orc.direct_forces(p_, m_, 0.05, 2.0)
        return (lam * a).sum() + (mu * ph).sum()

    for k in range(12):
        d, i = int(rng.integers(3)), int(rng.integers(n))
        e = np.zeros((3, n))
        e[d, i] = 1e-6
        assert gx[d, i] == pytest.approx((L(pos + e, m) - L(pos - e, m)) / 2e-6, rel=1e-6)
        em = np.zeros(n)
        em[i] = 1e-6 * m[i]
        assert gm[i] == pytest.approx((L(pos, m + em) - L(pos, m - em)) / (2e-6 * m[i]), rel=1e-6)


def test_tree_vjp_tends_to_direct_vjp(orc):
    """theta -> 0 opens every cell: the frozen tree adjoint is the O1 adjoint."""
    mdl = workloads.plummer(1500, seed=41)
    rng = np.random.default_rng(42)
    lam = rng.normal(size=(3, mdl.n))
    mu = rng.normal(size=mdl.n)
    gd, gmd = orc.direct_vjp(mdl.pos, mdl.mass, 0.01, 1.0, lam, mu)
    t = orc.Tree(mdl.pos, mdl.mass)
    t.freeze_lists(1e-4)
    x, m = t.sorted_state()
    gx, gm = t.frozen_vjp(0.01, 1.0, x, m, t.to_sorted(lam), t.to_sorted(mu))
    gx, gm = t.to_caller(gx), t.to_caller(gm)
    assert np.allclose(gx, gd, rtol=1e-11, atol=1e-12 * np.abs(gd).max())
    assert np.allclose(gm, gmd, rtol=1e-11, atol=1e-12 * np.abs(gmd).max())


def test_kdk_chain_vjp_matches_finite_differences(orc):
    """Four KDK steps with frozen per-step trees: the reverse pass equals the
    derivative of the re-integrated final state."""
    mdl = workloads.plummer(600, seed=51)
    dt = 1.0 / 64
    plan = orc.KdkPlan(mdl.pos, mdl.vel, mdl.mass, 4, dt, theta=0.4, eps=0.01)
    rng = np.random.default_rng(52)
    cx = rng.normal(size=(3, mdl.n))
    cv = rng.normal(size=(3, mdl.n))
    xb, vb, mb = plan.vjp(cx, cv)

    def L(p0, v0, m_):
        p, v = plan.run(p0, v0, m_)
        return (cx * p).sum() + (cv * v).sum()

    p_nom, v_nom = plan.run(mdl.pos, mdl.vel)
    ref = orc.kdk(mdl.pos, mdl.vel, mdl.mass, 4, dt, theta=0.4, eps=0.01)
    assert np.allclose(p_nom, ref[0], rtol=0, atol=1e-13) and np.allclose(v_nom, ref[1], rtol=0, atol=1e-12)
    # normwise: errors against max(|fd|, rms of the gradient)
    sx, sv, sm = (np.sqrt((g ** 2).mean()) for g in (xb, vb, mb))
    h = 1e-6
    for k in range(10):
        d, i = int(rng.integers(3)), int(rng.integers(mdl.n))
        e = np.zeros((3, mdl.n))
        e[d, i] = h
        fx = (L(mdl.pos + e, mdl.vel, mdl.mass) - L(mdl.pos - e, mdl.vel, mdl.mass)) / (2 * h)
        fv = (L(mdl.pos, mdl.vel + e, mdl.mass) - L(mdl.pos, mdl.vel - e, mdl.mass)) / (2 * h)
        assert abs(xb[d, i] - fx) <= 1e-6 * max(abs(fx), sx), (d, i, xb[d, i], fx)
        assert abs(vb[d, i] - fv) <= 1e-6 * max(abs(fv), sv), (d, i, vb[d, i], fv)
    for k in range(4):
        i = int(rng.integers(mdl.n))
        em = np.zeros(mdl.n)
        em[i] = 1e-5 * mdl.mass[i]
        fd = (L(mdl.pos, mdl.vel, mdl.mass + em) - L(mdl.pos, mdl.vel, mdl.mass - em)) / (2 * em[i])
        assert abs(mb[i] - fd) <= 1e-6 * max(abs(fd), sm), (i, mb[i], fd)
