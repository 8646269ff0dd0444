"""Pins for the oracle's leap-frog (Sec. III.B.2 end: second-order leap-frog)
and diagnostics (energy, momentum, angular momentum)."""
import math

import numpy as np


def _kepler(ecc_scale=0.8):
    # two bodies of mass 1/2 at separation 1; circular speed 1/2 each, scaled
    pos = np.array([[-0.5, 0.5], [0.0, 0.0], [0.0, 0.0]])
    vel = np.array([[0.0, 0.0], [-0.5, 0.5], [0.0, 0.0]]) * ecc_scale
    return pos, vel, np.array([0.5, 0.5])


def _energy(orc, pos, vel, m):
    _, pot = orc.direct_forces(pos, m, eps=0.0)
    return orc.diagnostics(pos, vel, m, pot)[2]


def test_kepler_energy_error_is_second_order(orc):
    pos, vel, m = _kepler()
    E0 = _energy(orc, pos, vel, m)
    period = 2 * math.pi * (1.0 / (2.0 - 0.64)) ** 1.5    # a = 1/(2 - v^2) for G M = 1
    errs = []
    for nstep in (200, 400):
        dt = period / nstep
        p, v = pos.copy(), vel.copy()
        worst = 0.0
        for _ in range(nstep // 20):
            p, v, _, _ = orc.kdk(p, v, m, 20, dt, theta=0.4, eps=0.0)
            worst = max(worst, abs(_energy(orc, p, v, m) / E0 - 1))
        errs.append(worst)
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.0, errs
    assert errs[1] < 1e-3


def test_kepler_time_reversible(orc):
    pos, vel, m = _kepler()
    p, v, _, _ = orc.kdk(pos, vel, m, 150, 0.01, theta=0.4, eps=0.0)
    p2, v2, _, _ = orc.kdk(p, -v, m, 150, 0.01, theta=0.4, eps=0.0)
    assert np.allclose(p2, pos, atol=1e-12)
    assert np.allclose(-v2, vel, atol=1e-12)


def test_free_particle_drifts_exactly(orc):
    pos = np.array([[1.0], [2.0], [3.0]])
    vel = np.array([[0.5], [-0.25], [0.125]])
    p, v, acc, pot = orc.kdk(pos, vel, np.array([1.0]), 8, 0.25, theta=0.4, eps=0.1)
    assert np.array_equal(p, pos + 8 * 0.25 * vel)
    assert np.array_equal(v, vel) and np.all(acc == 0) and np.all(pot == 0)


def test_diagnostics_by_hand(orc):
    pos = np.array([[1.0, -1.0], [0.0, 0.0], [0.0, 2.0]])
    vel = np.array([[0.0, 1.0], [2.0, 0.0], [0.0, -1.0]])
    m = np.array([2.0, 3.0])
    pot = np.array([-0.5, -4.0])
    out = orc.diagnostics(pos, vel, m, pot)
    ek = 0.5 * 2 * 4 + 0.5 * 3 * 2
    ep = 0.5 * (2 * -0.5 + 3 * -4.0)
    P = 2 * vel[:, 0] + 3 * vel[:, 1]
    L = 2 * np.cross(pos[:, 0], vel[:, 0]) + 3 * np.cross(pos[:, 1], vel[:, 1])
    assert np.allclose(out, [ek, ep, ek + ep, *P, *L, 5.0], rtol=1e-15, atol=0)


def test_momentum_conserved_by_direct_leapfrog(orc):
    rng = np.random.default_rng(17)
    pos = rng.standard_normal((3, 200))
    vel = rng.standard_normal((3, 200)) * 0.1
    m = rng.uniform(0.5, 1.5, 200) / 200
    p, v, _, _ = orc.kdk(pos, vel, m, 10, 0.01, theta=0.4, eps=0.05, direct=True)
    P0 = (vel * m).sum(1)
    P1 = (v * m).sum(1)
    assert np.allclose(P0, P1, atol=1e-14 * np.abs(vel * m).sum())
