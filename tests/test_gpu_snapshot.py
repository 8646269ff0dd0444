"""Snapshots and the on-the-fly surface density, through the C ABI.

A run saved, reloaded into a fresh context and continued is bit-identical
to the uninterrupted run (the tree order is a pure function of the keys
and caller indices, so the rebuilt tree, lists and forces are the same);
the file holds exactly the documented layout; bad files are reported; the
face-on surface density equals the oracle's, also at the 2^23 size."""
import struct

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _gravity(m):
    from gpu_helpers import DEV
    from paper_1412_0659_gb300 import TreeGravity
    g = TreeGravity(G=m.G, theta=m.theta, eps=m.eps)
    g.build(torch.from_numpy(m.pos).to(DEV), torch.from_numpy(m.mass).to(DEV))
    g.set_velocities(torch.from_numpy(m.vel).to(DEV))
    return g


def _coincident():
    m = workloads.plummer(3000, seed=44)
    pos, vel = m.pos.copy(), m.vel.copy()
    pos[:, 100:160] = pos[:, 7:8]   # 61 particles at one point, moving together
    vel[:, 100:160] = vel[:, 7:8]
    return workloads.Model(pos, vel, m.mass, m.G, 0.01, 0.4, 1.0 / 64, "coincident", {})


CASES = {
    "plummer16384": lambda: workloads.config_model(0),
    "milkyway30000": lambda: workloads.milky_way(30000, seed=77),
    "coincident3000": _coincident,
}


@pytest.mark.parametrize("name", list(CASES))
def test_restart_reproduces_the_uninterrupted_run_bit_for_bit(name, tmp_path):
    from paper_1412_0659_gb300 import TreeGravity
    m = CASES[name]()
    path = str(tmp_path / "snap.bin")
    a = _gravity(m)
    for _ in range(4):
        a.step(m.dt)
    a.save(path, time=4 * m.dt)
    for _ in range(4):
        a.step(m.dt)
    pa, va, ma = a.state()
    a.close()
    b = TreeGravity(G=m.G, theta=m.theta, eps=m.eps)
    t = b.load(path)
    assert t == 4 * m.dt
    for _ in range(4):
        b.step(m.dt)
    pb, vb, mb = b.state()
    b.close()
    assert torch.equal(pa, pb) and torch.equal(va, vb) and torch.equal(ma, mb)


def test_snapshot_file_layout(tmp_path):
    m = workloads.milky_way(5000, seed=3)
    g = _gravity(m)
    g.step(m.dt)
    path = tmp_path / "s.bin"
    g.save(str(path), time=1.25)
    pos, vel, mass = [x.cpu().numpy() for x in g.state()]
    g.close()
    raw = path.read_bytes()
    assert len(raw) == 64 + 7 * 8 * m.n
    magic, version, flags, n, time, G, theta, eps = struct.unpack("<8sIIqddff", raw[:48])
    assert (magic, version, flags, n, time) == (b"BONSAIGB", 1, 0, m.n, 1.25)
    assert G == m.G and theta == np.float32(m.theta) and eps == np.float32(m.eps)
    body = np.frombuffer(raw[64:], dtype="<f8")
    assert np.array_equal(body[:3 * m.n].reshape(3, m.n), pos)
    assert np.array_equal(body[3 * m.n:6 * m.n].reshape(3, m.n), vel)
    assert np.array_equal(body[6 * m.n:], mass)


def test_bad_snapshots_are_reported(tmp_path):
    from paper_1412_0659_gb300 import TreeGravity, capi
    m = workloads.plummer(2000, seed=9)
    g = _gravity(m)
    good = tmp_path / "good.bin"
    g.save(str(good))
    g.close()
    raw = good.read_bytes()
    (tmp_path / "short.bin").write_bytes(raw[:-8])
    (tmp_path / "magic.bin").write_bytes(b"NOTBONSA" + raw[8:])
    body = np.frombuffer(raw[64:], dtype="<f8").copy()
    body[5] = np.nan
    (tmp_path / "nan.bin").write_bytes(raw[:64] + body.tobytes())
    h = TreeGravity()
    for name, code in (("missing.bin", capi.BONSAI_EIO), ("short.bin", capi.BONSAI_EIO),
                       ("magic.bin", capi.BONSAI_EIO), ("nan.bin", capi.BONSAI_EINVAL)):
        with pytest.raises(capi.BonsaiError) as e:
            h.load(str(tmp_path / name))
        assert e.value.code == code, name
    assert h.load(str(good)) == 0.0  # usable afterwards
    h.close()


def test_surface_density_matches_oracle():
    from paper_1412_0659_gb300 import capi
    m = workloads.milky_way(30000, seed=77)
    g = _gravity(m)
    s0, nd = m.components["disk"]
    _, nb = m.components["bulge"]
    window = (-15.0, 15.0, -12.0, 12.0)
    got = g.surface_density(s0, nd + nb, window, 96, 80).cpu().numpy()
    want = oracle.surface_density(m.pos, m.mass, s0, nd + nb, window, 96, 80)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * want.max())
    for bad in ((1.0, 1.0, 0.0, 1.0), (0.0, float("nan"), 0.0, 1.0)):
        with pytest.raises(capi.BonsaiError) as e:
            g.surface_density(0, 10, bad, 4, 4)
        assert e.value.code == capi.BONSAI_EINVAL
    with pytest.raises(capi.BonsaiError) as e:
        g.surface_density(m.n - 5, 10, window, 4, 4)
    assert e.value.code == capi.BONSAI_EINVAL
    g.close()


def test_surface_density_fullsize():
    """The 2^23 benchmark model after one step: disk and bulge, 512 x 512
    pixels over 30 x 30 kpc."""
    m = workloads.config_model(1)
    g = _gravity(m)
    g.step(m.dt)
    pos, _, mass = [x.cpu().numpy() for x in g.state()]
    s0, nd = m.components["disk"]
    _, nb = m.components["bulge"]
    window = (-15.0, 15.0, -15.0, 15.0)
    got = g.surface_density(s0, nd + nb, window, 512, 512).cpu().numpy()
    g.close()
    want = oracle.surface_density(pos, mass, s0, nd + nb, window, 512, 512)
    assert np.allclose(got, want, rtol=1e-11, atol=1e-12 * want.max())
