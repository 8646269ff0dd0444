"""FP64 CPU oracle for the Bonsai tree-force path (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never imports, links
or executes anything here, and the two share no code.

The arithmetic lives in ``bonsai_oracle.c`` (plain C, FP64, no fused
multiply-add); this module compiles it with gcc on first use and marshals
numpy arrays through ctypes.  Arrays of positions and velocities are SoA
``(3, N)`` float64; masses ``(N,)`` float64.

Pins (tests/test_oracle_*.py): Hilbert bijection/adjacency/prefix on small
grids, octree invariants and a brute-force recursive octree, parallel-axis
multipoles against direct per-node sums, quadrupole truncation-error slope,
Plummer closed forms, Newton's third law, two- and three-body cases by hand,
theta -> 0 convergence of the tree to direct summation, Kepler energy and
time reversibility of the leap-frog, and the Table 2 flop arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bonsai_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NLEAF = 16
NCRIT = 64


def build(force: bool = False) -> str:
    """Compile bonsai_oracle.c into liboracle.so next to it (gcc, OpenMP).

    -ffp-contract=off keeps every multiply and add separately rounded on
    both x86-64 and aarch64 (gcc fuses them by default on aarch64)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, f32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_double
        sig = {
            "orc_hilbert_key": (ctypes.c_uint64, [ctypes.c_uint32] * 3 + [i32]),
            "orc_bounding_cube": (None, [i64, P, P, P, P, P]),
            "orc_tree_build": (P, [i64, P, P, i32, i32]),
            "orc_tree_build_cube": (P, [i64, P, P, i32, i32, P, f64]),
            "orc_let_mark": (i32, [P, P, f32, P, P]),
            "orc_cross_forces": (i32, [P, P, f32, f64, f64, P, P, P, P, P]),
            "orc_tree_free": (None, [P]),
            "orc_tree_num_nodes": (i64, [P]),
            "orc_tree_num_groups": (i64, [P]),
            "orc_tree_cube": (None, [P, P, P]),
            "orc_tree_keys": (None, [P, P, P]),
            "orc_tree_nodes": (None, [P, P, P, P, P, P]),
            "orc_tree_multipoles": (None, [P, P, P, P, P, P]),
            "orc_tree_groups": (None, [P, P, P, P, P]),
            "orc_tree_sorted_state": (None, [P, P, P]),
            "orc_cell_mac": (None, [P, f32, P, P]),
            "orc_group_box_f32": (None, [P, P, P]),
            "orc_tree_forces": (i32, [P, f32, f64, f64, i64, i64, P, P, P, P, P]),
            "orc_tree_forces_list": (i32, [P, f32, f64, f64, i64, P, P, P, P, P, P]),
            "orc_direct_forces": (None, [i64, P, P, f64, f64, i64, P, P, P]),
            "orc_forces": (i32, [i64, P, P, i32, i32, f32, f64, f64, i32, P, P, P]),
            "orc_kdk": (i32, [i64, P, P, P, i32, f64, i32, i32, f32, f64, f64, i32, P, P, i32]),
            "orc_diagnostics": (None, [i64, P, P, P, P, P]),
            "orc_surface_density": (None, [i64, P, P, i64, i64, P, ctypes.c_int, ctypes.c_int, P]),
            "orc_num_threads": (i32, []),
            "orc_eval_source": (None, [P, f64, P, f64, f64, P, P]),
            "orc_group_lists": (i32, [P, f32, i64, P, P, i64, P]),
            "orc_eval_source_vjp": (None, [P, f64, P, f64, f64, P, f64, P, P, P]),
            "orc_tree_freeze_lists": (i32, [P, f32]),
            "orc_tree_frozen_forces": (i32, [P, f64, f64, P, P, P, P]),
            "orc_tree_frozen_vjp": (i32, [P, f64, f64, P, P, P, P, P, P]),
            "orc_direct_vjp": (None, [i64, P, P, f64, f64, P, P, P, P]),
            "orc_kdk_plan_build": (P, [i64, P, P, P, i32, f64, f32, f64, f64, i32, i32]),
            "orc_kdk_plan_free": (None, [P]),
            "orc_kdk_plan_run": (i32, [P, P, P, P, P, P]),
            "orc_kdk_plan_vjp": (i32, [P, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def num_threads() -> int:
    return int(_load().orc_num_threads())


def hilbert_key(q0: int, q1: int, q2: int, bits: int = 21) -> int:
    """Peano-Hilbert index of integer cell (q0, q1, q2) on a 2^bits grid."""
    return int(_load().orc_hilbert_key(q0, q1, q2, bits))


def bounding_cube(pos: np.ndarray):
    pos = _f64(pos)
    n = pos.shape[1]
    lo = np.zeros(3)
    L = np.zeros(1)
    _load().orc_bounding_cube(n, _p(pos[0]), _p(pos[1]), _p(pos[2]), _p(lo), _p(L))
    return lo, float(L[0])


class Tree:
    """Steps 1-6 of the tree method (keys, sort, octree, groups, multipoles)
    built from caller-order positions ``(3, N)`` and masses ``(N,)``."""

    def __init__(self, pos: np.ndarray, mass: np.ndarray, nleaf: int = NLEAF, ncrit: int = NCRIT,
                 cube=None):
        """cube = (lo (3,), L): build in that cube (a branch of a global
        octree) instead of the particles' own bounding cube."""
        self._lib = _load()
        self.pos = _f64(pos)
        self.n = self.pos.shape[1]
        self.mass = _f64(mass, (self.n,))
        self.nleaf, self.ncrit = nleaf, ncrit
        if cube is None:
            h = self._lib.orc_tree_build(self.n, _p(self.pos), _p(self.mass), nleaf, ncrit)
        else:
            lo = np.ascontiguousarray(cube[0], dtype=np.float64)
            h = self._lib.orc_tree_build_cube(self.n, _p(self.pos), _p(self.mass), nleaf, ncrit, _p(lo),
                                              float(cube[1]))
        if not h:
            raise MemoryError("oracle tree build failed")
        self._h = ctypes.c_void_p(h)
        self.nnodes = int(self._lib.orc_tree_num_nodes(self._h))
        self.ngroups = int(self._lib.orc_tree_num_groups(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and self._lib is not None:
            self._lib.orc_tree_free(h)
            self._h = None

    def let_mark(self, dst: "Tree", theta: float):
        """(visited, opened) flags of this tree's cells for the walks of
        dst's groups (the local essential tree this tree sends to dst)."""
        v = np.zeros(self.nnodes, np.uint8)
        o = np.zeros(self.nnodes, np.uint8)
        if self._lib.orc_let_mark(self._h, dst._h, float(theta), _p(v), _p(o)):
            raise MemoryError("let mark failed")
        return v.astype(bool), o.astype(bool)

    def cross_forces(self, dst: "Tree", theta: float, eps: float, G: float = 1.0):
        """Forces of this tree's particles on dst's particles through dst's
        group walks over this tree: (acc (3, n_dst), pot (n_dst,)) in dst's
        caller order, per-group (n_pp, n_pc) of dst's groups, total counts."""
        acc = np.zeros((3, dst.n))
        pot = np.zeros(dst.n)
        g_npp = np.zeros(dst.ngroups, np.int64)
        g_npc = np.zeros(dst.ngroups, np.int64)
        counts = np.zeros(2, np.uint64)
        if self._lib.orc_cross_forces(self._h, dst._h, float(theta), float(eps), float(G), _p(acc), _p(pot),
                                      _p(g_npp), _p(g_npc), _p(counts)):
            raise MemoryError("cross forces failed")
        return dst.to_caller(acc), dst.to_caller(pot), g_npp, g_npc, (int(counts[0]), int(counts[1]))

    def cube(self):
        lo = np.zeros(3)
        L = np.zeros(1)
        self._lib.orc_tree_cube(self._h, _p(lo), _p(L))
        return lo, float(L[0])

    def keys(self):
        key = np.zeros(self.n, np.uint64)
        perm = np.zeros(self.n, np.uint32)
        self._lib.orc_tree_keys(self._h, _p(key), _p(perm))
        return key, perm

    def nodes(self) -> dict:
        out = {k: np.zeros(self.nnodes, np.uint32) for k in ("first", "count", "child", "nchild", "level")}
        self._lib.orc_tree_nodes(self._h, *[_p(out[k]) for k in ("first", "count", "child", "nchild", "level")])
        return out

    def multipoles(self) -> dict:
        nn = self.nnodes
        out = {"M": np.zeros(nn), "com": np.zeros((3, nn)), "Q": np.zeros((6, nn)),
               "centre": np.zeros((3, nn)), "side": np.zeros(nn)}
        self._lib.orc_tree_multipoles(self._h, *[_p(out[k]) for k in ("M", "com", "Q", "centre", "side")])
        return out

    def groups(self) -> dict:
        ng = self.ngroups
        out = {"first": np.zeros(ng, np.uint32), "count": np.zeros(ng, np.uint32),
               "centre": np.zeros((3, ng)), "half": np.zeros((3, ng))}
        self._lib.orc_tree_groups(self._h, *[_p(out[k]) for k in ("first", "count", "centre", "half")])
        return out

    def sorted_state(self):
        pos = np.zeros((3, self.n))
        m = np.zeros(self.n)
        self._lib.orc_tree_sorted_state(self._h, _p(pos), _p(m))
        return pos, m

    def cell_mac(self, theta: float):
        com_f = np.zeros((3, self.nnodes), np.float32)
        r2 = np.zeros(self.nnodes, np.float32)
        self._lib.orc_cell_mac(self._h, float(theta), _p(com_f), _p(r2))
        return com_f, r2

    def group_box_f32(self):
        c = np.zeros((3, self.ngroups), np.float32)
        h = np.zeros((3, self.ngroups), np.float32)
        self._lib.orc_group_box_f32(self._h, _p(c), _p(h))
        return c, h

    def group_lists(self, theta: float, g: int):
        """(accepted cells, opened leaves) of group g, in walk order."""
        cap = self.nnodes
        pc = np.zeros(cap, np.uint32)
        lv = np.zeros(cap, np.uint32)
        nout = np.zeros(2, np.int64)
        if self._lib.orc_group_lists(self._h, float(theta), int(g), _p(pc), _p(lv), cap, _p(nout)):
            raise IndexError(g)
        return pc[: nout[0]].copy(), lv[: nout[1]].copy()

    def forces_sorted(self, theta: float, eps: float, G: float = 1.0, g0: int = 0, g1: int | None = None):
        """FP64 tree forces for groups [g0, g1) in sorted order.

        Returns (acc (3,N), pot (N,), g_npp, g_npc, (n_pp, n_pc)); entries of
        particles outside the chosen groups are NaN."""
        g1 = self.ngroups if g1 is None else g1
        acc = np.full((3, self.n), np.nan)
        pot = np.full(self.n, np.nan)
        g_npp = np.zeros(self.ngroups, np.int64)
        g_npc = np.zeros(self.ngroups, np.int64)
        counts = np.zeros(2, np.uint64)
        rc = self._lib.orc_tree_forces(self._h, float(theta), float(eps), float(G), int(g0), int(g1),
                                       _p(acc), _p(pot), _p(g_npp), _p(g_npc), _p(counts))
        if rc:
            raise MemoryError("oracle forces failed")
        return acc, pot, g_npp, g_npc, (int(counts[0]), int(counts[1]))

    # -- adjoint with frozen lists (sorted order unless stated) -------------
    def freeze_lists(self, theta: float):
        """Record every group's interaction lists at this opening angle."""
        if self._lib.orc_tree_freeze_lists(self._h, float(theta)):
            raise MemoryError("freeze_lists failed")
        self._frozen = float(theta)

    def to_sorted(self, a):
        _, perm = self.keys()
        a = np.asarray(a, np.float64)
        return np.ascontiguousarray(a[..., perm])

    def to_caller(self, a):
        _, perm = self.keys()
        out = np.empty_like(a)
        out[..., perm] = a
        return out

    def frozen_forces(self, eps: float, G: float, pos_sorted, mass_sorted):
        x = _f64(pos_sorted, (3, self.n))
        m = _f64(mass_sorted, (self.n,))
        acc = np.zeros((3, self.n))
        pot = np.zeros(self.n)
        if self._lib.orc_tree_frozen_forces(self._h, float(eps), float(G), _p(x), _p(m), _p(acc), _p(pot)):
            raise RuntimeError("frozen_forces: call freeze_lists first")
        return acc, pot

    def frozen_vjp(self, eps: float, G: float, pos_sorted, mass_sorted, lam_sorted, mu_sorted=None):
        x = _f64(pos_sorted, (3, self.n))
        m = _f64(mass_sorted, (self.n,))
        lam = _f64(lam_sorted, (3, self.n))
        mu = None if mu_sorted is None else _f64(mu_sorted, (self.n,))
        gx = np.zeros((3, self.n))
        gm = np.zeros(self.n)
        if self._lib.orc_tree_frozen_vjp(self._h, float(eps), float(G), _p(x), _p(m), _p(lam), _p(mu),
                                         _p(gx), _p(gm)):
            raise RuntimeError("frozen_vjp: call freeze_lists first")
        return gx, gm

    def forces_groups(self, theta: float, eps: float, G: float, groups):
        """FP64 tree forces for the listed groups (sorted order, NaN elsewhere);
        returns (acc, pot, g_npp, g_npc, (n_pp, n_pc)) like forces_sorted."""
        gl = np.ascontiguousarray(groups, np.int64)
        acc = np.full((3, self.n), np.nan)
        pot = np.full(self.n, np.nan)
        g_npp = np.zeros(self.ngroups, np.int64)
        g_npc = np.zeros(self.ngroups, np.int64)
        counts = np.zeros(2, np.uint64)
        rc = self._lib.orc_tree_forces_list(self._h, float(theta), float(eps), float(G), gl.shape[0],
                                            _p(gl), _p(acc), _p(pot), _p(g_npp), _p(g_npc), _p(counts))
        if rc:
            raise ValueError("oracle forces failed (bad group index or out of memory)")
        return acc, pot, g_npp, g_npc, (int(counts[0]), int(counts[1]))

    def forces(self, theta: float, eps: float, G: float = 1.0):
        """FP64 tree forces for all particles in caller order, plus counts."""
        acc_s, pot_s, _, _, counts = self.forces_sorted(theta, eps, G)
        _, perm = self.keys()
        acc = np.empty_like(acc_s)
        pot = np.empty_like(pot_s)
        acc[:, perm] = acc_s
        pot[perm] = pot_s
        return acc, pot, counts


def eval_source(r, m: float, Q=None, eps: float = 0.0, G: float = 1.0):
    """Eq. 1-2 for one source at offset r (source minus target) with mass m and
    optional quadrupole Q = (xx, yy, zz, xy, xz, yz).  Returns (phi, a)."""
    r = _f64(r, (3,))
    Qa = None if Q is None else _f64(Q, (6,))
    phi = np.zeros(1)
    a = np.zeros(3)
    _load().orc_eval_source(_p(r), float(m), _p(Qa), float(eps), float(G), _p(phi), _p(a))
    return float(phi[0]), a


def eval_source_vjp(r, m: float, Q=None, eps: float = 0.0, G: float = 1.0, lam=(0, 0, 0), mu: float = 0.0):
    """Gradient of lam.a + mu phi for one source w.r.t. (r, m, Q)."""
    r = _f64(r, (3,))
    Qa = None if Q is None else _f64(Q, (6,))
    lam = _f64(lam, (3,))
    gr = np.zeros(3)
    gm = np.zeros(1)
    gq = np.zeros(6)
    _load().orc_eval_source_vjp(_p(r), float(m), _p(Qa), float(eps), float(G), _p(lam), float(mu),
                                _p(gr), _p(gm), _p(gq))
    return gr, float(gm[0]), gq


def direct_vjp(pos, mass, eps: float, G: float, lam, mu=None):
    """O1 adjoint: gradient of sum lam.a + mu phi of direct summation."""
    pos = _f64(pos)
    n = pos.shape[1]
    mass = _f64(mass, (n,))
    lam = _f64(lam, (3, n))
    mu = None if mu is None else _f64(mu, (n,))
    gx = np.zeros((3, n))
    gm = np.zeros(n)
    _load().orc_direct_vjp(n, _p(pos), _p(mass), float(eps), float(G), _p(lam), _p(mu), _p(gx), _p(gm))
    return gx, gm


class KdkPlan:
    """K kick-drift-kick steps with each step's tree and lists frozen at the
    nominal trajectory; run() re-integrates from perturbed initial data with
    those frozen structures, vjp() is the exact reverse of run()."""

    def __init__(self, pos0, vel0, mass, nsteps: int, dt: float, theta: float, eps: float,
                 G: float = 1.0, nleaf: int = NLEAF, ncrit: int = NCRIT):
        self._lib = _load()
        pos0 = _f64(pos0)
        self.n = pos0.shape[1]
        vel0 = _f64(vel0, (3, self.n))
        self.mass = _f64(mass, (self.n,))
        h = self._lib.orc_kdk_plan_build(self.n, _p(pos0), _p(vel0), _p(self.mass), int(nsteps), float(dt),
                                         float(theta), float(eps), float(G), nleaf, ncrit)
        if not h:
            raise MemoryError("kdk plan failed")
        self._h = ctypes.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None:
            self._lib.orc_kdk_plan_free(h)
            self._h = None

    def run(self, pos0, vel0, mass=None):
        mass = self.mass if mass is None else _f64(mass, (self.n,))
        pos0 = _f64(pos0, (3, self.n))
        vel0 = _f64(vel0, (3, self.n))
        pos = np.zeros((3, self.n))
        vel = np.zeros((3, self.n))
        if self._lib.orc_kdk_plan_run(self._h, _p(pos0), _p(vel0), _p(mass), _p(pos), _p(vel)):
            raise MemoryError("kdk run failed")
        return pos, vel

    def vjp(self, xbar, vbar, mbar=None):
        xb = _f64(xbar, (3, self.n)).copy()
        vb = _f64(vbar, (3, self.n)).copy()
        mb = np.zeros(self.n) if mbar is None else _f64(mbar, (self.n,)).copy()
        if self._lib.orc_kdk_plan_vjp(self._h, _p(self.mass), _p(xb), _p(vb), _p(mb)):
            raise MemoryError("kdk vjp failed")
        return xb, vb, mb


def direct_forces(pos, mass, eps: float, G: float = 1.0, targets=None):
    """O1: FP64 direct summation for the given caller indices (all if None).

    Returns acc (3, nt), pot (nt,)."""
    pos = _f64(pos)
    n = pos.shape[1]
    mass = _f64(mass, (n,))
    if targets is None:
        nt, tp = n, None
    else:
        targets = np.ascontiguousarray(targets, np.int64)
        nt, tp = targets.shape[0], targets
    acc = np.zeros((3, nt))
    pot = np.zeros(nt)
    _load().orc_direct_forces(n, _p(pos), _p(mass), float(eps), float(G), nt, _p(tp), _p(acc), _p(pot))
    return acc, pot


def forces(pos, mass, theta: float, eps: float, G: float = 1.0, direct: bool = False,
           nleaf: int = NLEAF, ncrit: int = NCRIT):
    pos = _f64(pos)
    n = pos.shape[1]
    mass = _f64(mass, (n,))
    acc = np.zeros((3, n))
    pot = np.zeros(n)
    counts = np.zeros(2, np.uint64)
    rc = _load().orc_forces(n, _p(pos), _p(mass), nleaf, ncrit, float(theta), float(eps), float(G),
                            int(direct), _p(acc), _p(pot), _p(counts))
    if rc:
        raise MemoryError("oracle forces failed")
    return acc, pot, (int(counts[0]), int(counts[1]))


def kdk(pos, vel, mass, nsteps: int, dt: float, theta: float, eps: float, G: float = 1.0,
        direct: bool = False, nleaf: int = NLEAF, ncrit: int = NCRIT):
    """Kick-drift-kick leap-frog for nsteps; returns (pos, vel, acc, pot)."""
    pos = _f64(pos).copy()
    n = pos.shape[1]
    vel = _f64(vel, (3, n)).copy()
    mass = _f64(mass, (n,))
    acc = np.zeros((3, n))
    pot = np.zeros(n)
    rc = _load().orc_kdk(n, _p(pos), _p(vel), _p(mass), int(nsteps), float(dt), nleaf, ncrit,
                         float(theta), float(eps), float(G), int(direct), _p(acc), _p(pot), 0)
    if rc:
        raise MemoryError("oracle kdk failed")
    return pos, vel, acc, pot


def surface_density(pos, mass, first: int, count: int, window, nx: int, ny: int):
    """Face-on cloud-in-cell surface density of particles [first, first +
    count) over window = (xmin, xmax, ymin, ymax); returns (ny, nx)."""
    pos = _f64(pos)
    n = pos.shape[1]
    mass = _f64(mass, (n,))
    w = np.ascontiguousarray(window, dtype=np.float64)
    out = np.zeros((ny, nx))
    _load().orc_surface_density(n, _p(pos), _p(mass), int(first), int(count), _p(w), int(nx), int(ny),
                                _p(out))
    return out


def diagnostics(pos, vel, mass, pot):
    """{E_kin, E_pot, E_tot, Px, Py, Pz, Lx, Ly, Lz, M_tot} in FP64."""
    pos = _f64(pos)
    n = pos.shape[1]
    vel = _f64(vel, (3, n))
    mass = _f64(mass, (n,))
    pot = _f64(pot, (n,))
    out = np.zeros(10)
    _load().orc_diagnostics(n, _p(pos), _p(vel), _p(mass), _p(pot), _p(out))
    return out
