"""Thin ctypes binding of the C ABI declared in include/bonsai_gb.h.

Every function here only marshals arguments: torch CUDA tensors become
device pointers, the current torch stream becomes the context's stream, and
non-zero status codes become :class:`BonsaiError`.  All computation happens
in the CUDA library; if the library is missing the first call raises
immediately (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbonsai_gb.so")

_lock = threading.Lock()
_lib = None

BONSAI_OK = 0
BONSAI_EINVAL = -1
BONSAI_ENOMEM = -2
BONSAI_EOVERFLOW = -3
BONSAI_ECUDA = -4
BONSAI_ESTATE = -5
BONSAI_EIO = -6
BONSAI_ETIMEOUT = -7

# every symbol include/bonsai_gb.h declares
EXPORTED = (
    "bonsai_create", "bonsai_destroy", "bonsai_set_stream", "tree_build", "tree_forces",
    "tree_set_velocities", "tree_step", "tree_get_state", "tree_get_forces",
    "bonsai_diagnostics", "tree_get_stats", "tree_solve_host", "tree_debug_cube",
    "tree_debug_keys", "tree_debug_nodes", "tree_debug_multipoles", "tree_debug_groups",
    "bonsai_strerror", "bonsai_sfc_order_noalloc", "tree_forces_vjp", "tree_run", "tree_run_vjp",
    "tree_debug_set_frontier_capacity", "tree_forces_fp64", "tree_direct_forces",
    "tree_save_snapshot", "tree_load_snapshot", "tree_surface_density",
    "tree_build_cube", "tree_domain_state", "let_create", "let_destroy", "let_build", "let_get_info",
    "let_debug_cells", "let_forces", "bonsai_galaxy_sec4", "bonsai_galaxy_generate",
    "bonsai_galaxy_tables", "tree_debug_lists", "bonsai_set_wait_timeout", "tree_debug_hold_stream",
    "tree_get_group_boxes", "let_build_boxes", "let_pack", "let_unpack", "bonsai_cube_from_bounds",
    "tree_bounds",
)

BONSAI_NOALLOC_MAX_N = 1 << 20
BONSAI_ICS_K = 4096
BONSAI_ICS_V = 256
BONSAI_ICS_KD = 4096
BONSAI_ICS_NRAD_OUT = 15
BONSAI_ICS_NDISK_OUT = 7


class BonsaiError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class bonsai_params(ctypes.Structure):
    _fields_ = [("G", ctypes.c_double), ("theta", ctypes.c_float), ("eps", ctypes.c_float),
                ("nleaf", ctypes.c_int32), ("ncrit", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class bonsai_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_nodes", ctypes.c_int64), ("n_groups", ctypes.c_int64),
                ("depth", ctypes.c_int32), ("max_frontier", ctypes.c_int32),
                ("n_pp", ctypes.c_uint64), ("n_pc", ctypes.c_uint64), ("flops", ctypes.c_double),
                ("ms_keys", ctypes.c_float), ("ms_tree", ctypes.c_float),
                ("ms_force", ctypes.c_float), ("ms_integrate", ctypes.c_float),
                ("ms_walk", ctypes.c_float), ("launches", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class bonsai_galaxy(ctypes.Structure):
    _fields_ = [("n_halo", ctypes.c_int64), ("n_disk", ctypes.c_int64), ("n_bulge", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("G", ctypes.c_double),
                ("M_halo", ctypes.c_double), ("a_halo", ctypes.c_double),
                ("M_bulge", ctypes.c_double), ("a_bulge", ctypes.c_double),
                ("r_t", ctypes.c_double), ("dr_t", ctypes.c_double),
                ("M_disk", ctypes.c_double), ("R_d", ctypes.c_double), ("z0", ctypes.c_double),
                ("R_max", ctypes.c_double), ("Q", ctypes.c_double), ("R_Q", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def load(path: str | None = None):
    """Load the CUDA library (build it first with ``paper_1412_0659_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} is missing "
                               "(run paper_1412_0659_gb300.build.build())")
        lib = ctypes.CDLL(p)
        P, i32, i64, f32, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_double
        sig = {
            "bonsai_create": (i32, [ctypes.POINTER(P), ctypes.POINTER(bonsai_params), P]),
            "bonsai_destroy": (None, [P]),
            "bonsai_set_stream": (i32, [P, P]),
            "tree_build": (i32, [P, P, P, i64]),
            "tree_forces": (i32, [P, f32, f32, P, P]),
            "tree_set_velocities": (i32, [P, P]),
            "tree_step": (i32, [P, f64]),
            "tree_get_state": (i32, [P, P, P, P]),
            "tree_get_forces": (i32, [P, P, P]),
            "bonsai_diagnostics": (i32, [P, P]),
            "tree_get_stats": (i32, [P, ctypes.POINTER(bonsai_stats)]),
            "tree_solve_host": (i32, [P, P, P, i64, f32, f32, P, P]),
            "tree_debug_cube": (i32, [P, P, P]),
            "tree_debug_keys": (i32, [P, P, P]),
            "tree_debug_nodes": (i32, [P, P, P, P, P, P]),
            "tree_debug_multipoles": (i32, [P, P, P, P]),
            "tree_debug_groups": (i32, [P, P, P, P, P]),
            "tree_debug_lists": (i32, [P, P, P, P, P]),
            "bonsai_set_wait_timeout": (i32, [f64]),
            "tree_get_group_boxes": (i32, [P, P, P, ctypes.POINTER(i64)]),
            "let_build_boxes": (i32, [P, P, P, P, i64, f32]),
            "let_pack": (i32, [P, P, i64, ctypes.POINTER(i64)]),
            "let_unpack": (i32, [P, P, i64]),
            "bonsai_cube_from_bounds": (i32, [ctypes.POINTER(f64), ctypes.POINTER(f64), ctypes.POINTER(f64)]),
            "tree_bounds": (i32, [P, P, P, i64, ctypes.POINTER(f64), ctypes.POINTER(f64)]),
            "tree_debug_hold_stream": (i32, [P, f64]),
            "bonsai_strerror": (ctypes.c_char_p, [i32]),
            "bonsai_sfc_order_noalloc": (i32, [P, P, i64, P, P, P, P]),
            "tree_forces_vjp": (i32, [P, P, P, P, P]),
            "tree_run": (i32, [P, i32, f64, i32]),
            "tree_run_vjp": (i32, [P, P, P, P, P, P, P]),
            "tree_debug_set_frontier_capacity": (i32, [P, i32]),
            "tree_direct_forces": (i32, [P, P, i64, f32, P, P]),
            "tree_save_snapshot": (i32, [P, ctypes.c_char_p, f64]),
            "tree_build_cube": (i32, [P, P, P, i64, ctypes.POINTER(f64)]),
            "tree_domain_state": (i32, [P, i64, i64, P, P, P, P]),
            "let_create": (i32, [ctypes.POINTER(P), P]),
            "let_destroy": (None, [P]),
            "let_build": (i32, [P, P, P, f32]),
            "let_get_info": (i32, [P, ctypes.POINTER(i64)]),
            "let_debug_cells": (i32, [P, P, P]),
            "let_forces": (i32, [P, P, f32]),
            "tree_load_snapshot": (i32, [P, ctypes.c_char_p, ctypes.POINTER(f64)]),
            "tree_surface_density": (i32, [P, i64, i64, ctypes.POINTER(f64), i32, i32, P]),
            "tree_forces_fp64": (i32, [P, f32, f32, P, P]),
            "bonsai_galaxy_sec4": (i32, [ctypes.POINTER(bonsai_galaxy), i64, ctypes.c_uint64]),
            "bonsai_galaxy_generate": (i32, [ctypes.POINTER(bonsai_galaxy), P, P, P, P]),
            "bonsai_galaxy_tables": (i32, [ctypes.POINTER(bonsai_galaxy), P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load().bonsai_strerror(code).decode()
    except RuntimeError:
        return f"status {code}"


def _check(rc: int, where: str):
    if rc != BONSAI_OK:
        raise BonsaiError(rc, where)


def _ptr(t, dtype=None, numel=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    import torch
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    """Host pointer of a contiguous numpy array or CPU tensor."""
    if a is None:
        return None
    if hasattr(a, "ctypes"):
        return ctypes.c_void_p(a.ctypes.data)
    if a.is_cuda or not a.is_contiguous():
        raise ValueError("host buffer must be a contiguous CPU array")
    return ctypes.c_void_p(a.data_ptr())


def _stream_handle(stream=None) -> ctypes.c_void_p:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
# same-name wrappers of the C ABI
# ---------------------------------------------------------------------------

def bonsai_create(G: float = 1.0, theta: float = 0.4, eps: float = 0.01, nleaf: int = 16,
                  ncrit: int = 64, stream=None) -> ctypes.c_void_p:
    lib = load()
    prm = bonsai_params(G, theta, eps, nleaf, ncrit)
    h = ctypes.c_void_p()
    _check(lib.bonsai_create(ctypes.byref(h), ctypes.byref(prm), _stream_handle(stream)), "bonsai_create")
    return h


def bonsai_destroy(ctx) -> None:
    if ctx:
        load().bonsai_destroy(ctx)


def bonsai_set_stream(ctx, stream=None) -> None:
    _check(load().bonsai_set_stream(ctx, _stream_handle(stream)), "bonsai_set_stream")


def tree_build(ctx, pos, mass) -> None:
    import torch
    n = mass.numel()
    _check(load().tree_build(ctx, _ptr(pos, torch.float64, 3 * n, "pos"),
                             _ptr(mass, torch.float64, n, "mass"), n), "tree_build")


def tree_forces(ctx, theta: float, eps: float, acc=None, pot=None) -> None:
    import torch
    _check(load().tree_forces(ctx, float(theta), float(eps), _ptr(acc, torch.float32, None, "acc"),
                              _ptr(pot, torch.float32, None, "pot")), "tree_forces")


def tree_forces_fp64(ctx, theta: float, eps: float, acc=None, pot=None) -> None:
    import torch
    _check(load().tree_forces_fp64(ctx, float(theta), float(eps), _ptr(acc, torch.float64, None, "acc"),
                                   _ptr(pot, torch.float64, None, "pot")), "tree_forces_fp64")


def tree_direct_forces(ctx, targets, nt: int, eps: float, acc=None, pot=None) -> None:
    import torch
    _check(load().tree_direct_forces(ctx, _ptr(targets, torch.int64, nt, "targets"), int(nt), float(eps),
                                     _ptr(acc, torch.float64, 3 * nt, "acc"),
                                     _ptr(pot, torch.float64, nt, "pot")), "tree_direct_forces")


def tree_build_cube(ctx, pos, mass, cube) -> None:
    import torch
    n = int(mass.numel())
    c = (ctypes.c_double * 4)(*[float(x) for x in cube])
    _check(load().tree_build_cube(ctx, _ptr(pos, torch.float64, 3 * n, "pos"), _ptr(mass, torch.float64, n, "mass"),
                                  n, c), "tree_build_cube")


def tree_domain_state(ctx, first: int, count: int, pos=None, vel=None, mass=None, caller_id=None) -> None:
    import torch
    _check(load().tree_domain_state(ctx, int(first), int(count), _ptr(pos, torch.float64, 3 * count, "pos"),
                                    _ptr(vel, torch.float64, 3 * count, "vel"),
                                    _ptr(mass, torch.float64, count, "mass"),
                                    _ptr(caller_id, torch.int32, count, "caller_id")), "tree_domain_state")


def let_create(stream=None):
    h = ctypes.c_void_p()
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(load().let_create(ctypes.byref(h), s), "let_create")
    return h


def let_destroy(let) -> None:
    load().let_destroy(let)


def let_build(let, src, dst, theta: float) -> None:
    _check(load().let_build(let, src, dst, float(theta)), "let_build")


def let_get_info(let) -> dict:
    out = (ctypes.c_int64 * 4)()
    _check(load().let_get_info(let, out), "let_get_info")
    return {"cells": out[0], "particles": out[1], "bytes": out[2], "source_cells": out[3]}


def let_debug_cells(let, src_node=None, kind=None) -> None:
    import torch
    _check(load().let_debug_cells(let, _ptr(src_node, torch.int32, None, "src_node"),
                                  _ptr(kind, torch.int32, None, "kind")), "let_debug_cells")


def tree_get_group_boxes(ctx, box=None, half=None) -> int:
    """The group boxes (float32 CUDA tensors (ng, 4) each, or None); returns ng."""
    import torch
    ng = ctypes.c_int64()
    _check(load().tree_get_group_boxes(ctx, _ptr(box, torch.float32, None, "box"),
                                       _ptr(half, torch.float32, None, "half"), ctypes.byref(ng)),
           "tree_get_group_boxes")
    return ng.value


def let_build_boxes(let, src, box, half, theta: float) -> None:
    import torch
    ng = int(box.shape[0])
    if tuple(box.shape) != (ng, 4) or tuple(half.shape) != (ng, 4):
        raise ValueError("box and half must be (ngroups, 4)")
    if ng == 0:
        box = half = None
        bp = hp = ctypes.c_void_p(16)  # never read with no groups
    else:
        bp, hp = _ptr(box, torch.float32, 4 * ng, "box"), _ptr(half, torch.float32, 4 * ng, "half")
    _check(load().let_build_boxes(let, src, bp, hp, ng, float(theta)), "let_build_boxes")


def let_pack(let, buf=None) -> int:
    """Packed size in bytes; with buf (uint8 CUDA tensor) also the packed LET."""
    import torch
    nb = ctypes.c_int64()
    cap = 0 if buf is None else int(buf.numel())
    _check(load().let_pack(let, _ptr(buf, torch.uint8, None, "buf"), cap, ctypes.byref(nb)), "let_pack")
    return nb.value


def let_unpack(let, buf) -> None:
    import torch
    _check(load().let_unpack(let, _ptr(buf, torch.uint8, None, "buf"), int(buf.numel())), "let_unpack")


def bonsai_cube_from_bounds(mn, mx) -> list:
    a = (ctypes.c_double * 3)(*[float(v) for v in mn])
    b = (ctypes.c_double * 3)(*[float(v) for v in mx])
    out = (ctypes.c_double * 4)()
    _check(load().bonsai_cube_from_bounds(a, b, out), "bonsai_cube_from_bounds")
    return list(out)


def tree_bounds(ctx, pos, mass):
    """(mn[3], mx[3]) of device positions (3, n) float64 with masses (n,)."""
    import torch
    n = int(mass.numel())
    mn = (ctypes.c_double * 3)()
    mx = (ctypes.c_double * 3)()
    _check(load().tree_bounds(ctx, _ptr(pos, torch.float64, 3 * n, "pos"), _ptr(mass, torch.float64, n, "mass"),
                              n, mn, mx), "tree_bounds")
    return list(mn), list(mx)


def let_forces(dst, let, eps: float) -> None:
    _check(load().let_forces(dst, let, float(eps)), "let_forces")


def tree_save_snapshot(ctx, path: str, time: float = 0.0) -> None:
    _check(load().tree_save_snapshot(ctx, os.fsencode(path), float(time)), "tree_save_snapshot")


def tree_load_snapshot(ctx, path: str) -> float:
    t = ctypes.c_double()
    _check(load().tree_load_snapshot(ctx, os.fsencode(path), ctypes.byref(t)), "tree_load_snapshot")
    return t.value


def tree_surface_density(ctx, first: int, count: int, window, nx: int, ny: int, out) -> None:
    import torch
    w = (ctypes.c_double * 4)(*[float(x) for x in window])
    _check(load().tree_surface_density(ctx, int(first), int(count), w, int(nx), int(ny),
                                       _ptr(out, torch.float64, nx * ny, "map")), "tree_surface_density")


def tree_set_velocities(ctx, vel) -> None:
    import torch
    _check(load().tree_set_velocities(ctx, _ptr(vel, torch.float64, None, "vel")), "tree_set_velocities")


def tree_step(ctx, dt: float) -> None:
    _check(load().tree_step(ctx, float(dt)), "tree_step")


def tree_get_state(ctx, pos=None, vel=None, mass=None) -> None:
    import torch
    _check(load().tree_get_state(ctx, _ptr(pos, torch.float64), _ptr(vel, torch.float64),
                                 _ptr(mass, torch.float64)), "tree_get_state")


def tree_get_forces(ctx, acc=None, pot=None) -> None:
    import torch
    _check(load().tree_get_forces(ctx, _ptr(acc, torch.float32), _ptr(pot, torch.float32)),
           "tree_get_forces")


def bonsai_diagnostics(ctx):
    out = (ctypes.c_double * 10)()
    _check(load().bonsai_diagnostics(ctx, out), "bonsai_diagnostics")
    return list(out)


def tree_get_stats(ctx) -> dict:
    st = bonsai_stats()
    _check(load().tree_get_stats(ctx, ctypes.byref(st)), "tree_get_stats")
    return st.as_dict()


def tree_solve_host(ctx, pos, mass, theta: float, eps: float, acc, pot) -> None:
    """Host-buffer entry: pos (3, n) / mass (n,) float64 and acc (3, n) / pot (n,)
    float32 are host arrays (numpy or CPU tensors, ideally pinned)."""
    n = int(mass.shape[0])
    _check(load().tree_solve_host(ctx, _hptr(pos), _hptr(mass), n, float(theta), float(eps),
                                  _hptr(acc), _hptr(pot)), "tree_solve_host")


def tree_forces_vjp(ctx, gacc, gpos, gmass, gpot=None) -> None:
    import torch
    _check(load().tree_forces_vjp(ctx, _ptr(gacc, torch.float32, None, "gacc"),
                                  _ptr(gpot, torch.float32, None, "gpot"),
                                  _ptr(gpos, torch.float64, None, "gpos"),
                                  _ptr(gmass, torch.float64, None, "gmass")), "tree_forces_vjp")


def tree_run(ctx, nsteps: int, dt: float, ckpt_every: int) -> None:
    _check(load().tree_run(ctx, int(nsteps), float(dt), int(ckpt_every)), "tree_run")


def tree_run_vjp(ctx, xbar, vbar, mbar, xbar0, vbar0, mbar0) -> None:
    import torch
    f64 = torch.float64
    _check(load().tree_run_vjp(ctx, _ptr(xbar, f64), _ptr(vbar, f64), _ptr(mbar, f64),
                               _ptr(xbar0, f64), _ptr(vbar0, f64), _ptr(mbar0, f64)), "tree_run_vjp")


def tree_debug_set_frontier_capacity(ctx, cap: int) -> None:
    _check(load().tree_debug_set_frontier_capacity(ctx, int(cap)), "tree_debug_set_frontier_capacity")


def tree_debug_cube(ctx):
    lo = (ctypes.c_double * 3)()
    L = ctypes.c_double()
    _check(load().tree_debug_cube(ctx, lo, ctypes.byref(L)), "tree_debug_cube")
    return list(lo), L.value


def tree_debug_keys(ctx, keys=None, perm=None) -> None:
    _check(load().tree_debug_keys(ctx, _ptr(keys), _ptr(perm)), "tree_debug_keys")


def tree_debug_nodes(ctx, first=None, count=None, child=None, nchild=None, level=None) -> None:
    _check(load().tree_debug_nodes(ctx, _ptr(first), _ptr(count), _ptr(child), _ptr(nchild),
                                   _ptr(level)), "tree_debug_nodes")


def tree_debug_multipoles(ctx, M=None, com=None, Q=None) -> None:
    _check(load().tree_debug_multipoles(ctx, _ptr(M), _ptr(com), _ptr(Q)), "tree_debug_multipoles")


def tree_debug_groups(ctx, first=None, count=None, npp=None, npc=None) -> None:
    _check(load().tree_debug_groups(ctx, _ptr(first), _ptr(count), _ptr(npp), _ptr(npc)),
           "tree_debug_groups")


def tree_debug_lists(ctx, pc_off, pp_off, pc_cells, pp_sources) -> None:
    """Each group's accepted cells and p-p sources at the given offsets
    (int64 CUDA tensors [n_groups + 1]; outputs int32 CUDA tensors)."""
    _check(load().tree_debug_lists(ctx, _ptr(pc_off), _ptr(pp_off), _ptr(pc_cells), _ptr(pp_sources)),
           "tree_debug_lists")


def bonsai_set_wait_timeout(seconds: float) -> None:
    """Limit of every host wait on the device (seconds, process-wide)."""
    _check(load().bonsai_set_wait_timeout(float(seconds)), "bonsai_set_wait_timeout")


def tree_debug_hold_stream(ctx, seconds: float) -> None:
    """Queue a host-side sleep on the context's stream (test hook)."""
    _check(load().tree_debug_hold_stream(ctx, float(seconds)), "tree_debug_hold_stream")


def bonsai_strerror(code: int) -> str:
    return strerror(code)


def bonsai_sfc_order_noalloc(pos, mass, keys, perm, stream=None):
    """Sorted Peano-Hilbert keys and order of pos/mass written into the
    caller's keys (int64/uint64 CUDA tensor, n) and perm (int32 CUDA tensor,
    n) without any device allocation; returns the cube (lo_x, lo_y, lo_z, L).
    n is limited to BONSAI_NOALLOC_MAX_N."""
    import torch
    n = int(mass.numel())
    if n > BONSAI_NOALLOC_MAX_N:
        raise ValueError(f"bonsai_sfc_order_noalloc: n = {n} exceeds the fixed scratch limit "
                         f"{BONSAI_NOALLOC_MAX_N}")
    cube = (ctypes.c_double * 4)()
    _check(load().bonsai_sfc_order_noalloc(_ptr(pos, torch.float64, 3 * n, "pos"),
                                           _ptr(mass, torch.float64, n, "mass"), n,
                                           _ptr(keys, None, n, "keys"), _ptr(perm, None, n, "perm"),
                                           cube, _stream_handle(stream)), "bonsai_sfc_order_noalloc")
    return list(cube)


def bonsai_galaxy_sec4(n: int, seed: int) -> bonsai_galaxy:
    """The Sec. IV Milky Way model for n particles (host struct)."""
    g = bonsai_galaxy()
    _check(load().bonsai_galaxy_sec4(ctypes.byref(g), int(n), int(seed)), "bonsai_galaxy_sec4")
    return g


def bonsai_galaxy_generate(g: bonsai_galaxy, pos, vel, mass, stream=None) -> None:
    """Sample the model into pos, vel (float64 CUDA tensors, 3 x n) and mass (n)."""
    import torch
    n = int(g.n_halo + g.n_disk + g.n_bulge)
    _check(load().bonsai_galaxy_generate(ctypes.byref(g), _ptr(pos, torch.float64, 3 * n, "pos"),
                                         _ptr(vel, torch.float64, 3 * n, "vel"),
                                         _ptr(mass, torch.float64, n, "mass"),
                                         _stream_handle(stream)), "bonsai_galaxy_generate")


def bonsai_galaxy_tables(g: bonsai_galaxy, radial, vcdf, disk, stream=None) -> None:
    """The generator's tables into float64 CUDA tensors: radial (15 x K),
    vcdf (2 x K x V or None), disk (7 x KD)."""
    import torch
    _check(load().bonsai_galaxy_tables(
        ctypes.byref(g), _ptr(radial, torch.float64, BONSAI_ICS_NRAD_OUT * BONSAI_ICS_K, "radial"),
        _ptr(vcdf, torch.float64, 2 * BONSAI_ICS_K * BONSAI_ICS_V, "vcdf"),
        _ptr(disk, torch.float64, BONSAI_ICS_NDISK_OUT * BONSAI_ICS_KD, "disk"),
        _stream_handle(stream)), "bonsai_galaxy_tables")
