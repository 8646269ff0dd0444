"""Object wrapper over the C ABI: one context, torch tensors in and out.

    g = TreeGravity(G=1.0, theta=0.4, eps=0.01)
    g.build(pos, mass)            # pos (3, N) float64 CUDA, mass (N,) float64 CUDA
    acc, pot = g.forces()         # (3, N) / (N,) float32, caller order
    g.set_velocities(vel)
    g.step(dt)                    # kick-drift-kick, FP64 state on the device
    pos, vel, mass = g.state()

Only marshalling happens here; every step runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import capi


class TreeGravity:
    def __init__(self, G: float = 1.0, theta: float = 0.4, eps: float = 0.01, stream=None):
        self.G, self.theta, self.eps = float(G), float(theta), float(eps)
        self.ctx = capi.bonsai_create(G=G, theta=theta, eps=eps, stream=stream)
        self.n = 0

    def close(self):
        if getattr(self, "ctx", None):
            capi.bonsai_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream=None):
        capi.bonsai_set_stream(self.ctx, stream)

    # -- the path ---------------------------------------------------------
    def build(self, pos: torch.Tensor, mass: torch.Tensor):
        capi.tree_build(self.ctx, pos, mass)
        self.n = int(mass.numel())
        return self

    def build_cube(self, pos: torch.Tensor, mass: torch.Tensor, cube):
        """Build with the keys taken in cube = (lo_x, lo_y, lo_z, L): the tree
        is then a branch of the octree of that cube."""
        capi.tree_build_cube(self.ctx, pos, mass, cube)
        self.n = int(mass.numel())
        return self

    def cube(self):
        """(lo_x, lo_y, lo_z, L) of the current tree."""
        lo, L = capi.tree_debug_cube(self.ctx)
        return (lo[0], lo[1], lo[2], L)

    def domain_state(self, first: int, count: int):
        """pos, vel (3, count), mass (count,) float64 and caller ids (count,)
        int32 of key-order slots [first, first + count)."""
        dev = torch.device("cuda", torch.cuda.current_device())
        pos = torch.empty((3, count), dtype=torch.float64, device=dev)
        vel = torch.empty((3, count), dtype=torch.float64, device=dev)
        mass = torch.empty(count, dtype=torch.float64, device=dev)
        ids = torch.empty(count, dtype=torch.int32, device=dev)
        capi.tree_domain_state(self.ctx, first, count, pos, vel, mass, ids)
        return pos, vel, mass, ids

    def forces(self, theta: float | None = None, eps: float | None = None, acc=None, pot=None):
        theta = self.theta if theta is None else theta
        eps = self.eps if eps is None else eps
        dev = torch.device("cuda", torch.cuda.current_device())
        if acc is None:
            acc = torch.empty((3, self.n), dtype=torch.float32, device=dev)
        if pot is None:
            pot = torch.empty(self.n, dtype=torch.float32, device=dev)
        capi.tree_forces(self.ctx, theta, eps, acc, pot)
        return acc, pot

    def forces_fp64(self, theta: float | None = None, eps: float | None = None):
        """All-FP64 evaluation of the same lists; (3, N) / (N,) float64."""
        theta = self.theta if theta is None else theta
        eps = self.eps if eps is None else eps
        dev = torch.device("cuda", torch.cuda.current_device())
        acc = torch.empty((3, self.n), dtype=torch.float64, device=dev)
        pot = torch.empty(self.n, dtype=torch.float64, device=dev)
        capi.tree_forces_fp64(self.ctx, theta, eps, acc, pot)
        return acc, pot

    def direct_forces(self, targets: torch.Tensor | None = None, eps: float | None = None):
        """Direct summation over all particles of the current tree for the
        given caller indices (all if None); (3, nt) / (nt,) float64."""
        eps = self.eps if eps is None else eps
        dev = torch.device("cuda", torch.cuda.current_device())
        nt = self.n if targets is None else int(targets.numel())
        if targets is not None:
            targets = targets.to(device=dev, dtype=torch.int64).contiguous()
        acc = torch.empty((3, nt), dtype=torch.float64, device=dev)
        pot = torch.empty(nt, dtype=torch.float64, device=dev)
        capi.tree_direct_forces(self.ctx, targets, nt, eps, acc, pot)
        return acc, pot

    def save(self, path: str, time: float = 0.0):
        """Write the FP64 state (caller order) to a snapshot file."""
        capi.tree_save_snapshot(self.ctx, path, time)

    def load(self, path: str) -> float:
        """Read a snapshot into this context (tree built, velocities set);
        returns its stored time."""
        t = capi.tree_load_snapshot(self.ctx, path)
        self.n = self.stats()["n"]
        return t

    def surface_density(self, first: int, count: int, window, nx: int, ny: int) -> torch.Tensor:
        """Face-on cloud-in-cell surface density of caller indices
        [first, first + count) over window = (xmin, xmax, ymin, ymax);
        (ny, nx) float64."""
        dev = torch.device("cuda", torch.cuda.current_device())
        out = torch.empty((ny, nx), dtype=torch.float64, device=dev)
        capi.tree_surface_density(self.ctx, first, count, window, nx, ny, out)
        return out

    def set_velocities(self, vel: torch.Tensor):
        capi.tree_set_velocities(self.ctx, vel)

    def step(self, dt: float):
        capi.tree_step(self.ctx, dt)

    def state(self):
        dev = torch.device("cuda", torch.cuda.current_device())
        pos = torch.empty((3, self.n), dtype=torch.float64, device=dev)
        vel = torch.empty((3, self.n), dtype=torch.float64, device=dev)
        mass = torch.empty(self.n, dtype=torch.float64, device=dev)
        capi.tree_get_state(self.ctx, pos, vel, mass)
        return pos, vel, mass

    def last_forces(self):
        dev = torch.device("cuda", torch.cuda.current_device())
        acc = torch.empty((3, self.n), dtype=torch.float32, device=dev)
        pot = torch.empty(self.n, dtype=torch.float32, device=dev)
        capi.tree_get_forces(self.ctx, acc, pot)
        return acc, pot

    def diagnostics(self) -> dict:
        v = capi.bonsai_diagnostics(self.ctx)
        keys = ("E_kin", "E_pot", "E_tot", "Px", "Py", "Pz", "Lx", "Ly", "Lz", "M")
        return dict(zip(keys, v))

    def stats(self) -> dict:
        return capi.tree_get_stats(self.ctx)

    def solve_host(self, pos, mass, acc, pot, theta: float | None = None, eps: float | None = None):
        theta = self.theta if theta is None else theta
        eps = self.eps if eps is None else eps
        capi.tree_solve_host(self.ctx, pos, mass, theta, eps, acc, pot)
        self.n = int(mass.shape[0])

    # -- adjoint -----------------------------------------------------------
    def forces_vjp(self, gacc: torch.Tensor, gpot: torch.Tensor | None = None):
        """(dL/dx, dL/dm) for L = sum gacc.a + gpot.phi of the last forces()."""
        dev = torch.device("cuda", torch.cuda.current_device())
        gpos = torch.empty((3, self.n), dtype=torch.float64, device=dev)
        gmass = torch.empty(self.n, dtype=torch.float64, device=dev)
        capi.tree_forces_vjp(self.ctx, gacc.contiguous(), gpos, gmass,
                             None if gpot is None else gpot.contiguous())
        return gpos, gmass

    def run(self, nsteps: int, dt: float, ckpt_every: int = 8):
        capi.tree_run(self.ctx, nsteps, dt, ckpt_every)

    def run_vjp(self, xbar: torch.Tensor, vbar: torch.Tensor, mbar: torch.Tensor | None = None):
        dev = torch.device("cuda", torch.cuda.current_device())
        out = [torch.empty((3, self.n), dtype=torch.float64, device=dev) for _ in range(2)]
        mb = torch.empty(self.n, dtype=torch.float64, device=dev)
        capi.tree_run_vjp(self.ctx, xbar.contiguous(), vbar.contiguous(),
                          None if mbar is None else mbar.contiguous(), out[0], out[1], mb)
        return out[0], out[1], mb

    # -- internal views (key-sorted order) -------------------------------
    def debug(self) -> dict:
        st = self.stats()
        n, nn, ng = st["n"], st["n_nodes"], st["n_groups"]
        dev = torch.device("cuda", torch.cuda.current_device())
        u64 = torch.empty(n, dtype=torch.int64, device=dev)
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        capi.tree_debug_keys(self.ctx, u64, perm)
        nodes = {k: torch.empty(nn, dtype=torch.int32, device=dev)
                 for k in ("first", "count", "child", "nchild", "level")}
        capi.tree_debug_nodes(self.ctx, *[nodes[k] for k in ("first", "count", "child", "nchild", "level")])
        M = torch.empty(nn, dtype=torch.float64, device=dev)
        com = torch.empty((3, nn), dtype=torch.float64, device=dev)
        Q = torch.empty((6, nn), dtype=torch.float64, device=dev)
        capi.tree_debug_multipoles(self.ctx, M, com, Q)
        gf = torch.empty(ng, dtype=torch.int32, device=dev)
        gc = torch.empty(ng, dtype=torch.int32, device=dev)
        capi.tree_debug_groups(self.ctx, gf, gc)
        lo, L = capi.tree_debug_cube(self.ctx)
        return {"keys": u64, "perm": perm, "nodes": nodes, "M": M, "com": com, "Q": Q,
                "group_first": gf, "group_count": gc, "lo": lo, "L": L}

    def group_lists(self):
        st = self.stats()
        dev = torch.device("cuda", torch.cuda.current_device())
        npp = torch.empty(st["n_groups"], dtype=torch.int32, device=dev)
        npc = torch.empty(st["n_groups"], dtype=torch.int32, device=dev)
        capi.tree_debug_groups(self.ctx, None, None, npp, npc)
        return npp, npc

    def group_list_members(self):
        """(pc_off, pc_cells, pp_off, pp_sources): every group's accepted
        cells (node indices) and p-p sources (key-sorted particle indices)
        from the last forces, group g at [off[g], off[g + 1])."""
        npp, npc = self.group_lists()
        dev = npp.device
        pc_off = torch.zeros(npc.numel() + 1, dtype=torch.int64, device=dev)
        pp_off = torch.zeros(npp.numel() + 1, dtype=torch.int64, device=dev)
        torch.cumsum(npc.to(torch.int64), 0, out=pc_off[1:])
        torch.cumsum(npp.to(torch.int64), 0, out=pp_off[1:])
        npc_tot, npp_tot = int(pc_off[-1].item()), int(pp_off[-1].item())
        pc = torch.empty(max(1, npc_tot), dtype=torch.int32, device=dev)  # never a null pointer
        pp = torch.empty(max(1, npp_tot), dtype=torch.int32, device=dev)
        capi.tree_debug_lists(self.ctx, pc_off, pp_off, pc, pp)
        return pc_off, pc[:npc_tot], pp_off, pp[:npp_tot]
