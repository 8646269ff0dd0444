"""Domains and local essential trees (Sec. III.B) on one GPU.

The paper's processes each own a piece of the global Peano-Hilbert order,
build their tree as a branch of the global octree, and send each remote
process the local essential tree (LET) it needs; the receiving process walks
every LET like a local tree.  Here one context stands for one process and
the exchange is the LET's own device arrays.  Every step runs in the CUDA
library (tree_domain_state, tree_build_cube, let_build, let_forces); this
module only orders the calls and, for the emulation, places each domain's
forces back at the global caller indices.
"""
from __future__ import annotations

import torch

from . import capi
from .gravity import TreeGravity


class Let:
    """One local essential tree (owns its device arrays)."""

    def __init__(self, stream=None):
        self.h = capi.let_create(stream)

    def close(self):
        if getattr(self, "h", None):
            capi.let_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build(self, src: TreeGravity, dst: TreeGravity, theta: float) -> "Let":
        capi.let_build(self.h, src.ctx, dst.ctx, theta)
        return self

    def build_boxes(self, src: TreeGravity, box: torch.Tensor, half: torch.Tensor, theta: float) -> "Let":
        """The LET of src's tree for group boxes received from elsewhere."""
        capi.let_build_boxes(self.h, src.ctx, box, half, theta)
        return self

    def pack(self) -> torch.Tensor:
        """The LET as one contiguous uint8 CUDA tensor (the message)."""
        dev = torch.device("cuda", torch.cuda.current_device())
        buf = torch.empty(capi.let_pack(self.h), dtype=torch.uint8, device=dev)
        capi.let_pack(self.h, buf)
        return buf

    def unpack(self, buf: torch.Tensor) -> "Let":
        capi.let_unpack(self.h, buf)
        return self

    def info(self) -> dict:
        return capi.let_get_info(self.h)

    def cells(self):
        """(source cell, kind) of every LET cell; kind 0 used whole, 1 opened
        cell, 2 opened leaf."""
        n = self.info()["cells"]
        dev = torch.device("cuda", torch.cuda.current_device())
        src = torch.empty(n, dtype=torch.int32, device=dev)
        kind = torch.empty(n, dtype=torch.int32, device=dev)
        capi.let_debug_cells(self.h, src, kind)
        return src, kind

    def add_forces(self, dst: TreeGravity, eps: float):
        capi.let_forces(dst.ctx, self.h, eps)


def split(world: TreeGravity, R: int):
    """R domains: equal pieces of the key order of the tree in `world`, each
    a context built in world's cube.  Returns [(context, caller ids)]."""
    cube = world.cube()
    n = world.n
    out = []
    for r in range(R):
        first, last = n * r // R, n * (r + 1) // R
        pos, vel, mass, ids = world.domain_state(first, last - first)
        g = TreeGravity(G=world.G, theta=world.theta, eps=world.eps)
        g.build_cube(pos, mass, cube)
        g.set_velocities(vel)
        out.append((g, ids))
    return out


def domain_forces(domains, theta: float, eps: float):
    """Forces of all particles from the R domains: each domain's own tree
    plus the LETs of all the others.  Returns (acc (3, N) float32, pot (N,)
    in the global caller order, per-pair LET sizes {(src, dst): info})."""
    n = sum(int(ids.numel()) for _, ids in domains)
    dev = domains[0][1].device
    acc = torch.empty((3, n), dtype=torch.float32, device=dev)
    pot = torch.empty(n, dtype=torch.float32, device=dev)
    let = Let()
    sizes = {}
    try:
        for i, (gi, _) in enumerate(domains):
            gi.forces(theta, eps)
            for j, (gj, _) in enumerate(domains):
                if j == i:
                    continue
                let.build(gj, gi, theta)
                let.add_forces(gi, eps)
                sizes[(j, i)] = let.info()
        for gi, ids in domains:
            a, p = gi.last_forces()
            idx = ids.long()
            acc[:, idx] = a
            pot[idx] = p
    finally:
        let.close()
    return acc, pot, sizes
