"""Local essential trees exchanged between processes (Sec. III.B.2), one
process per GPU, over torch.distributed.

Each process holds one domain, a piece of the global Peano-Hilbert order
(Sec. III.B.1).  One force evaluation:

1. The global cube.  Every process reduces its particles' bounds with the
   library's bounding-box kernels (tree_bounds); an all-reduce of the
   minima and maxima gives all processes the same bounds and
   bonsai_cube_from_bounds the same cube, in which each builds its tree
   (tree_build_cube): the trees are branches of one global octree.
2. The boundary exchange.  Every process sends all others the boxes of its
   walk groups (an all-gather of variable size; the paper all-gathers
   boundary structures for the same purpose).
3. The LETs.  For every other process, each builds the part of its tree
   that the other's groups need (let_build_boxes), packs it into one
   buffer (let_pack) and sends it point to point.  Each received LET is
   unpacked into local device memory (let_unpack) and walked like a local
   tree (let_forces), in source-rank order, so the result does not depend
   on arrival times.

With NCCL the messages are device buffers; with gloo they pass through
host memory.  Remote data is always copied into this GPU's memory before
it is read: no peer access and no multicast.  Every step on the particles
and trees runs in the CUDA library; this module only moves bytes and
orders the calls.  How the particles are distributed over the processes
(the paper's sampling decomposition and particle exchange) is the
caller's: each process passes its own domain.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import capi
from .domains import Let
from .gravity import TreeGravity


def comm_device(group=None) -> torch.device:
    """Where messages live: the current GPU for NCCL, host memory otherwise."""
    if dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def all_reduce_bounds(mn, mx, group=None):
    """Componentwise minimum of mn and maximum of mx over all processes
    (one MIN all-reduce of (mn, -mx), exact)."""
    t = torch.tensor([*mn, *[-v for v in mx]], dtype=torch.float64, device=comm_device(group))
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    v = t.cpu().tolist()
    return v[:3], [-x for x in v[3:]]


def all_gather_var(t: torch.Tensor, group=None) -> list:
    """All-gather of a 1-D uint8 tensor whose length differs between
    processes; returns every process's tensor, in rank order."""
    dev = comm_device(group)
    world = dist.get_world_size(group)
    n = torch.tensor([t.numel()], dtype=torch.int64, device=dev)
    sizes = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(x.item()) for x in sizes]
    cap = max(1, max(sizes))
    pad = torch.zeros(cap, dtype=torch.uint8, device=dev)
    pad[: t.numel()] = t.to(dev)
    out = [torch.empty(cap, dtype=torch.uint8, device=dev) for _ in range(world)]
    dist.all_gather(out, pad, group=group)
    return [o[:s] for o, s in zip(out, sizes)]


def exchange_var(send: dict, group=None) -> dict:
    """Point-to-point messages of any length: send[d] (1-D uint8 tensor) goes
    to process d; returns {s: the message from s} for every other process.
    The lengths are all-gathered first, then every send and receive is
    posted at once."""
    dev = comm_device(group)
    world = dist.get_world_size(group)
    me = dist.get_rank(group)
    row = torch.tensor([send[d].numel() if d in send else 0 for d in range(world)], dtype=torch.int64,
                       device=dev)
    rows = [torch.zeros(world, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(rows, row, group=group)
    incoming = {s: int(rows[s][me].item()) for s in range(world) if s != me}
    ops, recv = [], {}
    for s, nbytes in incoming.items():
        recv[s] = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        if nbytes:
            ops.append(dist.P2POp(dist.irecv, recv[s], s, group=group))
    for d, msg in send.items():
        if d != me and msg.numel():
            ops.append(dist.P2POp(dist.isend, msg.to(dev).contiguous(), d, group=group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    return recv


def global_cube(g: TreeGravity, pos: torch.Tensor, mass: torch.Tensor, group=None) -> list:
    """The cube of the union of all processes' particles."""
    mn, mx = capi.tree_bounds(g.ctx, pos, mass)
    mn, mx = all_reduce_bounds(mn, mx, group)
    return capi.bonsai_cube_from_bounds(mn, mx)


def build_domain(pos: torch.Tensor, vel: torch.Tensor | None, mass: torch.Tensor, G: float, theta: float,
                 eps: float, group=None) -> TreeGravity:
    """This process's domain as a context whose tree is a branch of the
    global octree."""
    g = TreeGravity(G=G, theta=theta, eps=eps)
    g.build_cube(pos, mass, global_cube(g, pos, mass, group))
    if vel is not None:
        g.set_velocities(vel)
    return g


def _boxes_bytes(g: TreeGravity) -> torch.Tensor:
    dev = torch.device("cuda", torch.cuda.current_device())
    ng = capi.tree_get_group_boxes(g.ctx)
    bh = torch.empty((2, max(ng, 1), 4), dtype=torch.float32, device=dev)
    if ng:
        capi.tree_get_group_boxes(g.ctx, bh[0], bh[1])
    return bh[:, :ng].contiguous().view(torch.uint8).reshape(-1)


def distributed_forces(g: TreeGravity, theta: float, eps: float, group=None):
    """Forces on this domain's particles from all domains: its own tree plus
    the LET of every other process.  Returns (acc (3, n), pot (n,)) in the
    order this process passed its particles, and per-source LET sizes."""
    dev = torch.device("cuda", torch.cuda.current_device())
    world = dist.get_world_size(group)
    me = dist.get_rank(group)
    g.forces(theta, eps)
    boxes = all_gather_var(_boxes_bytes(g), group)
    let = Let()
    sizes = {}
    try:
        send = {}
        for d in range(world):
            if d == me:
                continue
            bh = boxes[d].to(dev).view(torch.float32).reshape(2, -1, 4)
            let.build_boxes(g, bh[0].contiguous(), bh[1].contiguous(), theta)
            send[d] = let.pack() if let.info()["cells"] else torch.empty(0, dtype=torch.uint8, device=dev)
        recv = exchange_var(send, group)
        for s in sorted(recv):
            if recv[s].numel() == 0:
                continue
            buf = recv[s].to(dev).contiguous()
            let.unpack(buf)
            let.add_forces(g, eps)
            sizes[s] = let.info()
    finally:
        let.close()
    acc, pot = g.last_forces()
    return acc, pot, sizes
