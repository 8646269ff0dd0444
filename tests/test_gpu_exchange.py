"""Local essential trees exchanged between processes (Sec. III.B.2): two
processes, each holding one domain (an equal piece of the global
Peano-Hilbert order), agree on the global cube through an all-reduce of
their bounds, all-gather their group boxes, and send each other packed
LETs, which each unpacks and walks.  Their forces must equal those of the
single-process emulation (domains.domain_forces) for the same domains.
The processes share this machine's one GPU and talk through gloo; no
kernel of one waits on the other's."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import workloads

pytestmark = pytest.mark.gpu

G_MW = 4.498502151469554e-12


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _model():
    return workloads.milky_way(30000, seed=77)


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    from paper_1412_0659_gb300 import TreeGravity, exchange
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = _model()
        dev = torch.device("cuda", 0)
        # this process's domain: its piece of the key order of the whole model
        with TreeGravity(G=G_MW, theta=0.4, eps=0.01) as w:
            w.build(torch.from_numpy(m.pos).to(dev), torch.from_numpy(m.mass).to(dev))
            w.set_velocities(torch.from_numpy(m.vel).to(dev))
            cube_w = w.cube()
            first, last = m.n * rank // world, m.n * (rank + 1) // world
            pos, vel, mass, ids = w.domain_state(first, last - first)
        g = exchange.build_domain(pos, vel, mass, G_MW, 0.4, 0.01)
        acc, pot, sizes = exchange.distributed_forces(g, 0.4, 0.01)
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), acc=acc.cpu().numpy(), pot=pot.cpu().numpy(),
                 ids=ids.cpu().numpy().astype(np.int64), cube=np.array(g.cube()), cube_w=np.array(cube_w),
                 let_cells=np.array([sizes[s]["cells"] for s in sorted(sizes)]))
        g.close()
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_exchanged_lets_give_the_single_process_forces(tmp_path, world):
    from gpu_helpers import DEV
    from paper_1412_0659_gb300 import TreeGravity, domains
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    m = _model()
    with TreeGravity(G=G_MW, theta=0.4, eps=0.01) as w:
        w.build(torch.from_numpy(m.pos).to(DEV), torch.from_numpy(m.mass).to(DEV))
        w.set_velocities(torch.from_numpy(m.vel).to(DEV))
        doms = domains.split(w, world)
        acc_ref, pot_ref, _ = domains.domain_forces(doms, 0.4, 0.01)
        for gi, _ in doms:
            gi.close()
    acc_ref, pot_ref = acc_ref.cpu().numpy(), pot_ref.cpu().numpy()
    seen = np.zeros(m.n, bool)
    for r in range(world):
        d = np.load(tmp_path / f"r{r}.npz")
        assert np.array_equal(d["cube"], d["cube_w"])  # the cube of the whole model, bit for bit
        assert np.all(d["let_cells"] > 0)
        ids = d["ids"]
        seen[ids] = True
        # the same lists in the same order: the same FP32 sums
        assert np.array_equal(d["acc"], acc_ref[:, ids]), r
        assert np.array_equal(d["pot"], pot_ref[ids]), r
    assert seen.all()
