"""The message layer of the local-essential-tree exchange between processes
(Sec. III.B.2), on CPU gloo ranks (world sizes 2 and 4): the bounds
all-reduce that gives every process the global cube, the variable-length
all-gather of group boxes, and the point-to-point LET messages of any
length (empty ones included).  The cube itself comes from the library's
host function and must equal the oracle's bounding cube of all particles."""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _payload(src: int, dst: int) -> bytes:
    """The seeded message from src to dst: lengths 0 .. ~3000, one empty."""
    rng = np.random.default_rng(1000 * src + dst)
    n = 0 if (src + dst) % 3 == 0 else int(rng.integers(1, 3000))
    return rng.integers(0, 256, n, dtype=np.uint8).tobytes()


def _positions(rank: int) -> np.ndarray:
    return np.random.default_rng(77 + rank).normal(rank, 1.0 + rank, (3, 500))


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    from paper_1412_0659_gb300 import capi, exchange
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _positions(rank)
        mn, mx = exchange.all_reduce_bounds(p.min(axis=1).tolist(), p.max(axis=1).tolist())
        cube = capi.bonsai_cube_from_bounds(mn, mx)
        mine = torch.frombuffer(bytearray(_payload(rank, rank)), dtype=torch.uint8) \
            if _payload(rank, rank) else torch.empty(0, dtype=torch.uint8)
        gathered = [bytes(t.numpy().tobytes()) for t in exchange.all_gather_var(mine)]
        send = {}
        for d in range(world):
            if d != rank:
                b = _payload(rank, d)
                send[d] = torch.frombuffer(bytearray(b), dtype=torch.uint8) if b else torch.empty(0, dtype=torch.uint8)
        recv = exchange.exchange_var(send)
        got = {s: bytes(t.numpy().tobytes()) == _payload(s, rank) for s, t in recv.items()}
        dist.barrier()
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"mn": mn, "mx": mx, "cube": cube,
                       "gathered_ok": [g == _payload(s, s) for s, g in enumerate(gathered)],
                       "recv_ok": got, "recv_from": sorted(recv)}, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_bounds_boxes_and_let_messages_between_gloo_ranks(tmp_path, world):
    import oracle
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    allp = np.concatenate([_positions(r) for r in range(world)], axis=1)
    lo, L = oracle.bounding_cube(allp)
    for r in range(world):
        with open(tmp_path / f"r{r}.json") as f:
            got = json.load(f)
        assert got["mn"] == allp.min(axis=1).tolist() and got["mx"] == allp.max(axis=1).tolist()
        assert got["cube"] == [*lo.tolist(), L]       # bit for bit the oracle's cube of all particles
        assert all(got["gathered_ok"]) and len(got["gathered_ok"]) == world
        assert got["recv_from"] == [s for s in range(world) if s != r]
        assert all(got["recv_ok"].values())


def test_cube_from_bounds_matches_the_oracle_and_rejects_bad_bounds():
    import oracle
    from paper_1412_0659_gb300 import capi
    rng = np.random.default_rng(5)
    for scale in (1e-3, 1.0, 3e4):
        p = rng.normal(0, scale, (3, 1000)) + rng.normal(0, 10 * scale, (3, 1))
        lo, L = oracle.bounding_cube(p)
        assert capi.bonsai_cube_from_bounds(p.min(axis=1), p.max(axis=1)) == [*lo.tolist(), L]
    lo, L = oracle.bounding_cube(np.ones((3, 4)))   # all points coincide: L = 1
    assert capi.bonsai_cube_from_bounds([1, 1, 1], [1, 1, 1]) == [*lo.tolist(), L]
    for mn, mx in (([0, 0, 1], [1, 1, 0]), ([0, 0, float("nan")], [1, 1, 1]), ([0, 0, 0], [1, 1, float("inf")])):
        with pytest.raises(capi.BonsaiError) as ex:
            capi.bonsai_cube_from_bounds(mn, mx)
        assert ex.value.code == capi.BONSAI_EINVAL
