"""Shared helpers of the GPU parity tests: run the CUDA path through the C
ABI and the oracle on the same seeded inputs."""
import numpy as np
import torch

import oracle
from paper_1412_0659_gb300 import TreeGravity

DEV = torch.device("cuda", 0)


def gpu_run(pos, mass, theta=0.4, eps=0.01, G=1.0, debug=True):
    g = TreeGravity(G=G, theta=theta, eps=eps)
    g.build(torch.from_numpy(np.ascontiguousarray(pos)).to(DEV),
            torch.from_numpy(np.ascontiguousarray(mass)).to(DEV))
    acc, pot = g.forces(theta, eps)
    torch.cuda.synchronize()
    out = {"g": g, "acc": acc.cpu().numpy().astype(np.float64), "pot": pot.cpu().numpy().astype(np.float64),
           "stats": g.stats()}
    if debug:
        d = g.debug()
        out["keys"] = d["keys"].cpu().numpy().view(np.uint64)
        out["perm"] = d["perm"].cpu().numpy().view(np.uint32)
        out["nodes"] = {k: v.cpu().numpy().view(np.uint32) for k, v in d["nodes"].items()}
        out["M"] = d["M"].cpu().numpy()
        out["com"] = d["com"].cpu().numpy()
        out["Q"] = d["Q"].cpu().numpy()
        out["group_first"] = d["group_first"].cpu().numpy().view(np.uint32)
        out["group_count"] = d["group_count"].cpu().numpy().view(np.uint32)
        out["lo"], out["L"] = np.array(d["lo"]), d["L"]
        npp, npc = g.group_lists()
        out["g_npp"], out["g_npc"] = npp.cpu().numpy(), npc.cpu().numpy()
    return out


def rel_err_vec(a, b):
    return np.linalg.norm(a - b, axis=0) / np.maximum(np.linalg.norm(b, axis=0), 1e-300)


def assert_force_tolerance(acc, pot, acc_o, pot_o, median=2e-6, p999=1e-4):
    """The acceleration tolerance: median relative error <= 2e-6 and the
    99.9th percentile <= 1e-4 against the FP64 oracle tree with the same
    interaction lists; the potential is held to the same bounds."""
    e = rel_err_vec(acc, acc_o)
    pe = np.abs(pot - pot_o) / np.maximum(np.abs(pot_o), 1e-300)
    assert np.median(e) <= median, ("acc median", np.median(e))
    assert np.quantile(e, 0.999) <= p999, ("acc p99.9", np.quantile(e, 0.999))
    assert np.median(pe) <= median, ("pot median", np.median(pe))
    assert np.quantile(pe, 0.999) <= p999, ("pot p99.9", np.quantile(pe, 0.999))
    return float(np.median(e)), float(np.quantile(e, 0.999))


def oracle_tree(pos, mass):
    return oracle.Tree(pos, mass)
