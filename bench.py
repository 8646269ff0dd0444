"""Benchmark: tree-force Tflop/s (the paper's 23/65-flop convention) and
particles/s of the full Bonsai step on one GB300.

Workload (default): the Milky-Way-like model with N = 2^23 particles
(Hernquist halo : exponential disk : Hernquist bulge = 5 : 1 : 0.2,
theta = 0.4, eps = 10 pc, dt = 0.1 Myr), seeded and synthetic.  One step is
the whole hot path: kick, drift, bounding box, Peano-Hilbert keys, radix
sort, gather, octree, groups, FP64 multipoles, cell pack, the fused walk +
force kernel, kick, and the FP64 energy/momentum diagnostics.

value = sum over timed steps of (23 n_pp + 65 n_pc) / timed wall time on the
device (CUDA events, max over ranks).  The state (about 1.7 GB) is far larger
than the 129 MB L2, so no flush is needed between steps.

Keys beside the contract's: ``roofline`` (the walk kernel against the
derived FP32 peak, with its captured DRAM bytes), ``e2e`` (tree_solve_host
with host buffers), ``cpu_baseline`` (the oracle on the host cores),
``adjoint`` (forward and force VJP on the same tree), ``direct`` (direct
summation of 2^16 targets, the paper's Fig. 1 comparison), ``io`` (snapshot
save / load and the face-on surface density), ``ics`` (the Sec. IV model
generated on the device), ``domains`` (eight domains with local essential
trees on this GPU), ``clocks`` and ``gpu_launches``.  ``--no-adjoint``,
``--no-direct``, ``--no-io``, ``--no-ics`` and ``--domains 0`` skip the
extras; ``--workload`` selects another configuration.

``--impl reference`` times the FP64 CPU oracle (the stand-in for the
paper's own code, which is not available) on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# DRAM bytes (read + written) of one walk/force launch, from a one-pass ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of the benchmark
# command, valid only for the walk source it was taken on (checked by hash).
WALK_TRAFFIC = {"walk_cu_sha256": "f3e50b2961f83dc556f74d353fdd631929d31e752f92fb8591f1e539ffa6231e",
                "bytes": {"milky-way-2^23": 822.408192e6 + 327.783424e6}}

METRIC = "tree-force Tflop/s (23 flops/p-p + 65 flops/p-c, Sec. VI.A) per full KDK step, theta=0.4"
UNIT = "Tflop/s"
FP32_LANES_PER_SM = 128


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(t_ms: float, work: float, world: int, device=None):
    """Whole-job figures of a timed region: the maximum wall time over ranks
    and the sum of the work (flops) done by all ranks.  Every rank calls it;
    with one rank it returns its inputs."""
    if world <= 1:
        return t_ms, work
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ww = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(ww)
    return float(tt.item()), float(ww.item())


def walk_traffic(workload: str):
    """The captured DRAM bytes per walk launch for this workload, or None
    when there is no capture of the current walk source."""
    import hashlib
    path = os.path.join(ROOT, "paper_1412_0659_gb300", "csrc", "walk.cu")
    with open(path, "rb") as f:
        digest = hashlib.sha256(f.read()).hexdigest()
    if digest != WALK_TRAFFIC["walk_cu_sha256"]:
        return None
    return WALK_TRAFFIC["bytes"].get(workload)


def _sec4_model(n: int, seed: int, on_gpu: bool):
    """The Sec. IV model (NFW halo, exponential disk, Hernquist bulge) as a
    workload: generated by the library on the device for our arm, by the
    FP64 oracle on the host for the reference arm (the two agree particle
    for particle)."""
    import workloads
    if on_gpu:
        from paper_1412_0659_gb300 import galaxy
        gal = galaxy.sec4(n, seed)
        pos, vel, mass = [x.cpu().numpy() for x in galaxy.generate(gal)]
        counts = (int(gal.n_halo), int(gal.n_disk), int(gal.n_bulge))
        G = gal.G
    else:
        from oracle import galaxy_ics
        gal = galaxy_ics.milky_way_sec4(n, seed)
        pos, vel, mass = galaxy_ics.generate(gal)
        counts = (gal.n_halo, gal.n_disk, gal.n_bulge)
        G = gal.G
    h, d, b = counts
    comps = {"halo": (0, h), "disk": (h, d), "bulge": (h + d, b)}
    return workloads.Model(pos, vel, mass, G, 0.01, 0.4, 0.1, f"sec4-{n}", comps)


def _workload(name: str, rank: int, on_gpu: bool = True):
    import workloads
    if name == "sec4-2^23":
        m = _sec4_model(1 << 23, 1006 + 17 * rank, on_gpu)
        desc = ("Sec. IV Milky Way N=2^23 generated on the fly (NFW halo 6.0e11 Msun a=15 kpc, exp. "
                "disk 5e10 Msun Rd=2.5 kpc z0=0.3 kpc, Hernquist bulge 4.6e9 Msun a=0.5 kpc; counts "
                "in the paper's ratio), theta=0.4, eps=10 pc, dt=0.1 Myr")
    elif name == "milky-way-2^23":
        m = workloads.milky_way(1 << 23, seed=1002 + 17 * rank, eps=0.01, theta=0.4, dt=0.1)
        desc = ("Milky-Way-like N=2^23 (Hernquist halo 1e12 Msun a=30 kpc cut 200 kpc, exp. disk "
                "5e10 Msun Rd=2.5 kpc z0=0.3 kpc Q=1.5, Hernquist bulge 1e10 Msun a=0.5 kpc; "
                "5:1:0.2), theta=0.4, eps=10 pc, dt=0.1 Myr")
    elif name == "milky-way-2^20":
        m = workloads.milky_way(1 << 20, seed=1002 + 17 * rank, eps=0.01, theta=0.4, dt=0.1)
        desc = "Milky-Way-like N=2^20 (same profiles as the 2^23 model), theta=0.4, eps=10 pc, dt=0.1 Myr"
    elif name == "milky-way-2^25":
        m = workloads.milky_way(1 << 25, seed=1003 + 17 * rank, eps=0.01, theta=0.4, dt=0.1)
        desc = "Milky-Way-like N=2^25 (the precision-study model), theta=0.4, eps=10 pc, dt=0.1 Myr"
    elif name == "milky-way-2^28":
        m = workloads.milky_way(1 << 28, seed=1005 + 17 * rank, eps=0.005, theta=0.4, dt=0.1)
        desc = "Milky-Way-like N=2^28 (the largest single-GPU model), theta=0.4, eps=5 pc, dt=0.1 Myr"
    elif name == "halo-disk-2^20":
        m = workloads.halo_disk(1 << 19, 1 << 19, seed=1004 + 17 * rank, eps=0.02, dt=0.1)
        desc = "Plummer halo 2^19 (1e11 Msun, a=10 kpc) + exponential disk 2^19, theta=0.4, eps=20 pc"
    elif name == "plummer-2^14":
        m = workloads.plummer(1 << 14, seed=1001 + 17 * rank)
        desc = "Plummer N=2^14, G=M=a=1, theta=0.4, eps=0.01, dt=1/64"
    else:
        raise SystemExit(f"unknown workload {name}")
    return m, desc


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1412_0659_gb300 import TreeGravity, build, fp32_peak_tflops
    build.build()
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    m, desc = _workload(args.workload, rank)
    n = m.n
    pos = torch.from_numpy(m.pos).to(dev)
    vel = torch.from_numpy(m.vel).to(dev)
    mass = torch.from_numpy(m.mass).to(dev)
    stream = torch.cuda.current_stream()
    g = TreeGravity(G=m.G, theta=m.theta, eps=m.eps)
    g.build(pos, mass)
    g.set_velocities(vel)
    g.forces()
    for _ in range(args.warmup):
        g.step(m.dt)
        g.diagnostics()
    st0 = g.stats()
    launches0 = st0["launches"]
    flops, walk_ms, force_ms, keys_ms, tree_ms, npp, npc = 0.0, [], [], [], [], [], []
    clocks = ClockSampler(torch.cuda.current_device())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    diag = None
    for _ in range(args.steps):
        g.step(m.dt)
        diag = g.diagnostics()
        st = g.stats()
        flops += st["flops"]
        walk_ms.append(st["ms_walk"])
        force_ms.append(st["ms_force"])
        keys_ms.append(st["ms_keys"])
        tree_ms.append(st["ms_tree"])
        npp.append(st["n_pp"])
        npc.append(st["n_pc"])
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    t_ms = e0.elapsed_time(e1)
    launches = g.stats()["launches"] - launches0
    t_max, tot_flops = aggregate(t_ms, flops, world, dev)
    value = tot_flops / (t_max * 1e-3) / 1e12
    ms_per_step = t_max / args.steps

    # --- adjoint: force VJP on the same tree and lists, against the forward ---
    adjoint = None
    if not args.no_adjoint:
        lam = torch.randn(3, n, device=dev)
        mu = torch.randn(n, device=dev)
        g.forces()
        g.forces_vjp(lam, mu)
        tf, tb = [], []
        for _ in range(max(2, min(args.steps, 5))):
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a2 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            g.forces()
            a1.record(stream)
            g.forces_vjp(lam, mu)
            a2.record(stream)
            torch.cuda.synchronize()
            tf.append(a0.elapsed_time(a1))
            tb.append(a1.elapsed_time(a2))
        fwd, bwd = statistics.median(tf), statistics.median(tb)
        adjoint = {"fwd_ms": fwd, "vjp_ms": bwd, "ratio_fwd_plus_bwd_over_fwd": (fwd + bwd) / fwd,
                   "what": "tree_forces then tree_forces_vjp (random cotangents for a and phi) on the "
                           "same tree, median of repeats"}

    # --- end to end through the host-buffer C-ABI entry (copies timed) ---
    pin_pos = torch.from_numpy(m.pos).pin_memory()
    pin_mass = torch.from_numpy(m.mass).pin_memory()
    pin_acc = torch.empty((3, n), dtype=torch.float32).pin_memory()
    pin_pot = torch.empty(n, dtype=torch.float32).pin_memory()
    ge = TreeGravity(G=m.G, theta=m.theta, eps=m.eps)
    ge.solve_host(pin_pos, pin_mass, pin_acc, pin_pot)
    e_steps = max(1, min(args.steps, 3))
    e_flops = 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e_steps):
        ge.solve_host(pin_pos, pin_mass, pin_acc, pin_pot)
        e_flops += ge.stats()["flops"]
    torch.cuda.synchronize()
    e_s = time.perf_counter() - t0
    # the GPU forces of the initial state, kept for the comparison with the
    # oracle in the CPU-baseline leg
    g_npp0, g_npc0 = (x.cpu().numpy() for x in ge.group_lists())
    gpu_forces0 = (pin_acc.double().numpy().copy(), pin_pot.double().numpy().copy(), g_npp0, g_npc0)
    ge.close()
    e_s, e_flops = aggregate(e_s, e_flops, world, dev)
    e2e = {"value": e_flops / e_s / 1e12, "unit": UNIT,
           "h2d_bytes_per_step": int(pin_pos.numel() * 8 + pin_mass.numel() * 8),
           "d2h_bytes_per_step": int(pin_acc.numel() * 4 + pin_pot.numel() * 4),
           "what": "tree_solve_host: H2D pos+mass, build, forces, D2H acc+pot (one force evaluation)"}

    # --- roofline of the dominant kernel (the fused walk/force) ---
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    pk = _peaks()
    max_mhz = pk.get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0
    peak = fp32_peak_tflops(sms, FP32_LANES_PER_SM, max_mhz)
    walk_avg = sum(walk_ms) / len(walk_ms)
    flops_launch = flops / args.steps
    achieved = flops_launch / (walk_avg * 1e-3) / 1e12
    traffic = args.traffic if args.traffic is not None else walk_traffic(args.workload)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "k_walk (fused walk + p-p/p-c evaluation)",
                "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flops x {max_mhz:.0f} MHz",
                "convention_cap": "82 % of peak for p-p (23 flops in 14 FP32 instructions) and 93 % for p-c "
                                  "(65 flops in 35) at one FP32 instruction per lane and cycle"}

    # --- direct summation on the same particles (the paper's Fig. 1 compares
    # tree and direct N-body performance): 2^16 targets over all sources ---
    direct = None
    if not args.no_direct:
        nt = min(n, 1 << 16)
        tgt = torch.from_numpy(np.random.default_rng(5).choice(n, nt, replace=False)).to(dev)
        g.direct_forces(tgt)
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        g.direct_forces(tgt)
        d1.record(stream)
        torch.cuda.synchronize()
        d_s = d0.elapsed_time(d1) * 1e-3
        pairs = float(nt) * n
        direct = {"targets": nt, "sources": n, "ms": d_s * 1e3, "pairs_per_s": pairs / d_s,
                  "tflops_23_per_pair": 23.0 * pairs / d_s / 1e12,
                  "tree_speedup_per_particle": (n / (walk_avg * 1e-3)) / (nt / d_s),
                  "what": "tree_direct_forces: FP32 pair terms, FP64 tile sums; tree_speedup_per_particle = "
                          "particles/s of the tree walk / particles/s of direct summation"}

    # --- snapshot I/O and the on-the-fly face-on surface density (disk and
    # bulge, 1024 x 1024 pixels over 30 x 30 kpc) ---
    io = None
    if not args.no_io:
        import tempfile
        with tempfile.TemporaryDirectory() as td:
            path = os.path.join(td, f"snapshot{rank}.bin")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.save(path, 0.0)
            t1 = time.perf_counter()
            gl = TreeGravity(G=m.G, theta=m.theta, eps=m.eps)
            gl.load(path)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            gl.close()
            nbytes = os.path.getsize(path)
        comp = [v for k, v in m.components.items() if k != "halo"]
        first = min(c[0] for c in comp) if comp else 0
        count = sum(c[1] for c in comp) if comp else n
        window = (-15.0, 15.0, -15.0, 15.0)
        g.surface_density(first, count, window, 1024, 1024)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        g.surface_density(first, count, window, 1024, 1024)
        s1.record(stream)
        torch.cuda.synchronize()
        map_ms = s0.elapsed_time(s1)
        io = {"snapshot_bytes": nbytes, "save_gb_per_s": nbytes / (t1 - t0) / 1e9,
              "load_and_build_gb_per_s": nbytes / (t2 - t1) / 1e9,
              "surface_density_ms": map_ms, "surface_density_particles": count,
              "what": "tree_save_snapshot / tree_load_snapshot (includes the tree build) of the FP64 "
                      "state to a local temporary file; tree_surface_density of disk + bulge, "
                      "1024^2 pixels, CUDA events (includes the map clear and a stream sync)"}

    # --- on-the-fly initial conditions (Sec. IV): the Milky Way model (NFW
    # halo, exponential disk, Hernquist bulge) of the same size generated on
    # the device, tables and sampling, CUDA events around the whole call ---
    ics = None
    if not args.no_ics:
        from paper_1412_0659_gb300 import capi as _capi, galaxy
        gal = galaxy.sec4(n, 1006 + rank)
        ipos = torch.empty(3, n, dtype=torch.float64, device=dev)
        ivel = torch.empty_like(ipos)
        imass = torch.empty(n, dtype=torch.float64, device=dev)
        cs = torch.cuda.current_stream()
        _capi.bonsai_galaxy_generate(gal, ipos, ivel, imass, cs)
        ts = []
        for _ in range(3):
            i0 = torch.cuda.Event(enable_timing=True)
            i1 = torch.cuda.Event(enable_timing=True)
            i0.record(cs)
            _capi.bonsai_galaxy_generate(gal, ipos, ivel, imass, cs)
            i1.record(cs)
            torch.cuda.synchronize()
            ts.append(i0.elapsed_time(i1))
        ics = {"model": "Sec. IV Milky Way: NFW halo 6.0e11, exponential disk 5.0e10, Hernquist bulge "
                        f"4.6e9 Msun; {int(gal.n_halo)} + {int(gal.n_disk)} + {int(gal.n_bulge)} particles",
               "ms": min(ts), "particles_per_s": n / (min(ts) * 1e-3), "launches_per_call": 14,
               "what": "bonsai_galaxy_generate: Eddington tables, speed and disk tables, Philox sampling, "
                       "centre-of-mass shift; FP64 throughout"}
        del ipos, ivel, imass

    # --- domains and local essential trees (Sec. III.B) emulated on this GPU:
    # the state split into R pieces of the key order, each domain's own walk
    # plus the walks of the R - 1 LETs it receives ---
    dom = None
    if args.domains > 1:
        from paper_1412_0659_gb300 import domains as dmod
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        doms = dmod.split(g, args.domains)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        let = dmod.Let()
        own_ms, let_ms, let_build_s, dflops, nbytes = 0.0, 0.0, 0.0, 0.0, []
        for i, (gi, _) in enumerate(doms):
            gi.forces(m.theta, m.eps)
            st = gi.stats()
            own_ms += st["ms_walk"]
            dflops += st["flops"]
            for j, (gj, _) in enumerate(doms):
                if j == i:
                    continue
                tb = time.perf_counter()
                let.build(gj, gi, m.theta)
                let_build_s += time.perf_counter() - tb
                nbytes.append(let.info()["bytes"])
                let.add_forces(gi, m.eps)
                st = gi.stats()
                let_ms += st["ms_walk"]
                dflops += st["flops"]
        let.close()
        for gi, _ in doms:
            gi.close()
        dom = {"domains": args.domains, "split_and_build_s": t1 - t0, "own_walks_ms": own_ms,
               "let_walks_ms": let_ms, "let_build_s": let_build_s, "let_bytes_total": int(sum(nbytes)),
               "let_bytes_max_pair": int(max(nbytes)),
               "walk_tflops": dflops / ((own_ms + let_ms) * 1e-3) / 1e12,
               "flops_vs_single_tree": dflops / (flops / args.steps),
               "what": "domains.split + tree_build_cube per domain; tree_forces (own walk) and, per "
                       "source domain, let_build (host-timed, includes its syncs) and let_forces "
                       "(CUDA events of the walk); flops in the 23/65 convention"}

    cpu, accuracy = None, None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, accuracy = cpu_baseline(m, args.cpu_groups, gpu_forces0)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded generator; the paper's Milky Way realisation is not available)",
            "config": _config(desc, n, world),
            "particles_per_s": world * n * args.steps / (t_max * 1e-3),
            "force_particles_per_s": n / (walk_avg * 1e-3),
            "force_kernel_tflops": achieved,
            "pct_fp32_peak": 100.0 * value / peak,
            "n_pp_per_particle": statistics.mean(npp) / n, "n_pc_per_particle": statistics.mean(npc) / n,
            "phase_ms": {"keys_sort": statistics.mean(keys_ms), "tree_groups_multipoles": statistics.mean(tree_ms),
                         "force": statistics.mean(force_ms), "walk_kernel": walk_avg},
            "energy": {"E_tot": diag["E_tot"] if diag else None},
            "adjoint": adjoint, "direct": direct, "io": io, "ics": ics, "domains": dom,
            "clocks": clk, "gpu_launches": int(launches), "roofline": roofline, "e2e": e2e,
            "cpu_baseline": cpu, "accuracy": accuracy,
        }
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        dist.destroy_process_group()


def _config(desc: str, n: int, world: int) -> dict:
    """The workload description, identical in both arms."""
    return {"workload": desc, "n_per_gpu": n,
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2_flush": "none: inputs (~1.7 GB state) larger than L2",
            "arith": "FP32 forces on group-relative coordinates; FP64 keys, multipoles, state, diagnostics"}


def cpu_baseline(m, n_groups: int, gpu=None):
    """The FP64 oracle on the host cores: full tree build of the same workload
    plus the force walk of a seeded sample of groups; the force time is scaled
    to all groups by flops.  Returns the oracle's Tflop/s for one step, and,
    when gpu = (acc, pot, g_npp, g_npc) holds the GPU's forces of the same
    state (caller order) and its per-group list lengths, the GPU's error
    against the oracle on the sampled groups' particles."""
    import numpy as np

    import oracle
    t0 = time.perf_counter()
    t = oracle.Tree(m.pos, m.mass)
    t_build = time.perf_counter() - t0
    rng = np.random.default_rng(7)
    sel = np.sort(rng.choice(t.ngroups, min(n_groups, t.ngroups), replace=False))
    g = t.groups()
    t1 = time.perf_counter()
    acc_s, pot_s, g_npp, g_npc, _ = t.forces_groups(m.theta, m.eps, m.G, sel)
    t_force = time.perf_counter() - t1
    cnt = g["count"][sel].astype(np.float64)
    f_sample = float((23.0 * cnt * g_npp[sel] + 65.0 * cnt * g_npc[sel]).sum())
    n_sample = float(cnt.sum())
    # the whole step's flops estimated from the sample's flops per particle
    f_total = f_sample * m.n / n_sample
    t_total = t_build + t_force * (f_total / f_sample)
    cpu = {"value": f_total / t_total / 1e12, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": (f"FP64 C oracle: full tree build of the same N={m.n} workload ({t_build:.1f} s) + force walk "
                      f"of {len(sel)} seeded random groups ({int(n_sample)} particles, {t_force:.1f} s), "
                      "force time scaled to all particles by flops"),
           "force_only_tflops": f_sample / t_force / 1e12}
    if gpu is None:
        return cpu, None
    acc_g, pot_g, gnpp, gnpc = gpu
    _, perm = t.keys()
    rows = np.concatenate([np.arange(g["first"][k], g["first"][k] + g["count"][k]) for k in sel])
    ci = perm[rows]                                   # caller indices of the sampled particles
    ao, po = acc_s[:, rows], pot_s[rows]
    e = np.linalg.norm(acc_g[:, ci] - ao, axis=0) / np.linalg.norm(ao, axis=0)
    pe = np.abs(pot_g[ci] - po) / np.abs(po)
    acc = {"median_rel": float(np.median(e)), "p999_rel": float(np.quantile(e, 0.999)),
           "max_rel": float(e.max()), "pot_median_rel": float(np.median(pe)),
           "pot_p999_rel": float(np.quantile(pe, 0.999)),
           "n_pp_match": float(np.mean(gnpp[sel] == g_npp[sel])),
           "n_pc_match": float(np.mean(gnpc[sel] == g_npc[sel])),
           "groups": int(len(sel)), "particles": int(len(rows)),
           "tolerance": {"median_rel": 2e-6, "p999_rel": 1e-4, "counts": "equal"},
           "within_tolerance": bool(np.median(e) <= 2e-6 and np.quantile(e, 0.999) <= 1e-4
                                    and np.median(pe) <= 2e-6 and np.quantile(pe, 0.999) <= 1e-4
                                    and np.all(gnpp[sel] == g_npp[sel]) and np.all(gnpc[sel] == g_npc[sel])),
           "what": "GPU forces of the initial state (tree_solve_host) against the FP64 oracle tree on the "
                   "particles of the sampled groups; per-group list lengths compared"}
    return cpu, acc


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, as it stands, on the host cores."""
    rank, world, local = _dist()
    if rank != 0:
        return
    m, desc = _workload(args.workload, 0, on_gpu=False)
    import oracle
    for _ in range(args.warmup):
        # untimed: a small force walk (threads spun up, code and tables paged in)
        oracle.forces(m.pos[:, :4096], m.mass[:4096], m.theta, m.eps, m.G)
    vals = []
    t0 = time.perf_counter()
    cpu = None
    for _ in range(max(1, args.steps)):
        cpu, _ = cpu_baseline(m, args.cpu_groups)
        vals.append(cpu["value"])
    wall = time.perf_counter() - t0
    value = statistics.mean(vals)
    cpu = dict(cpu, value=value)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generator; the paper's Milky Way realisation is not available)",
            "config": _config(desc, m.n, world),
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="milky-way-2^23",
                    choices=["milky-way-2^23", "milky-way-2^20", "milky-way-2^25", "milky-way-2^28",
                             "halo-disk-2^20", "plummer-2^14", "sec4-2^23"])
    ap.add_argument("--cpu-groups", type=int, default=24000,
                    help="groups walked by the CPU oracle sample (about 10 s of CPU work at 2^23)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward timing")
    ap.add_argument("--no-direct", action="store_true", help="skip the direct-summation comparison")
    ap.add_argument("--no-io", action="store_true", help="skip the snapshot and surface-density timing")
    ap.add_argument("--no-ics", action="store_true", help="skip the on-the-fly initial-condition timing")
    ap.add_argument("--domains", type=int, default=8,
                    help="domains of the local-essential-tree emulation (0 or 1 to skip)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per walk launch from an ncu capture (null when not captured)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
