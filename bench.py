"""Benchmark of the coupled LB-MD step (one JSON line on rank 0).

A step is one coupled lattice-Boltzmann / MD time step (dense stream-collide
of every node, interpolation at every atom, n_md velocity-Verlet substeps,
spread-back, sparse fix-up), launched as one CUDA graph through the C ABI.

Default workload: the 512^3 z-channel (bounce-back walls, Poiseuille forcing
1e-6, tau 0.8) with ten 20,000-bead synthetic globules (200,000 atoms),
n_md = 128. Both FP16 shifted storage (the headline `value`) and FP32 storage
are timed on it, on the same GPU, and reported on one line.
Metric: coupled MLUPS = nodes x steps / time (whole job, all ranks).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--store f16,f32]

N > 1 runs under torchrun: every rank simulates its own replica (independent
runs; no collective on the data path), timed between barriers, max over ranks.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2305_05025_gb300 import synth  # noqa: E402

DEFAULT_WORKLOAD = "channel10x20k_lattice512"
RELAX_STEPS = 200  # steps from the synthetic start to the flat-cost regime (see timed_run)
# Choices the workload description leaves open: n_md resolves the LJ
# repulsion, gamma keeps the explicit friction exchange stable once the
# globule is dense, skin sets how long a neighbour list lasts.
# Verlet-list skin 0.1: in the relaxed globules (at rest in the fluid) lists
# are rarely rebuilt, so the shortest lists win; measured at 512^3 (FP16):
# skin 0.3 / 0.2 / 0.15 / 0.1 / 0.05 -> 126 / 120 / 101 / 90 / 88 us per
# substep. The skin changes the speed, not the result.
DEFAULT_OVERRIDES = dict(n_md=128, gamma=0.05, skin=0.1)
METRIC = "coupled LB-MD MLUPS"


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(values):
    """Element-wise max over ranks (no-op without a process group). Timing on
    N > 1 takes the slowest rank."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def job_mlups(nodes, steps, world, seconds):
    """Whole-job throughput: every rank advances its own replica of the
    workload (weak scaling), so the job updates nodes*steps*world lattice
    nodes in the slowest rank's time."""
    return nodes * steps * world / seconds / 1e6


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _kernel_hash(files):
    """Hash of the CUDA sources a kernel is built from: a recorded DRAM
    traffic figure is valid only for the source it was measured on."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2305_05025_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


LATTICE_SOURCES = ("lb_step.cu", "lattice.cuh")
MD_SOURCES = ("md.cu", "lbmd_internal.cuh", "lattice.cuh")


def _recorded(name, key, sources):
    """An entry of profiles/<name> (written from one ncu capture) if it was
    taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(key)
    if not e or e.get("kernel_hash") != _kernel_hash(sources):
        return None
    return e


def _traffic(store, nodes):
    """DRAM bytes per launch of the lattice kernel (bytes per node from the
    capture times the nodes of a launch), or None."""
    e = _recorded("lb_step_traffic.json", store, LATTICE_SOURCES)
    return None if e is None else e["dram_bytes_per_node"] * nodes


def _md_traffic(na):
    """DRAM bytes per launch of the substep kernel (per atom from the capture
    times the atoms of a launch), or None."""
    e = _recorded("md_substep_traffic.json", "k_md_substep", MD_SOURCES)
    return None if e is None else e["dram_bytes_per_atom"] * na


class Clocks:
    """Samples nvidia-smi during the timed region."""

    def __init__(self, index):
        self.proc = None
        self.index = index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.result = None
        if self.proc is None:
            return
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        loaded = [s for s in sm if s > 0.5 * max(sm)]
        self.result = {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": max(r[1] for r in rows),
                       "reasons": reasons, "samples": len(rows)}


def _sub_box(cfg, inp, chain, side=48):
    """The atoms of one chain (the first `chain` atoms of the solute, with their
    bonds) moved to the centre of a side^3 box with the workload's walls and
    forcing: one globule of the workload, for the oracle's solute sample."""
    n = chain
    x = inp["x"][:, :n]
    x = x - x.mean(1, keepdims=True) + side / 2.0
    b = inp["bonds"]
    keep = (b[:, 0] < n) & (b[:, 1] < n)
    sub = dict(cfg, nx=side, ny=side, nz=side)
    rho, u = synth.velocity_field((side, side, side), 0.0, 1, cfg.get("rho0", 1.0))
    return sub, dict(rho=rho, u=u, x=x, v=inp["v"][:, :n], mass=inp["mass"][:n], bonds=b[keep],
                     bond_k=inp["bond_k"][keep], bond_r0=inp["bond_r0"][keep])


def oracle_step_seconds(cfg, inp):
    """Seconds the FP64 oracle (single thread) takes for one coupled step of the
    workload, and a description of how it was obtained. Lattices up to 128^3
    nodes: one full step, timed. Larger ones (the 512^3 channel: one full step
    needs ~55 GB of host memory and minutes of CPU time): extrapolated from two
    timed samples that add up to the step: the lattice update of an
    nx x ny x nz_s slab of the same lattice (walls and forcing included,
    nz_s = 2^21 / (nx ny) planes), scaled by nz/nz_s, plus one coupled step of
    the workload's first chain (one 20,000-bead globule) in a 48^3 box, less
    that box's own lattice update, times atoms / chain length."""
    import oracle

    oracle.build.build_oracle()
    nodes = cfg["nx"] * cfg["ny"] * cfg["nz"]

    def one_step(c, i):
        topo = oracle.Topology(i["mass"], i["bonds"], i["bond_k"], i["bond_r0"])
        f = oracle.equilibrium(i["rho"], i["u"])
        t0 = time.perf_counter()
        oracle.run(c, topo, f, i["x"], i["v"], 1)
        return time.perf_counter() - t0

    if nodes <= 128 ** 3:
        t = one_step(cfg, inp)
        return t, f"one full coupled step of {cfg['name']}, timed"
    nz_slab = max(2, min(cfg["nz"], (1 << 21) // (cfg["nx"] * cfg["ny"])))
    slab = dict(cfg, nz=nz_slab)
    t_slab = one_step(slab, synth.inputs(slab, 1, atoms=False))
    b = inp["bonds"]
    links = set(b[b[:, 1] == b[:, 0] + 1, 0].tolist())
    chain = 1  # length of the first chain: beads 0..chain-1 linked by consecutive bonds
    while chain - 1 in links:
        chain += 1
    n_chains = inp["x"].shape[1] / chain
    sub, sub_inp = _sub_box(cfg, inp, chain)
    t_glob = one_step(sub, sub_inp)
    t_sub_lat = one_step(sub, synth.inputs(sub, 1, atoms=False))
    t = t_slab * cfg["nz"] / nz_slab + n_chains * max(t_glob - t_sub_lat, 0.0)
    how = (f"extrapolated: lattice update of a {cfg['nx']}x{cfg['ny']}x{nz_slab} slab ({t_slab:.2f} s) x "
           f"{cfg['nz'] / nz_slab:g}, plus {n_chains:g} x one coupled step of one {chain}-bead globule in a 48^3 box "
           f"less that box's lattice update ({t_glob:.2f} - {t_sub_lat:.2f} s); one coupled step of the "
           f"full workload estimated at {t:.1f} s")
    return t, how


def run_reference(args, cfg):
    """The FP64 oracle on the host cores: each step is one bounded sample of a
    coupled step of the workload (oracle_step_seconds), single thread."""
    inp = synth.inputs(cfg, 1)
    for _ in range(args.warmup):
        oracle_step_seconds(cfg, inp)
    times, how = [], ""
    for _ in range(args.steps):
        t, how = oracle_step_seconds(cfg, inp)
        times.append(t)
    dt = float(np.mean(times))
    nodes = cfg["nx"] * cfg["ny"] * cfg["nz"]
    val = nodes / dt / 1e6
    sample = f"{args.steps} samples after {args.warmup} warm-up, each: {how}"
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(cfg, inp, args.stores),
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _config(cfg, inp, stores):
    na = inp["x"].shape[1]
    nodes = cfg["nx"] * cfg["ny"] * cfg["nz"]
    lat = nodes * 19 * (4 if stores[0] == "f32" else 2) * 2
    return {"workload": cfg["name"], "lattice": [cfg["nx"], cfg["ny"], cfg["nz"]], "tau": cfg["tau"],
            "forcing": cfg["forcing"], "force_amp": cfg["force_amp"], "walls_z": cfg["walls_z"],
            "n_atoms": na, "n_md": cfg["n_md"], "gamma": cfg["gamma"], "skin": cfg["skin"],
            "store": stores[0], "compared_store": stores[1] if len(stores) > 1 else None,
            "coupling": "re-interpolated at every substep" if cfg.get("reinterp") else "held over the step",
            "relaxed_steps": cfg.get("relax", 0),
            "l2": f"inputs larger than L2: {lat / 1e6:.0f} MB of populations per step vs 126 MB L2"}


def cpu_baseline(cfg, inp):
    """Bounded sample of the oracle on this host (oracle_step_seconds)."""
    t, how = oracle_step_seconds(cfg, inp)
    nodes = cfg["nx"] * cfg["ny"] * cfg["nz"]
    return {"value": nodes / t / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": how + ", single thread"}


ADJOINT_WORKLOAD = "chain5k_lattice64_uniform"


def adjoint_timing(stream):
    """Forward + discrete adjoint of the 64^3 / 5,000-bead workload: 200
    steps, checkpoints every 20, gradient of the mean drag with respect to
    gamma, tau and the forcing amplitude; timed with CUDA events around one
    lbmd_backward call, after one untimed call."""
    import torch

    from paper_2305_05025_gb300 import lbmd

    cfg = synth.workload(ADJOINT_WORKLOAD, **DEFAULT_OVERRIDES)
    inp = synth.inputs(cfg, 1)
    steps, ckpt = cfg["steps"], cfg["ckpt_every"]

    def fresh():
        h = lbmd.lbmd_create(cfg, inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"])
        lbmd.lbmd_set_state(h, rho=inp["rho"].astype(np.float32), u=inp["u"].astype(np.float32), x=inp["x"],
                            v=inp["v"].astype(np.float32))
        return h

    h = fresh()
    lbmd.lbmd_backward(h, steps, ckpt, lbmd.OBS_DRAG_X)
    lbmd.lbmd_destroy(h)
    h = fresh()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    lbmd.lbmd_backward(h, steps, ckpt, lbmd.OBS_DRAG_X)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    lbmd.lbmd_destroy(h)
    h = fresh()
    torch.cuda.synchronize()
    t0.record(stream)
    lbmd.lbmd_step(h, steps)
    t1.record(stream)
    torch.cuda.synchronize()
    ms_fwd = t0.elapsed_time(t1)
    lbmd.lbmd_destroy(h)
    nodes = cfg["nx"] * cfg["ny"] * cfg["nz"]
    return {"workload": ADJOINT_WORKLOAD, "steps": steps, "ckpt_every": ckpt, "n_md": cfg["n_md"],
            "gamma": cfg["gamma"], "ms_forward_and_adjoint": ms, "ms_forward_only": ms_fwd,
            "adjoint_over_forward": ms / ms_fwd, "mlups_forward_and_adjoint": nodes * steps / (ms * 1e-3) / 1e6}


def timed_run(args, cfg, inp, store, local, barrier):
    """Creates a handle with storage `store`, runs the warm-up steps, then
    times args.steps coupled steps (one graph launch each) with CUDA events on
    the caller's stream; the lattice kernel and the chain of substep kernels
    of every timed step are timed with events recorded by the step graph on
    their own streams. Returns the handle and the timings."""
    import torch

    from paper_2305_05025_gb300 import lbmd

    c = dict(cfg, store=store)
    na = inp["x"].shape[1]
    h = lbmd.lbmd_create(c, inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"])
    if args.reinterp:
        lbmd.lbmd_set_reinterpolation(h, True)
    lbmd.lbmd_set_state(h, rho=inp["rho32"], u=inp["u32"], x=inp["x"], v=inp["v32"])
    stream = torch.cuda.current_stream()
    # Relaxation, part of the workload's definition: the synthetic globules
    # start as confined random walks and collapse over ~150 steps (the step
    # costs up to 40 % more meanwhile); from ~160 steps on the step time is
    # flat, so the timed window no longer depends on --steps and --warmup.
    relax = getattr(args, "relax", 0)
    if relax:
        lbmd.lbmd_step(h, relax)
    lbmd.lbmd_step(h, args.warmup)
    lbmd.lbmd_check(h)
    mk = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    ev_lb = [mk() for _ in range(args.steps)]
    ev_md = [mk() for _ in range(args.steps)] if na > 0 else []
    ev_step = [mk() for _ in range(args.steps)]
    t0, t1 = mk()
    barrier()
    with Clocks(local) as clk:
        t0.record(stream)
        for i in range(args.steps):
            # torch only reads events it recorded itself: record each pair here
            # first; the step graph's record nodes (later, on the library's
            # streams) set the times that are read.
            for a, b in [ev_lb[i]] + ([ev_md[i]] if na > 0 else []):
                a.record(stream)
                b.record(stream)
            lbmd.lbmd_set_timing_events(h, ev_lb[i][0], ev_lb[i][1])
            if na > 0:
                lbmd.lbmd_set_md_timing_events(h, ev_md[i][0], ev_md[i][1])
            ev_step[i][0].record(stream)
            lbmd.lbmd_step(h, 1)
            ev_step[i][1].record(stream)
        t1.record(stream)
        barrier()
    lbmd.lbmd_set_timing_events(h, None, None)
    if na > 0:
        lbmd.lbmd_set_md_timing_events(h, None, None)
    lbmd.lbmd_check(h)
    steps_ms = [a.elapsed_time(b) for a, b in ev_step]
    return h, {"ms": t0.elapsed_time(t1),
               "lb_ms": float(np.mean([a.elapsed_time(b) for a, b in ev_lb])),
               "md_ms": float(np.mean([a.elapsed_time(b) for a, b in ev_md])) if na > 0 else 0.0,
               "step_ms": steps_ms, "clocks": clk.result}


def _lattice_roofline(store, nodes, lb_ms, hbm, peak_kind):
    bpn = 152 if store == "f32" else 76
    achieved = bpn * nodes / (lb_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": _traffic(store, nodes),
            "kernel": f"dense stream-collide ({'k_lb_step' if store == 'f32' else 'k_lb_step_pair16'}<{store}>), "
                      f"{bpn} B/node algorithmic, {lb_ms * 1e3:.1f} us per launch inside the timed steps "
                      f"(CUDA events on the lattice stream); peak {peak_kind} copy bandwidth",
            "mlups": nodes / (lb_ms * 1e-3) / 1e6}


def run_ours(args, cfg):
    import torch

    from paper_2305_05025_gb300 import lbmd

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    inp = synth.inputs(cfg, 1 + rank)
    inp["rho32"], inp["u32"] = inp["rho"].astype(np.float32), inp["u"].astype(np.float32)
    inp["v32"] = inp["v"].astype(np.float32)
    na = inp["x"].shape[1]
    nodes = cfg["nx"] * cfg["ny"] * cfg["nz"]
    n_md = cfg["n_md"]

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    hbm, peak_kind = _peaks()
    stores = args.stores
    runs = {}
    handle = None
    for store in stores:
        h, r = timed_run(args, cfg, inp, store, local, barrier)
        r["ms"], = reduce_max([r["ms"]])
        runs[store] = r
        if store == stores[0]:
            handle = h
        else:
            lbmd.lbmd_destroy(h)
    prim = runs[stores[0]]
    ms = prim["ms"]
    value = job_mlups(nodes, args.steps, world, ms * 1e-3)

    # End to end through the public API with host buffers: every step loads
    # the whole state (the populations in their storage format, positions,
    # velocities) from pinned host memory with lbmd_load_state, advances one
    # step and saves the state back with lbmd_save_state.
    h = handle
    e2e_steps = 0 if args.no_e2e else 5
    io_bytes = 0
    e2e_s = 0.0
    if e2e_steps:
        import ctypes as C

        pop_t = torch.float32 if stores[0] == "f32" else torch.int16
        pin = {"pop": torch.empty((19, nodes), dtype=pop_t, pin_memory=True),
               "x": torch.empty((3, na), dtype=torch.float64, pin_memory=True),
               "v": torch.empty((3, na), dtype=torch.float32, pin_memory=True)}
        outs = {k: torch.empty_like(t).pin_memory() for k, t in pin.items()}
        L = lbmd.lib()
        vp = lambda t: C.c_void_p(t.data_ptr()) if t.numel() else None
        assert L.lbmd_save_state(h, vp(pin["pop"]), vp(pin["x"]), vp(pin["v"]), 0) == 0
        barrier()
        e0 = time.perf_counter()
        for _ in range(e2e_steps):
            assert L.lbmd_load_state(h, vp(pin["pop"]), vp(pin["x"]), vp(pin["v"]), 0) == 0
            assert L.lbmd_step(h, 1) == 0
            assert L.lbmd_save_state(h, vp(outs["pop"]), vp(outs["x"]), vp(outs["v"]), 0) == 0
        barrier()
        e2e_s = (time.perf_counter() - e0) / e2e_steps
        e2e_s, = reduce_max([e2e_s])
        io_bytes = sum(t.numel() * t.element_size() for t in pin.values())
        del pin, outs
    lbmd.lbmd_destroy(h)

    launches = (n_md + 9) if na > 0 else 2  # 4 sort + interp + (n_md + 1) substeps + spread + dense + fix-up
    lat_roof = {s: _lattice_roofline(s, nodes, runs[s]["lb_ms"], hbm, peak_kind) for s in stores}
    # The dominant kernel: the velocity-Verlet substep (n_md + 1 launches per
    # step). Algorithmic bytes per atom and substep: ~100 (position hi + lo,
    # velocity, force, interpolated velocity, impulse, drift, list length:
    # read and written once), as the scope table's measurement row states.
    md_us = prim["md_ms"] * 1e3 / (n_md + 1) if na > 0 else 0.0
    md_roof = None
    if na > 0:
        md_achieved = 100.0 * na / (md_us * 1e-6) / 1e9
        md_roof = {"bound": "hbm", "achieved": md_achieved, "peak": hbm, "unit": "GB/s", "frac": md_achieved / hbm,
                   "traffic": _md_traffic(na),
                   "kernel": f"k_md_substep (velocity-Verlet substep, {n_md + 1} launches per step, "
                             f"{100 * prim['md_ms'] / (ms / args.steps):.0f}% of the step): 100 B per atom-substep "
                             f"algorithmic x {na} atoms, {md_us:.1f} us per launch (CUDA events around the "
                             f"substep chain on its stream); latency-bound (dependent neighbour-list loads), "
                             f"peak {peak_kind} copy bandwidth"}
    out = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": _config(cfg, inp, stores),
           "roofline": md_roof if md_roof is not None else lat_roof[stores[0]],
           "roofline_lattice": lat_roof[stores[0]],
           "e2e": ({"value": job_mlups(nodes, 1, world, e2e_s), "unit": "MLUPS", "h2d_bytes_per_step": io_bytes,
                    "d2h_bytes_per_step": io_bytes} if e2e_steps else None),
           "gpu_launches": args.steps * launches,
           "atom_updates_per_s": na * args.steps * world / (ms * 1e-3),
           "md_substeps_ms_per_step": prim["md_ms"],
           "md_us_per_substep": prim["md_ms"] * 1e3 / (n_md + 1),
           "step_ms_min_median_max": [min(prim["step_ms"]), float(np.median(prim["step_ms"])), max(prim["step_ms"])],
           "clocks": prim["clocks"]}
    for s in stores[1:]:
        r = runs[s]
        out[s] = {"value": job_mlups(nodes, args.steps, world, r["ms"] * 1e-3), "unit": "MLUPS",
                  "ms_per_step": r["ms"] / args.steps, "lattice": lat_roof[s], "md_substeps_ms_per_step": r["md_ms"],
                  "step_ms_min_median_max": [min(r["step_ms"]), float(np.median(r["step_ms"])), max(r["step_ms"])],
                  "clocks": r["clocks"]}
        out[f"{stores[0]}_over_{s}"] = {"coupled": runs[s]["ms"] / ms,
                                       "lattice_kernel": runs[s]["lb_ms"] / prim["lb_ms"]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(cfg, inp)
    if world == 1 and not args.no_adjoint:
        out["adjoint"] = adjoint_timing(torch.cuda.current_stream())
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return out if rank == 0 else None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--store", default="f16,f32",
                    help="storage formats, comma separated: the first is the headline, the others are timed "
                         "on the same workload and reported beside it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the timing of the adjoint workload")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end timing with host buffers")
    ap.add_argument("--skin", type=float, default=None,
                    help=f"Verlet-list skin (default {DEFAULT_OVERRIDES['skin']}): changes the speed, not the result")
    ap.add_argument("--relax", type=int, default=RELAX_STEPS,
                    help="untimed steps from the synthetic start before the warm-up (part of the workload: the "
                         "globules' collapse; 0 times the transient)")
    ap.add_argument("--reinterp", action="store_true",
                    help="re-interpolate the fluid velocity at every substep (the coupling variant; default: "
                         "held over the step)")
    args = ap.parse_args()
    args.stores = [s.strip() for s in args.store.split(",") if s.strip()]
    for s in args.stores:
        if s not in ("f32", "f16", "bf16"):
            ap.error(f"unknown store {s}")
    overrides = dict(DEFAULT_OVERRIDES)
    if args.skin is not None:
        overrides["skin"] = args.skin
    cfg = synth.workload(args.workload, **overrides)
    cfg["store"] = args.stores[0]
    cfg["reinterp"] = int(args.reinterp)
    cfg["relax"] = args.relax
    if args.impl == "reference":
        world, rank, _ = _dist()
        if rank != 0:
            return
        # Each oracle sample takes ~10-30 s on one core: at most 5 timed
        # samples after at most 1 warm-up keep the run within a few minutes
        # (the line reports the samples actually taken).
        args.steps = min(args.steps, 5)
        args.warmup = min(args.warmup, 1)
        out = run_reference(args, cfg)
    else:
        out = run_ours(args, cfg)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
