"""Benchmark of the coupled LB-MD step (one JSON line on rank 0).

A step is one coupled lattice-Boltzmann / MD time step (dense stream-collide
of every node, interpolation at every atom, n_md velocity-Verlet substeps,
spread-back, sparse fix-up), launched as one CUDA graph through the C ABI.

Default workload: 128^3 periodic lattice, tau 0.6, Kolmogorov forcing 1e-5,
20,000-bead synthetic globule (radius 20), FP32 populations, n_md = 128.
Metric: coupled MLUPS = nodes x steps / time (whole job, all ranks).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--store f32|f16|bf16]

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

DEFAULT_WORKLOAD = "globule20k_lattice128"
# Choices the workload description leaves open: n_md resolves the LJ
# repulsion, gamma keeps the explicit friction exchange stable once the
# globule is dense, skin sets how long a neighbour list lasts.
DEFAULT_OVERRIDES = dict(n_md=128, gamma=0.05, skin=0.3)
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


def _kernel_hash():
    h = hashlib.sha256()
    for f in ("lb.cu", "lbmd_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2305_05025_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(store, nodes):
    """DRAM bytes per launch of the lattice kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "lb_step_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(store)
    if not e or e.get("kernel_hash") != _kernel_hash():
        return None
    return e["dram_bytes_per_node"] * nodes


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


def run_reference(args, cfg):
    """The FP64 oracle on the host cores: each step is one full coupled step of
    the workload (single thread)."""
    import oracle

    oracle.build.build_oracle()
    inp = synth.inputs(cfg, 1)
    topo = oracle.Topology(inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"])
    f = oracle.equilibrium(inp["rho"], inp["u"])
    x, v = inp["x"], inp["v"]
    if args.warmup:
        f, x, v, _ = oracle.run(cfg, topo, f, x, v, args.warmup)
    t0 = time.perf_counter()
    f, x, v, _ = oracle.run(cfg, topo, f, x, v, args.steps)
    dt = time.perf_counter() - t0
    nodes = cfg["nx"] * cfg["ny"] * cfg["nz"]
    val = nodes * args.steps / dt / 1e6
    sample = f"{args.steps} full coupled steps of {cfg['name']} after {args.warmup} warm-up steps"
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(cfg, inp),
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _config(cfg, inp):
    na = inp["x"].shape[1]
    lat = cfg["nx"] * cfg["ny"] * cfg["nz"] * 19 * (4 if cfg["store"] == "f32" else 2) * 2
    return {"workload": cfg["name"], "lattice": [cfg["nx"], cfg["ny"], cfg["nz"]], "tau": cfg["tau"],
            "forcing": cfg["forcing"], "force_amp": cfg["force_amp"], "walls_z": cfg["walls_z"],
            "n_atoms": na, "n_md": cfg["n_md"], "gamma": cfg["gamma"], "store": cfg["store"],
            "l2": f"inputs larger than L2: {lat / 1e6:.0f} MB of populations per step vs 126 MB L2"}


def cpu_baseline(cfg, inp, steps=3):
    """Bounded sample of the oracle on this host: `steps` full coupled steps."""
    import oracle

    oracle.build.build_oracle()
    topo = oracle.Topology(inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"])
    f = oracle.equilibrium(inp["rho"], inp["u"])
    t0 = time.perf_counter()
    oracle.run(cfg, topo, f, inp["x"], inp["v"], steps)
    dt = time.perf_counter() - t0
    nodes = cfg["nx"] * cfg["ny"] * cfg["nz"]
    return {"value": nodes * steps / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"{steps} full coupled steps of {cfg['name']} from the initial state, single thread, "
                      f"{dt:.1f} s"}


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


def run_ours(args, cfg):
    import torch

    from paper_2305_05025_gb300 import lbmd

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    inp = synth.inputs(cfg, 1 + rank)
    na = inp["x"].shape[1]
    nodes = cfg["nx"] * cfg["ny"] * cfg["nz"]
    h = lbmd.lbmd_create(cfg, inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"])
    rho32, u32 = inp["rho"].astype(np.float32), inp["u"].astype(np.float32)
    v32 = inp["v"].astype(np.float32)
    lbmd.lbmd_set_state(h, rho=rho32, u=u32, x=inp["x"], v=v32)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    lbmd.lbmd_step(h, args.warmup)
    lbmd.lbmd_check(h)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with Clocks(local) as clk:
        t0.record(stream)
        for i in range(args.steps):
            # torch only reads events it recorded itself: record both here; the
            # graph's record nodes (later on the same stream) set the times used.
            ev[i][0].record(stream)
            ev[i][1].record(stream)
            lbmd.lbmd_set_timing_events(h, ev[i][0], ev[i][1])
            lbmd.lbmd_step(h, 1)
        t1.record(stream)
        barrier()
    lbmd.lbmd_set_timing_events(h, None, None)
    lbmd.lbmd_check(h)
    ms = t0.elapsed_time(t1)
    lb_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    ms, = reduce_max([ms])
    value = job_mlups(nodes, args.steps, world, ms * 1e-3)

    # End to end through the public API with host buffers: every step copies
    # the full state in (populations, positions, velocities) from pinned host
    # memory, advances one step and copies the state out again.
    e2e_steps = max(3, min(args.steps // 10, 20))
    st = lbmd.lbmd_get_fields(h, f=True, x=True, v=True)
    pin = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for k, a in st.items()}
    host = {k: t.numpy() for k, t in pin.items()}
    outs = {k: torch.empty_like(t).pin_memory().numpy() for k, t in pin.items()}
    import ctypes as C

    L = lbmd.lib()
    vp = lambda a: a.ctypes.data_as(C.c_void_p)
    barrier()
    e0 = time.perf_counter()
    for _ in range(e2e_steps):
        assert L.lbmd_set_state(h, vp(host["f"]), None, None, vp(host["x"]), vp(host["v"]), 0) == 0
        assert L.lbmd_step(h, 1) == 0
        assert L.lbmd_get_fields(h, vp(outs["f"]), None, None, vp(outs["x"]), vp(outs["v"]), 0) == 0
    barrier()
    e2e_s = (time.perf_counter() - e0) / e2e_steps
    e2e_s, = reduce_max([e2e_s])
    io_bytes = host["f"].nbytes + host["x"].nbytes + host["v"].nbytes

    hbm, peak_kind = _peaks()
    bpn = 152 if cfg["store"] == "f32" else 76
    achieved = bpn * nodes / (lb_ms * 1e-3) / 1e9
    traffic = _traffic(cfg["store"], nodes)
    out = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": _config(cfg, inp),
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                        "frac": achieved / hbm, "traffic": traffic,
                        "kernel": f"k_lb_step<{cfg['store']}> (dense stream-collide), {bpn} B/node algorithmic, "
                                  f"{lb_ms * 1e3:.1f} us per launch inside the timed steps; peak {peak_kind}"},
           "e2e": {"value": job_mlups(nodes, 1, world, e2e_s), "unit": "MLUPS", "h2d_bytes_per_step": io_bytes,
                   "d2h_bytes_per_step": io_bytes},
           # per coupled step: 3 sort + interp + (n_md + 1) substeps + spread + dense step + fix-up
           "gpu_launches": args.steps * ((cfg["n_md"] + 8) if na > 0 else 2),
           "atom_updates_per_s": na * args.steps * world / (ms * 1e-3),
           "lattice_kernel_mlups": nodes / (lb_ms * 1e-3) / 1e6,
           "clocks": clk.result}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(cfg, inp)
    if world == 1 and not args.no_adjoint:
        out["adjoint"] = adjoint_timing(stream)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    lbmd.lbmd_destroy(h)
    return out if rank == 0 else None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--store", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the timing of the adjoint workload")
    args = ap.parse_args()
    overrides = dict(DEFAULT_OVERRIDES)
    overrides["store"] = args.store
    cfg = synth.workload(args.workload, **overrides)
    if args.impl == "reference":
        world, rank, _ = _dist()
        if rank != 0:
            return
        # Each oracle step of the 128^3 workload takes ~10 s on one core: at
        # most 10 timed steps after at most 1 warm-up keep the run near two
        # minutes (the line reports the steps actually taken).
        args.steps = min(args.steps, 10)
        args.warmup = min(args.warmup, 1)
        out = run_reference(args, cfg)
    else:
        out = run_ours(args, cfg)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
