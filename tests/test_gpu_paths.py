"""GPU parity with the FP64 oracle on the code paths and edge cases that the
workload tests alone would leave unreached:

- the 512^3 channel's kernel path on a lattice the oracle steps in seconds:
  more than 65,536 atoms (four lanes per atom in the substep kernel), a box
  side above 166 (coarse pair-search cells searched 3x3x3), z walls, and flat
  chains whose interpolation stencils touch the first and the last pair of
  fluid planes; FP32 (two steps, each from the GPU's own state) and FP16
  storage (one step);
- a chain across all three periodic seams, with positions given unwrapped
  (negative coordinates) and wrapped into the box (bonded neighbours a box
  length apart in the raw coordinates);
- a chain with random masses in [0.5, 2] (the friction gamma (u - v) is a
  force: a per-mass reading of gamma would differ).

Bounds: max(1e-5, FLOOR_FACTOR x the oracle's response to one FP32 rounding
of the step's inputs) per field, as in the other coupled tests; for FP16
storage the storage resolution of delta f (2^-11 relative, bound 2e-3)."""
import numpy as np
import pytest

from paper_2305_05025_gb300 import build, lbmd, synth
from gpu_helpers import (floor_bound, fp32_floor, make, oracle_start, rel_linf, report_ratios, step_errors,
                         teacher_forced, velocity)

pytestmark = pytest.mark.gpu

BENCH = dict(n_md=128, gamma=0.05, skin=0.1)  # bench.py's defaults
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbmd.lib()


def test_channel_code_path_matches_oracle(orc):
    cfg32 = synth.workload("channel4x17k_lattice176x48x48", **BENCH)
    inp = synth.inputs(cfg32, 1)
    na = inp["x"].shape[1]
    # The instantiation the 512^3 channel runs: > 65,536 atoms and a box side
    # with more than 256 half-size cells (coarse 3x3x3 search).
    assert na > 65536
    side = (cfg32["lj_sigma"] * cfg32["lj_rcut_over_sigma"] + cfg32["skin"]) / 2
    assert max(np.floor(cfg32[k] / side) for k in ("nx", "ny", "nz")) > 256
    # Flat chains on z = 0.5 and z = nz - 1.5: stencils on planes 0-1 and nz-2..nz-1.
    zs = inp["x"][2]
    assert np.any(np.floor(zs) == 0) and np.any(np.floor(zs) == cfg32["nz"] - 2)

    f0, x0, v0, topo = oracle_start(orc, cfg32, inp)
    floors, (fo, xo, vo) = fp32_floor(orc, cfg32, topo, f0, x0, v0, 1)

    # FP16 storage, one step from the same start.
    h16 = make(dict(cfg32, store="f16"), inp)
    lbmd.lbmd_step(h16, 1)
    lbmd.lbmd_check(h16)
    s = lbmd.lbmd_get_fields(h16, f=True, u=True, x=True, v=True)
    e16 = dict(df=rel_linf(s["f"] - W[:, None], fo - W[:, None]), u=rel_linf(s["u"], velocity(orc, cfg32, fo)),
               x=rel_linf(s["x"], xo), v=rel_linf(s["v"], vo))
    print("channel path FP16 one step:", {k: f"{e:.3e}" for k, e in e16.items()})
    lbmd.lbmd_destroy(h16)
    assert e16["df"] <= 2e-3 and e16["u"] <= 2e-3
    assert e16["x"] <= floor_bound(cfg32, floors["x"])
    # v sees the FP16 storage only through the friction with the interpolated u.
    assert e16["v"] <= max(2e-3, floor_bound(cfg32, floors["v"]))

    # FP32: the first step from the common start, then one more from the
    # GPU's own state.
    h = make(cfg32, inp)
    lbmd.lbmd_step(h, 1)
    s = lbmd.lbmd_get_fields(h, f=True, u=True, x=True, v=True)
    errs = step_errors(orc, cfg32, s, fo, xo, vo)
    report_ratios("channel path f32 step 0", errs, floors)
    for k, e in errs.items():
        assert e <= floor_bound(cfg32, floors[k]), (k, e, floors[k])
    lbmd.lbmd_check(h)
    worst, done = teacher_forced(orc, cfg32, inp, 1, "channel path f32 step 1", h=h)
    assert done == 1
    for k, r in worst.items():
        assert r <= 1.0, (k, r)
    # The wall-side chains stay on their planes (no force has a z part there).
    x = lbmd.lbmd_get_fields(h, x=True)["x"]
    assert np.abs(x[2, -600:] - inp["x"][2, -600:]).max() < 1e-6


@pytest.mark.parametrize("wrapped", [False, True])
def test_chain_across_periodic_seams(orc, wrapped):
    cfg = synth.workload("chain500_lattice32", **BENCH)
    inp = dict(synth.inputs(cfg, 1))
    box = np.array([[cfg["nx"]], [cfg["ny"]], [cfg["nz"]]], float)
    x = inp["x"] - inp["x"].mean(1, keepdims=True)  # centred on the corner (0, 0, 0) of the box
    if wrapped:
        x = np.mod(x, box)
        # Some bonded neighbours sit a box length apart in the raw coordinates.
        b = inp["bonds"]
        assert np.abs(x[:, b[:, 0]] - x[:, b[:, 1]]).max() > 0.5 * box.min()
    else:
        assert (x < 0).any(axis=1).all() and (x > 0).any(axis=1).all()
    inp["x"] = x
    worst, done = teacher_forced(orc, cfg, inp, 10, f"seams wrapped={wrapped}")
    assert done == 10
    for k, r in worst.items():
        assert r <= 1.0, (k, r)


def test_chain_with_random_masses(orc):
    cfg = synth.workload("chain500_lattice32", **BENCH)
    inp = dict(synth.inputs(cfg, 1))
    inp["mass"] = np.random.default_rng(31).uniform(0.5, 2.0, inp["x"].shape[1])
    worst, done = teacher_forced(orc, cfg, inp, 10, "random masses")
    assert done == 10
    for k, r in worst.items():
        assert r <= 1.0, (k, r)
    # The masses matter: the same chain with unit masses ends elsewhere.
    h1 = make(cfg, dict(inp, mass=np.ones(inp["x"].shape[1])))
    lbmd.lbmd_step(h1, 2)
    h2 = make(cfg, inp)
    lbmd.lbmd_step(h2, 2)
    assert rel_linf(lbmd.lbmd_get_fields(h1, v=True)["v"], lbmd.lbmd_get_fields(h2, v=True)["v"]) > 1e-2
