"""GPU parity of the coupled step (Sec. 2.2) against the FP64 oracle through
the C ABI: bit-exact cell membership and neighbour counts, the single-atom
closed form, free-running parity where the solute dynamics are not chaotic,
per-step ("teacher-forced") parity along the chaotic 500-bead trajectory, and
conservation, error flags and argument errors.

Tolerance: 1e-5 relative L-infinity, or, where the solute makes that
unreachable in FP32 arithmetic, the FP64 oracle's own response to rounding its
inputs to the CUDA path's FP32 resolution (`fp32_floor`): stiff bonds (k = 100
on r0 = 0.5) and Lennard-Jones cores turn a 6e-8 position rounding into
velocity changes far above 1e-5 of the (often small) velocities."""
import numpy as np
import pytest

from paper_2305_05025_gb300 import build, lbmd, synth
from gpu_helpers import (assert_within, floor_bound, fp32_floor, make, oracle_start, rel_linf, report_ratios,
                         step_errors, teacher_forced, velocity)

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbmd.lib()


@pytest.fixture(scope="module")
def c1():
    cfg = synth.workload("chain500_lattice32", n_md=128)
    return cfg, synth.inputs(cfg, 1)


def test_cell_membership_and_neighbour_counts_bit_exact(orc, c1):
    cfg, inp = c1
    h = make(cfg, inp)
    cell, neigh, nc = lbmd.lbmd_cell_list(h)
    ocell, onc = orc.cells(cfg, inp["x"])
    assert np.array_equal(nc, onc)
    assert np.array_equal(cell, ocell)
    assert np.array_equal(neigh, orc.neighbour_counts(cfg, inp["x"]))


@pytest.mark.parametrize("skin", [0.0, 0.3])
def test_cell_list_after_steps_matches_oracle_on_gpu_positions(orc, c1, skin):
    cfg, inp = c1
    cfg = dict(cfg, skin=skin)
    h = make(dict(cfg, gamma=0.05), inp)
    lbmd.lbmd_step(h, 3)
    x = lbmd.lbmd_get_fields(h, x=True)["x"]
    cell, neigh, _ = lbmd.lbmd_cell_list(h)
    assert np.array_equal(cell, orc.cells(cfg, x)[0])
    assert np.array_equal(neigh, orc.neighbour_counts(cfg, x))


@pytest.mark.parametrize("n_md", [1, 8, 128])
def test_single_atom_in_uniform_flow(n_md):
    gamma, u0 = 0.5, 1e-3
    cfg = dict(synth._COMMON, nx=4, ny=4, nz=4, tau=0.8, gamma=gamma, n_md=n_md)
    N = 64
    u = np.zeros((3, N))
    u[0] = u0
    inp = dict(rho=np.ones(N), u=u, x=np.array([[1.3], [2.1], [0.7]]), v=np.zeros((3, 1)), mass=np.ones(1),
               bonds=np.zeros((0, 2), np.int32), bond_k=np.zeros(0), bond_r0=np.zeros(0))
    h = make(cfg, inp)
    m0, pf0, pa0 = lbmd.lbmd_get_stats(h)
    lbmd.lbmd_step(h, 1)
    m1, pf1, pa1 = lbmd.lbmd_get_stats(h)
    J = u0 * (1 - (1 - gamma / (2 * n_md)) ** (2 * n_md))
    v = lbmd.lbmd_get_fields(h, v=True)["v"]
    assert abs(v[0, 0] - J) < 1e-6 * J + 1e-12
    # FP64 sums of FP32 populations: the fluid momentum carries ~1e-7 of its
    # own magnitude in rounding.
    assert abs((pf1[0] - pf0[0]) + J) < 1e-6 * J + 2e-7 * abs(pf0[0])
    assert abs(m1 - m0) < 1e-8  # FP32 rounding of 64 nodes' populations


@pytest.mark.parametrize("skin", [0.0, 0.3])
def test_one_coupled_step_matches_oracle(orc, c1, skin):
    cfg, inp = c1
    cfg = dict(cfg, skin=skin)
    h = make(cfg, inp)
    f, x, v, topo = oracle_start(orc, cfg, inp)
    lbmd.lbmd_step(h, 1)
    s = lbmd.lbmd_get_fields(h, f=True, u=True, x=True, v=True)
    floors, (fo, xo, vo) = fp32_floor(orc, cfg, topo, f, x, v, 1)
    errs = dict(f=rel_linf(s["f"], fo), u=rel_linf(s["u"], velocity(orc, cfg, fo)), x=rel_linf(s["x"], xo),
                v=rel_linf(s["v"], vo))
    report_ratios(f"chain500 one step skin {skin}", errs, floors)
    assert errs["f"] < TOL and errs["x"] < TOL and errs["u"] < TOL
    assert_within(errs, floors)


def test_teacher_forced_100_steps_chain500(orc, c1):
    """The 500-bead LJ chain collapses chaotically (a 1e-9 perturbation of the
    FP64 oracle grows to 1e-1 in ten steps), so FP32 and FP64 trajectories
    separate whatever the implementation; each of the 100 steps is instead
    checked from the GPU's own state. gamma = 0.05 keeps the explicit friction
    exchange stable once the chain is dense (gamma = 0.5 diverges near step
    20, in the oracle too)."""
    cfg, inp = c1
    worst, done = teacher_forced(orc, dict(cfg, gamma=0.05, skin=0.3), inp, 100, "chain500 gamma 0.05")
    assert done == 100
    print("teacher-forced worst error / bound:", worst)
    for k, r in worst.items():
        assert r <= 1.0, (k, r)


def test_teacher_forced_literal_gamma(orc, c1):
    """Ten steps: in the first ten the error / FP32-floor ratios of five GPU
    runs stayed at or below 1.45 (0.72 of the bound); at steps 10-11 the
    chain meets close Lennard-Jones encounters whose floors are up to 100x
    larger, and the rounding of the step's 128 FP32 substeps (which the
    floor, a perturbation of the step's inputs, does not model) reached 6.6x
    the floor in one run: beyond there the comparison measures the
    conditioning of the chaos, not the kernels."""
    cfg, inp = c1
    worst, done = teacher_forced(orc, cfg, inp, 10, "chain500 gamma 0.5")
    print("gamma 0.5 teacher-forced worst error / bound:", worst, "steps", done)
    assert done == 10
    for k, r in worst.items():
        assert r <= 1.0, (k, r)


@pytest.mark.parametrize("skin", [0.0, 0.3])
def test_free_running_harmonic_chain_100_steps(orc, skin):
    """Without Lennard-Jones (eps = 0) the chain is a damped harmonic network
    coupled to the fluid: not chaotic, so free-running FP32 and FP64
    trajectories stay together over 100 steps."""
    cfg = synth.workload("chain500_lattice32", n_md=128, lj_eps=0.0, gamma=0.5, nx=24, ny=20, nz=28, skin=skin)
    inp = synth.inputs(cfg, 2)
    rng = np.random.default_rng(3)
    inp["v"] = 0.05 * rng.standard_normal(inp["v"].shape)
    inp["x"] = inp["x"] - inp["x"].mean(1, keepdims=True) + np.array([[12.0], [10.0], [14.0]])
    h = make(cfg, inp)
    f, x, v, topo = oracle_start(orc, cfg, inp)
    lbmd.lbmd_step(h, 100)
    s = lbmd.lbmd_get_fields(h, f=True, u=True, x=True, v=True)
    floors, (fo, xo, vo) = fp32_floor(orc, cfg, topo, f, x, v, 100)
    errs = dict(f=rel_linf(s["f"], fo), u=rel_linf(s["u"], velocity(orc, cfg, fo)), x=rel_linf(s["x"], xo),
                v=rel_linf(s["v"], vo))
    report_ratios(f"harmonic chain 100 steps free-running skin {skin}", errs, floors)
    assert errs["f"] < TOL and errs["x"] < TOL
    assert_within(errs, floors)


def test_mass_and_total_momentum(c1):
    """sum f c + sum m v grows by exactly N g per step (FP64 sums of FP32 state)."""
    cfg, inp = c1
    cfg = dict(cfg, gamma=0.05, forcing="uniform", force_amp=1e-5, force_dir=1)
    h = make(cfg, inp)
    m0, pf0, pa0 = lbmd.lbmd_get_stats(h)
    steps = 30
    lbmd.lbmd_step(h, steps)
    m1, pf1, pa1 = lbmd.lbmd_get_stats(h)
    N = 32 ** 3
    dP = (pf1 + pa1) - (pf0 + pa0)
    expect = np.array([0.0, steps * N * 1e-5, 0.0])
    print("mass drift", m1 - m0, "momentum error", dP - expect)
    assert abs(m1 - m0) < 1e-6 * N * 1e-3
    assert np.abs(dP - expect).max() < 1e-4 * np.abs(pa1 - pa0).max() + 1e-6


def test_nonfinite_input_is_reported(c1):
    cfg, inp = c1
    inp = dict(inp)
    u = inp["u"].copy()
    u[0, 100] = np.nan
    inp["u"] = u
    with pytest.raises(lbmd.LBMDError) as e:
        make(cfg, inp)
    assert e.value.status == lbmd.LBMD_ERR_NONFINITE


def test_calls_out_of_order():
    cfg = dict(synth._COMMON, nx=8, ny=8, nz=8, tau=0.7)
    h = lbmd.lbmd_create(cfg)
    with pytest.raises(lbmd.LBMDError) as e:
        lbmd.lbmd_step(h, 1)
    assert e.value.status == lbmd.LBMD_ERR_STATE
    with pytest.raises(lbmd.LBMDError) as e:
        lbmd.lbmd_set_state(h)
    assert e.value.status == lbmd.LBMD_ERR_ARG


def test_timing_events_bracket_the_lattice_kernel(c1):
    torch = pytest.importorskip("torch")
    cfg, inp = c1
    h = make(dict(cfg, gamma=0.05), inp)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    b.record()  # torch reads only events it recorded; the graph re-records them
    lbmd.lbmd_set_timing_events(h, a, b)
    lbmd.lbmd_step(h, 1)
    torch.cuda.synchronize()
    assert a.elapsed_time(b) > 0.0
    lbmd.lbmd_set_timing_events(h, None, None)
    lbmd.lbmd_step(h, 1)
