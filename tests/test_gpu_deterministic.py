"""Deterministic mode (lbmd_params.deterministic = 1): two runs of the same
state give bit-identical states (the Verlet lists sorted by atom index, the
spread summed in exact fixed point per touched node, the set-up forces in
fixed point), on the 8-lane path with half-size cells and on the 4-lane path
with coarse cells, in FP32 and FP16 storage; the mode still matches the FP64
oracle step by step; it refuses what it does not cover."""
import numpy as np
import pytest

from paper_2305_05025_gb300 import build, lbmd, synth
from gpu_helpers import make, teacher_forced

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbmd.lib()


def _twice(cfg, inp, steps):
    snaps = []
    for _ in range(2):
        h = make(cfg, inp)
        lbmd.lbmd_step(h, steps)
        lbmd.lbmd_check(h)
        snaps.append(lbmd.lbmd_save_state(h))
        lbmd.lbmd_destroy(h)
    return snaps


@pytest.mark.parametrize("store", ["f32", "f16"])
def test_chain_runs_are_bit_identical(store):
    cfg = synth.workload("chain500_lattice32", n_md=128, gamma=0.05, skin=0.3, store=store, deterministic=1)
    inp = synth.inputs(cfg, 1)
    a, b = _twice(cfg, inp, 6)
    for k in ("pop", "x", "v"):
        assert np.array_equal(a[k], b[k]), k
    assert np.abs(a["x"] - inp["x"]).max() > 1e-3  # the atoms did move


def test_channel_path_runs_are_bit_identical():
    """More than 65,536 atoms (4 lanes per atom), coarse cells, z walls."""
    cfg = synth.workload("channel4x17k_lattice176x48x48", n_md=128, gamma=0.05, skin=0.1, store="f16",
                         deterministic=1)
    inp = synth.inputs(cfg, 1)
    assert inp["x"].shape[1] > 65536
    a, b = _twice(cfg, inp, 3)
    for k in ("pop", "x", "v"):
        assert np.array_equal(a[k], b[k]), k


def test_deterministic_mode_matches_the_oracle(orc):
    cfg = synth.workload("chain500_lattice32", n_md=128, gamma=0.05, skin=0.3, deterministic=1)
    inp = synth.inputs(cfg, 1)
    worst, done = teacher_forced(orc, cfg, inp, 5, "deterministic chain500")
    assert done == 5
    for k, r in worst.items():
        assert r <= 1.0, (k, r)


def test_deterministic_mode_refusals():
    cfg = synth.workload("chain500_lattice32", n_md=16, gamma=0.05, skin=0.3, deterministic=1)
    inp = synth.inputs(cfg, 1)
    h = make(cfg, inp)
    with pytest.raises(lbmd.LBMDError) as e:
        lbmd.lbmd_set_reinterpolation(h, True)
    assert e.value.status == lbmd.LBMD_ERR_ARG
    with pytest.raises(lbmd.LBMDError) as e:
        lbmd.lbmd_backward(h, 2, 1)
    assert e.value.status == lbmd.LBMD_ERR_ARG
