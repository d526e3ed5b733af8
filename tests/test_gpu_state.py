"""Raw state snapshots (lbmd_save_state / lbmd_load_state): the lattice in
its storage format and the atoms, restored bit for bit, for every storage
format, from host and from device buffers; the restored handle continues the
trajectory (to rounding: the first forces are recomputed from the positions,
in another summation order than the substep that cached them)."""
import numpy as np
import pytest

from paper_2305_05025_gb300 import build, lbmd, synth
from gpu_helpers import make, rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbmd.lib()


def _cfg(store):
    # A harmonic bead network (no Lennard-Jones) in a Kolmogorov flow, so the
    # continuation after a restore can be compared near rounding: in the
    # FP64 oracle a 1e-7 relative perturbation at step 3 moves f by 6e-8, x
    # by 1.3e-7 and v by 2.5e-4 two steps later (the Lennard-Jones chain
    # turns even 1e-9 into a 23 % velocity difference).
    return synth.workload("chain500_lattice32", n_md=128, gamma=0.05, skin=0.3, lj_eps=0.0, store=store,
                          forcing="kolmogorov", force_amp=1e-5)


@pytest.mark.parametrize("store", ["f32", "f16", "bf16"])
def test_snapshot_round_trip_from_host(store):
    cfg = _cfg(store)
    inp = dict(synth.inputs(cfg, 3))
    inp["v"] = 0.05 * np.random.default_rng(3).standard_normal(inp["v"].shape)
    h1 = make(cfg, inp)
    lbmd.lbmd_step(h1, 3)
    snap = lbmd.lbmd_save_state(h1)
    assert snap["pop"].dtype == (np.float32 if store == "f32" else np.uint16)
    before = lbmd.lbmd_get_fields(h1, f=True, rho=True, u=True, x=True, v=True)
    h2 = make(cfg, inp)  # another state first: the load replaces all of it
    lbmd.lbmd_step(h2, 1)
    lbmd.lbmd_load_state(h2, snap["pop"], snap["x"], snap["v"])
    again = lbmd.lbmd_save_state(h2)
    for k in ("pop", "x", "v"):
        assert np.array_equal(again[k], snap[k]), k
    after = lbmd.lbmd_get_fields(h2, f=True, rho=True, u=True, x=True, v=True)
    for k in before:
        assert np.array_equal(after[k], before[k]), k
    # Both handles continue: the same trajectory up to rounding.
    lbmd.lbmd_step(h1, 2)
    lbmd.lbmd_step(h2, 2)
    a = lbmd.lbmd_get_fields(h1, f=True, x=True, v=True)
    b = lbmd.lbmd_get_fields(h2, f=True, x=True, v=True)
    errs = {k: rel_linf(b[k], a[k]) for k in a}
    print(f"snapshot continuation ({store}):", {k: f"{e:.2e}" for k, e in errs.items()})
    assert errs["f"] < 1e-5 and errs["x"] < 1e-5 and errs["v"] < 1e-2
    lbmd.lbmd_check(h2)


def test_snapshot_round_trip_on_device():
    torch = pytest.importorskip("torch")
    cfg = _cfg("f16")
    inp = synth.inputs(cfg, 4)
    h1 = make(cfg, inp)
    lbmd.lbmd_step(h1, 2)
    N, na = 32 ** 3, inp["x"].shape[1]
    out = {"pop": torch.empty(19 * N, dtype=torch.int16, device="cuda"),
           "x": torch.empty((3, na), dtype=torch.float64, device="cuda"),
           "v": torch.empty((3, na), dtype=torch.float32, device="cuda")}
    lbmd.lbmd_save_state(h1, out=out)
    torch.cuda.synchronize()
    host = lbmd.lbmd_save_state(h1)
    assert np.array_equal(out["pop"].cpu().numpy().view(np.uint16).reshape(19, N), host["pop"])
    h2 = make(cfg, inp)
    lbmd.lbmd_load_state(h2, out["pop"], out["x"], out["v"])
    assert np.array_equal(lbmd.lbmd_save_state(h2)["pop"], host["pop"])


def test_snapshot_argument_errors():
    cfg = _cfg("f32")
    inp = synth.inputs(cfg, 1)
    h = lbmd.lbmd_create(cfg, inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"])
    with pytest.raises(lbmd.LBMDError) as e:
        lbmd.lbmd_save_state(h)
    assert e.value.status == lbmd.LBMD_ERR_STATE
    with pytest.raises(lbmd.LBMDError) as e:
        lbmd.lbmd_load_state(h, np.zeros((19, 32 ** 3), np.float32))  # atoms missing
    assert e.value.status == lbmd.LBMD_ERR_ARG
