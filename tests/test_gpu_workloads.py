"""GPU checks at the sizes of the benchmark workloads, in the configuration
bench.py times (one CUDA graph per step, n_md = 128, gamma = 0.05, skin 0.3):

- 128^3 / 20k-bead globule: per-step (teacher-forced) parity with the oracle
  for two steps, and mass / momentum balance over twenty steps;
- 256^3 / 60k-bead trimer: one step in FP32, FP16 and BF16 storage against the
  oracle, with the per-field error table (f - w rho0, rho - rho0, u, x, v);
- 512^3 z-channel with ten globules: FP32 and FP16 storage run, no flag
  raised, mass kept, and the FP16-vs-FP32 difference per field after one
  step."""
import numpy as np
import pytest

from paper_2305_05025_gb300 import build, lbmd, synth
from gpu_helpers import floor_bound, fp32_floor, make, rel_linf, report_ratios, step_errors, velocity

pytestmark = pytest.mark.gpu

BENCH = dict(n_md=128, gamma=0.05, skin=0.3)
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbmd.lib()


def _rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.sqrt((b * b).sum())
    return float(np.sqrt(((a - b) ** 2).sum()) / den) if den > 0 else float(np.sqrt(((a - b) ** 2).sum()))


def _fields(h):
    return lbmd.lbmd_get_fields(h, f=True, rho=True, u=True, x=True, v=True)


def _table(name, s, fo, xo, vo, cfg, orc):
    rho_o, _ = orc.moments(fo)
    uo = velocity(orc, cfg, fo)
    rows = dict(df=(s["f"] - W[:, None], fo - W[:, None]), drho=(s["rho"] - 1.0, rho_o - 1.0), u=(s["u"], uo),
                x=(s["x"], xo), v=(s["v"], vo))
    out = {}
    for k, (a, b) in rows.items():
        out[k] = (rel_linf(a, b), _rel_l2(a, b))
    print(name, " ".join(f"{k}: Linf {e[0]:.2e} L2 {e[1]:.2e}" for k, e in out.items()))
    return out


def test_globule20k_lattice128_teacher_forced(orc):
    cfg = synth.workload("globule20k_lattice128", **BENCH)
    inp = synth.inputs(cfg, 1)
    h = make(cfg, inp)
    topo = orc.Topology(inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"])
    s = lbmd.lbmd_get_fields(h, f=True, x=True, v=True)
    for n in range(2):
        floors, (fo, xo, vo) = fp32_floor(orc, cfg, topo, s["f"].astype(np.float64), s["x"],
                                          s["v"].astype(np.float64), 1, seed=n)
        lbmd.lbmd_step(h, 1)
        s = _fields(h)
        _table(f"128^3 step {n}", s, fo, xo, vo, cfg, orc)
        errs = step_errors(orc, cfg, s, fo, xo, vo)
        report_ratios(f"globule20k 128^3 step {n}", errs, floors)
        for key, e in errs.items():
            bound = floor_bound(cfg, floors[key])
            assert e <= bound, (n, key, e, bound)
    lbmd.lbmd_check(h)


def test_globule20k_lattice128_balances():
    """Kolmogorov forcing sums to zero over the box: the total momentum stays
    put and the mass is kept, over twenty graph steps at full size."""
    cfg = synth.workload("globule20k_lattice128", **BENCH)
    inp = synth.inputs(cfg, 1)
    h = make(cfg, inp)
    m0, pf0, pa0 = lbmd.lbmd_get_stats(h)
    lbmd.lbmd_step(h, 20)
    m1, pf1, pa1 = lbmd.lbmd_get_stats(h)
    dP = (pf1 + pa1) - (pf0 + pa0)
    print("mass drift", m1 - m0, "momentum change", dP, "solute momentum", pa1)
    assert abs(m1 - m0) < 1e-7 * m0
    assert np.abs(dP).max() < 1e-4 * max(1.0, np.abs(pa1 - pa0).max())


def test_trimer60k_lattice256_storage_formats(orc):
    cfg32 = synth.workload("trimer60k_lattice256", **BENCH)
    inp = synth.inputs(cfg32, 1)
    topo = orc.Topology(inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"])
    f0 = orc.equilibrium(inp["rho"].astype(np.float32).astype(np.float64),
                         inp["u"].astype(np.float32).astype(np.float64))
    floors, (fo, xo, vo) = fp32_floor(orc, cfg32, topo, f0, inp["x"], inp["v"].astype(np.float64), 1)
    bounds = dict(f32=None, f16=2e-3, bf16=2e-2)
    for store in ("f32", "f16", "bf16"):
        cfg = dict(cfg32, store=store)
        h = make(cfg, inp)
        lbmd.lbmd_step(h, 1)
        lbmd.lbmd_check(h)
        s = _fields(h)
        errs = _table(f"256^3 trimer {store}", s, fo, xo, vo, cfg, orc)
        if store == "f32":
            report_ratios("trimer60k 256^3 f32 one step", step_errors(orc, cfg, s, fo, xo, vo), floors)
            assert rel_linf(s["f"], fo) <= floor_bound(cfg, floors["f"])
            assert errs["x"][0] <= floor_bound(cfg, floors["x"])
        else:
            assert errs["df"][0] <= bounds[store] and errs["u"][0] <= bounds[store]
            assert errs["x"][0] <= 1e-5
        lbmd.lbmd_destroy(h)


def test_channel10x20k_lattice512_runs():
    """FP16 against FP32 storage after one coupled step (the dense collapsing
    globules are chaotic: a second step already amplifies the storage
    difference in the atom positions by orders of magnitude), then one more
    step each with no flag raised and mass kept."""
    cfg32 = synth.workload("channel10x20k_lattice512", **BENCH)
    inp = synth.inputs(cfg32, 1)
    res = {}
    for store in ("f32", "f16"):
        cfg = dict(cfg32, store=store)
        h = make(cfg, inp)
        m0, _, _ = lbmd.lbmd_get_stats(h)
        lbmd.lbmd_step(h, 1)
        lbmd.lbmd_check(h)
        res[store] = lbmd.lbmd_get_fields(h, u=True, x=True, v=True)
        lbmd.lbmd_step(h, 1)
        lbmd.lbmd_check(h)
        m1, _, _ = lbmd.lbmd_get_stats(h)
        assert abs(m1 - m0) < 1e-7 * m0, (store, m1 - m0)
        lbmd.lbmd_destroy(h)
    # FP16 resolution of delta f (2^-11 relative) in u; x and v see it only
    # through the friction with the interpolated u.
    bounds = dict(u=1e-2, x=1e-6, v=2e-3)
    for k, b in bounds.items():
        e = rel_linf(res["f16"][k], res["f32"][k])
        print(f"512^3 channel FP16 vs FP32 after one step, {k}: rel Linf {e:.2e}, "
              f"max |FP32| {np.abs(res['f32'][k]).max():.2e}")
        assert e < b, (k, e)
