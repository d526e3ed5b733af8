"""GPU thermal noise (the xi_i of the fluctuating lattice-Boltzmann source
term S_i = p_i + xi_i, Sec. 2.2) against the FP64 oracle: element by element
(both sides draw the same Philox integers and the same 23-bit uniforms; the
Gaussians differ only by the FP32 rounding of log, sqrt, sin and cos), on the
lattice alone in all storage formats and in a coupled step (the sparse
fix-up must add the same noise as the dense kernel), then statistically:
equipartition of the fluctuating fluid at rest."""
import numpy as np
import pytest

from paper_2305_05025_gb300 import build, lbmd, synth
from gpu_helpers import floor_bound, fp32_floor, lattice_inputs, make, oracle_start, rel_linf, report_ratios, \
    step_errors, velocity

pytestmark = pytest.mark.gpu

TOL = 1e-5
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)[:, None]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbmd.lib()


def _thermal(cfg, inp):
    h = make(cfg, inp)
    lbmd.lbmd_set_thermal(h, cfg["kT"], cfg["seed"])
    return h


@pytest.mark.parametrize("store,bound", [("f32", TOL), ("f16", 2e-3), ("bf16", 2e-2)])
def test_noisy_lattice_matches_oracle(orc, store, bound):
    cfg = dict(synth._COMMON, nx=20, ny=18, nz=16, tau=0.7, forcing="kolmogorov", force_amp=1e-4, store=store,
               kT=1e-5, seed=0x1234567890ABCDEF)
    inp = lattice_inputs((20, 18, 16), 0.005, 11)
    h = _thermal(cfg, inp)
    f, _, _, topo = oracle_start(orc, cfg, inp)
    lbmd.lbmd_step(h, 20)
    g = lbmd.lbmd_get_fields(h, f=True, u=True)
    fo, _, _, _ = orc.run(cfg, topo, f, np.zeros((3, 0)), np.zeros((3, 0)), 20)
    uo = velocity(orc, cfg, fo)
    e_f, e_df, e_u = rel_linf(g["f"], fo), rel_linf(g["f"] - W, fo - W), rel_linf(g["u"], uo)
    print(f"noisy lattice {store}: f {e_f:.2e} delta f {e_df:.2e} u {e_u:.2e}")
    # the noise moved the fluid well beyond the deterministic flow
    fd, _, _, _ = orc.run(dict(cfg, kT=0.0), topo, f, np.zeros((3, 0)), np.zeros((3, 0)), 20)
    assert rel_linf(fd, fo) > 1e-4
    if store == "f32":
        assert e_f < TOL and e_u < TOL
    else:
        assert e_df < bound and e_u < bound


def test_noisy_coupled_step_matches_oracle(orc):
    """Coupled steps with noise: the touched nodes are re-collided by the
    sparse fix-up, which must add the same xi_i as the dense kernel. Checked
    on the first step and, from the GPU's state, on the fourth (oracle step
    index 3)."""
    cfg = synth.workload("chain500_lattice32", n_md=128, gamma=0.05, skin=0.3, kT=1e-6, seed=77)
    inp = synth.inputs(cfg, 1)
    h = _thermal(cfg, inp)
    f, x, v, topo = oracle_start(orc, cfg, inp)
    floors, (fo, xo, vo) = fp32_floor(orc, cfg, topo, f, x, v, 1)
    lbmd.lbmd_step(h, 1)
    s = lbmd.lbmd_get_fields(h, f=True, u=True, x=True, v=True)
    errs = step_errors(orc, cfg, s, fo, xo, vo)
    report_ratios("noisy coupled step 0", errs, floors)
    for k, e in errs.items():
        assert e <= floor_bound(cfg, floors[k]), (k, e, floors[k])
    lbmd.lbmd_step(h, 2)
    s = lbmd.lbmd_get_fields(h, f=True, x=True, v=True)
    c3 = dict(cfg, step0=3)
    floors, (fo, xo, vo) = fp32_floor(orc, c3, topo, s["f"].astype(np.float64), s["x"], s["v"].astype(np.float64), 1)
    lbmd.lbmd_step(h, 1)
    s = lbmd.lbmd_get_fields(h, f=True, u=True, x=True, v=True)
    errs = step_errors(orc, c3, s, fo, xo, vo)
    report_ratios("noisy coupled step 3", errs, floors)
    for k, e in errs.items():
        assert e <= floor_bound(cfg, floors[k]), (k, e, floors[k])
    lbmd.lbmd_check(h)


@pytest.mark.parametrize("store", ["f32", "f16"])
def test_equipartition(store):
    """A 32^3 periodic fluid at rest with kT = 1e-4, tau = 1: after 100 steps
    the density variance is rho0 kT / c_s^2 and each momentum component's
    rho0 kT (1 - 1/N) (total momentum stays zero), within 3%."""
    kT, n = 1e-4, 32
    cfg = dict(synth._COMMON, nx=n, ny=n, nz=n, tau=1.0, store=store)
    h = make(cfg, lattice_inputs((n, n, n), 0.0, 1))
    lbmd.lbmd_set_thermal(h, kT, 2024)
    lbmd.lbmd_step(h, 100)
    rv, jv = [], []
    for _ in range(100):
        lbmd.lbmd_step(h, 3)
        g = lbmd.lbmd_get_fields(h, rho=True, u=True)
        rho = g["rho"].astype(np.float64)
        rv.append(((rho - 1.0) ** 2).mean())
        jv.append(((rho * g["u"]) ** 2).mean())
    N = n ** 3
    r_rho, r_j = np.mean(rv) / (3 * kT), np.mean(jv) / (kT * (1 - 1 / N))
    print(f"equipartition {store}: density {r_rho:.4f}, momentum {r_j:.4f} of the expected variance")
    assert abs(r_rho - 1) < 0.03 and abs(r_j - 1) < 0.03
    # Mass and total momentum stay put up to FP32 rounding (uncorrelated
    # noise would have moved the total momentum by sqrt(N rho0 kT) ~ 2).
    m, pf, _ = lbmd.lbmd_get_stats(h)
    print(f"equipartition {store}: mass drift {m - N:.2e}, total momentum {np.abs(pf).max():.2e}")
    if store == "f32":
        assert abs(m - N) < 1e-4 and np.abs(pf).max() < 1e-4


def test_noise_is_reproducible_and_seeded():
    cfg = dict(synth._COMMON, nx=24, ny=8, nz=8, tau=0.8)
    inp = lattice_inputs((24, 8, 8), 0.0, 1)
    out = []
    for seed in (5, 5, 6):
        h = make(cfg, inp)
        lbmd.lbmd_set_thermal(h, 1e-5, seed)
        lbmd.lbmd_step(h, 5)
        out.append(lbmd.lbmd_get_fields(h, f=True)["f"])
    assert np.array_equal(out[0], out[1])
    assert not np.array_equal(out[0], out[2])
    # kT = 0 turns it off again: the rest state stays exact
    h = make(cfg, inp)
    lbmd.lbmd_set_thermal(h, 1e-5, 5)
    lbmd.lbmd_set_thermal(h, 0.0, 5)
    lbmd.lbmd_step(h, 5)
    assert np.array_equal(lbmd.lbmd_get_fields(h, f=True)["f"], np.repeat(W.astype(np.float32), 24 * 64, axis=1))


def test_adjoint_refuses_noise():
    cfg = synth.workload("chain500_lattice32", nx=12, ny=12, nz=12, n_md=16,
                         chains=[dict(n=20, centre="box", radius=None)])
    inp = synth.inputs(cfg, 1)
    inp["x"] = inp["x"] - inp["x"].mean(1, keepdims=True) + 6.0
    h = make(cfg, inp)
    lbmd.lbmd_set_thermal(h, 1e-6, 1)
    with pytest.raises(lbmd.LBMDError) as e:
        lbmd.lbmd_backward(h, 2, 1)
    assert e.value.status == lbmd.LBMD_ERR_ARG
    with pytest.raises(lbmd.LBMDError):
        lbmd.lbmd_set_thermal(h, -1.0, 1)
