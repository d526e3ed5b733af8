"""GPU discrete adjoint of the coupled step (lbmd_backward) against central
finite differences of the FP64 oracle with Richardson extrapolation: the
gradient of a time-averaged solute observable (mean drag along x, mean
squared radius of gyration) with respect to gamma, tau and the body-force
amplitude, through checkpointed segments (the last one partial)."""
import numpy as np
import pytest

from paper_2305_05025_gb300 import build, lbmd, synth
from gpu_helpers import make

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbmd.lib()


def _case(lj_eps, n_md, n_atoms, seed):
    cfg = synth.workload("chain500_lattice32", nx=12, ny=12, nz=12, tau=0.8, gamma=0.5, n_md=n_md, lj_eps=lj_eps,
                         forcing="uniform", force_amp=1e-4, force_dir=0, u_sigma=0.005,
                         chains=[dict(n=n_atoms, centre="box", radius=None)])
    inp = synth.inputs(cfg, seed)
    rng = np.random.default_rng(seed)
    inp["v"] = 0.02 * rng.standard_normal(inp["v"].shape)
    inp["x"] = inp["x"] - inp["x"].mean(1, keepdims=True) + 6.0
    return cfg, inp


def _oracle_obs(orc, cfg, inp, steps, observable):
    topo = orc.Topology(inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"])
    f = orc.equilibrium(inp["rho"].astype(np.float32).astype(np.float64),
                        inp["u"].astype(np.float32).astype(np.float64))
    _, _, _, obs = orc.run(cfg, topo, f, inp["x"], inp["v"].astype(np.float32).astype(np.float64), steps)
    return obs[:, 0].mean() if observable == lbmd.OBS_DRAG_X else obs[:, 3].mean()


def _fd(orc, cfg, inp, steps, observable, key, rel):
    """Richardson-extrapolated central difference of the oracle observable."""
    x0 = cfg[key]
    h = rel * abs(x0)

    def central(step):
        p = _oracle_obs(orc, dict(cfg, **{key: x0 + step}), inp, steps, observable)
        m = _oracle_obs(orc, dict(cfg, **{key: x0 - step}), inp, steps, observable)
        return (p - m) / (2 * step)

    d1, d2 = central(h), central(h / 2)
    return (4 * d2 - d1) / 3, abs(d2 - d1)


@pytest.mark.parametrize("observable", [lbmd.OBS_DRAG_X, lbmd.OBS_RG2])
def test_adjoint_matches_oracle_fd_harmonic_chain(orc, observable):
    cfg, inp = _case(lj_eps=0.0, n_md=16, n_atoms=30, seed=4)
    steps, ckpt = 12, 5
    h = make(cfg, inp)
    obs, dg, dtau, da = lbmd.lbmd_backward(h, steps, ckpt, observable)
    o_ref = _oracle_obs(orc, cfg, inp, steps, observable)
    assert abs(obs - o_ref) <= 1e-5 * abs(o_ref)
    got = dict(gamma=dg, tau=dtau, force_amp=da)
    for key, rel in (("gamma", 1e-3), ("tau", 1e-3), ("force_amp", 1e-2)):
        ref, spread = _fd(orc, cfg, inp, steps, observable, key, rel)
        print(f"obs {observable} d/d{key}: adjoint {got[key]:.8e} oracle FD {ref:.8e} (FD spread {spread:.1e})")
        assert abs(got[key] - ref) <= 1e-3 * abs(ref) + 3 * spread, key
    # The state ends advanced by n_steps, like lbmd_step(n_steps).
    x = lbmd.lbmd_get_fields(h, x=True)["x"]
    h2 = make(cfg, inp)
    lbmd.lbmd_step(h2, steps)
    assert np.abs(x - lbmd.lbmd_get_fields(h2, x=True)["x"]).max() < 1e-5


def test_adjoint_matches_oracle_fd_lennard_jones_short(orc):
    cfg, inp = _case(lj_eps=1.0, n_md=128, n_atoms=40, seed=5)
    steps, ckpt = 3, 2
    h = make(cfg, inp)
    obs, dg, dtau, da = lbmd.lbmd_backward(h, steps, ckpt, lbmd.OBS_DRAG_X)
    got = dict(gamma=dg, tau=dtau, force_amp=da)
    for key, rel in (("gamma", 1e-3), ("tau", 1e-3), ("force_amp", 1e-2)):
        ref, spread = _fd(orc, cfg, inp, steps, lbmd.OBS_DRAG_X, key, rel)
        print(f"LJ d/d{key}: adjoint {got[key]:.8e} oracle FD {ref:.8e} (FD spread {spread:.1e})")
        assert abs(got[key] - ref) <= 1e-3 * abs(ref) + 3 * spread, key


def test_autograd_function_returns_adjoint_gradients():
    torch = pytest.importorskip("torch")
    cfg, inp = _case(lj_eps=0.0, n_md=16, n_atoms=30, seed=4)
    h = make(cfg, inp)
    Fn = lbmd.observable_function()
    g = torch.tensor(cfg["gamma"], dtype=torch.float64, requires_grad=True)
    t = torch.tensor(cfg["tau"], dtype=torch.float64, requires_grad=True)
    a = torch.tensor(cfg["force_amp"], dtype=torch.float64, requires_grad=True)
    out = Fn.apply(g, t, a, h, 6, 3, lbmd.OBS_DRAG_X)
    (2.0 * out).backward()
    h2 = make(cfg, inp)
    _, dg, dtau, da = lbmd.lbmd_backward(h2, 6, 3, lbmd.OBS_DRAG_X)
    assert np.isclose(g.grad.item(), 2 * dg, rtol=1e-6)
    assert np.isclose(t.grad.item(), 2 * dtau, rtol=1e-6)
    assert np.isclose(a.grad.item(), 2 * da, rtol=1e-6)


def test_adjoint_full_size_matches_gpu_fd_chain5k_lattice64():
    """The adjoint workload at full size (64^3, 5,000-bead globule, uniform
    forcing 1e-5, 200 steps, checkpoints every 20) with harmonic bonds only:
    the Lennard-Jones globule is chaotic over 200 steps, so its exact
    derivative is dominated by exponential growth and has no converged finite
    difference. The adjoint must equal the Richardson central difference of
    the GPU's own forward observable (the same arithmetic it differentiates)."""
    cfg = synth.workload("chain5k_lattice64_uniform", lj_eps=0.0, n_md=128, skin=0.3)
    inp = synth.inputs(cfg, 1)
    steps, ckpt = cfg["steps"], cfg["ckpt_every"]
    h = make(cfg, inp)
    obs, dg, dtau, da = lbmd.lbmd_backward(h, steps, ckpt, lbmd.OBS_DRAG_X)
    lbmd.lbmd_destroy(h)
    got = dict(gamma=dg, tau=dtau, force_amp=da)

    def gpu_obs(key, value):
        hh = make(dict(cfg, **{key: value}), inp)
        o = lbmd.lbmd_backward(hh, steps, ckpt, lbmd.OBS_DRAG_X)[0]
        lbmd.lbmd_destroy(hh)
        return o

    for key, rel in (("gamma", 1e-2), ("tau", 1e-2), ("force_amp", 1e-2)):
        x0 = cfg[key]
        hstep = rel * abs(x0)
        d1 = (gpu_obs(key, x0 + hstep) - gpu_obs(key, x0 - hstep)) / (2 * hstep)
        d2 = (gpu_obs(key, x0 + hstep / 2) - gpu_obs(key, x0 - hstep / 2)) / hstep
        ref, spread = (4 * d2 - d1) / 3, abs(d2 - d1)
        print(f"chain5k 64^3 200 steps d/d{key}: adjoint {got[key]:.8e} GPU FD {ref:.8e} (spread {spread:.1e})")
        assert abs(got[key] - ref) <= 1e-3 * abs(ref) + 3 * spread, key
