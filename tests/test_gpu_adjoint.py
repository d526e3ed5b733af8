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


def _case(lj_eps, n_md, n_atoms, seed, v_scale=0.02, **kw):
    cfg = synth.workload("chain500_lattice32", nx=12, ny=12, nz=12, tau=0.8, gamma=0.5, n_md=n_md, lj_eps=lj_eps,
                         forcing="uniform", force_amp=1e-4, force_dir=0, u_sigma=0.005,
                         chains=[dict(n=n_atoms, centre="box", radius=None)], **kw)
    inp = synth.inputs(cfg, seed)
    rng = np.random.default_rng(seed)
    inp["v"] = v_scale * rng.standard_normal(inp["v"].shape)
    inp["x"] = inp["x"] - inp["x"].mean(1, keepdims=True) + 6.0
    return cfg, inp


def _oracle_obs(orc, cfg, inp, steps, observable):
    topo = orc.Topology(inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"])
    f = orc.equilibrium(inp["rho"].astype(np.float32).astype(np.float64),
                        inp["u"].astype(np.float32).astype(np.float64))
    _, _, _, obs = orc.run(cfg, topo, f, inp["x"], inp["v"].astype(np.float32).astype(np.float64), steps)
    return obs[:, 0].mean() if observable == lbmd.OBS_DRAG_X else obs[:, 3].mean()


def _fd(orc, cfg, inp, steps, observable, key, rel):
    """Richardson-extrapolated central difference of the oracle observable and
    its convergence: |D(h) - D(h/2)| relative to the result."""
    x0 = cfg[key]
    h = rel * abs(x0)

    def central(step):
        p = _oracle_obs(orc, dict(cfg, **{key: x0 + step}), inp, steps, observable)
        m = _oracle_obs(orc, dict(cfg, **{key: x0 - step}), inp, steps, observable)
        return (p - m) / (2 * step)

    d1, d2 = central(h), central(h / 2)
    ref = (4 * d2 - d1) / 3
    return ref, abs(d2 - d1) / abs(ref)


# FD steps at which the FP64 oracle's central differences have converged on
# these cases (D(h) and D(h/2) agree to < 1e-5 relative; for A the observable
# is nearly linear and smaller steps only add rounding).
FD_REL = dict(gamma=1e-4, tau=1e-4, force_amp=1e-2)


def _check(name, got, orc, cfg, inp, steps, observable, tol=1e-3, fd_rel=FD_REL):
    for key in ("gamma", "tau", "force_amp"):
        ref, spread = _fd(orc, cfg, inp, steps, observable, key, fd_rel[key])
        err = abs(got[key] - ref) / abs(ref)
        print(f"ADJ {name} d/d{key}: adjoint {got[key]:.8e} oracle FD {ref:.8e} rel err {err:.2e} "
              f"(FD convergence {spread:.1e})")
        assert spread < 1e-5, (key, "finite difference not converged", spread)
        assert err <= tol, (key, got[key], ref)


@pytest.mark.parametrize("observable", [lbmd.OBS_DRAG_X, lbmd.OBS_RG2])
def test_adjoint_matches_oracle_fd_harmonic_chain(orc, observable):
    cfg, inp = _case(lj_eps=0.0, n_md=16, n_atoms=30, seed=4)
    steps, ckpt = 12, 5
    h = make(cfg, inp)
    obs, dg, dtau, da = lbmd.lbmd_backward(h, steps, ckpt, observable)
    o_ref = _oracle_obs(orc, cfg, inp, steps, observable)
    assert abs(obs - o_ref) <= 1e-5 * abs(o_ref)
    _check(f"harmonic obs {observable}", dict(gamma=dg, tau=dtau, force_amp=da), orc, cfg, inp, steps, observable)
    # The state ends advanced by n_steps, like lbmd_step(n_steps).
    x = lbmd.lbmd_get_fields(h, x=True)["x"]
    h2 = make(cfg, inp)
    lbmd.lbmd_step(h2, steps)
    assert np.abs(x - lbmd.lbmd_get_fields(h2, x=True)["x"]).max() < 1e-5


def test_adjoint_matches_oracle_fd_lennard_jones_short(orc):
    """A 40-bead Lennard-Jones chain started at rest, two steps of 128
    substeps (two checkpoint segments): LJ pairs act throughout, and over this
    window the gradient is well conditioned (it moves by < 1e-4 relative when
    the start positions move by 1e-7), so the FP32 trajectory, which differs
    from the FP64 one by ~4e-5 in the observable, shares its gradient. Longer
    windows of such chains reach close encounters after which the d/dgamma of
    the FP32 and FP64 trajectories part (1.1e-2 after a third step, while
    d/dtau and d/dA still agree to 7e-5): there the exact gradient is not a
    property an FP32 computation can reproduce."""
    cfg, inp = _case(lj_eps=1.0, n_md=128, n_atoms=40, seed=7, v_scale=0.0)
    steps, ckpt = 2, 1
    h = make(cfg, inp)
    obs, dg, dtau, da = lbmd.lbmd_backward(h, steps, ckpt, lbmd.OBS_DRAG_X)
    _check("LJ chain40", dict(gamma=dg, tau=dtau, force_amp=da), orc, cfg, inp, steps, lbmd.OBS_DRAG_X,
           fd_rel=dict(gamma=1e-5, tau=1e-5, force_amp=1e-3))


def test_adjoint_with_fp16_storage(orc):
    """FP16 shifted storage: the forward rounds delta f to FP16 after every
    collision and the adjoint differentiates the FP32 arithmetic around it, so
    the gradient carries the storage resolution (2^-11 relative on delta f):
    within 2e-3 of the FP64 oracle's central difference."""
    cfg, inp = _case(lj_eps=0.0, n_md=16, n_atoms=30, seed=4, store="f16")
    steps, ckpt = 12, 5
    h = make(cfg, inp)
    obs, dg, dtau, da = lbmd.lbmd_backward(h, steps, ckpt, lbmd.OBS_DRAG_X)
    _check("harmonic f16", dict(gamma=dg, tau=dtau, force_amp=da), orc, dict(cfg, store="f32"), inp, steps,
           lbmd.OBS_DRAG_X, tol=2e-3)


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

    # FD steps of 4%: the GPU forward is FP32 with atomics in an unfixed order,
    # so the observable carries noise that small steps amplify (at 1% the two
    # central differences disagreed by 5e-4, at 4% by 1.1e-3, the h^2 term).
    # Richardson removes the h^2 term; what is left is O(h^4), about the
    # square of the h^2 term's relative size: below 1e-4 while that term
    # stays below 1e-2.
    for key, rel in (("gamma", 4e-2), ("tau", 4e-2), ("force_amp", 4e-2)):
        x0 = cfg[key]
        hstep = rel * abs(x0)
        d1 = (gpu_obs(key, x0 + hstep) - gpu_obs(key, x0 - hstep)) / (2 * hstep)
        d2 = (gpu_obs(key, x0 + hstep / 2) - gpu_obs(key, x0 - hstep / 2)) / hstep
        ref, spread = (4 * d2 - d1) / 3, abs(d2 - d1) / abs((4 * d2 - d1) / 3)
        err = abs(got[key] - ref) / abs(ref)
        print(f"ADJ chain5k 64^3 200 steps d/d{key}: adjoint {got[key]:.8e} GPU FD {ref:.8e} rel err {err:.2e} "
              f"(h^2 term {spread:.1e})")
        assert spread < 1e-2, (key, "finite difference outside its h^2 regime", spread)
        assert err <= 1e-3, (key, got[key], ref)


def test_adjoint_lennard_jones_globule_chain5k_lattice64_short(orc):
    """The adjoint workload as configured (64^3, 5,000-bead Lennard-Jones
    globule, uniform forcing 1e-5, n_md 128, gamma 0.05) over a window of two
    steps in two checkpoint segments, against the FP64 oracle's central
    differences: the oracle FD converges there (to < 3e-7) and the gradient
    moves by < 2e-5 when the start positions move by 1e-7."""
    cfg = synth.workload("chain5k_lattice64_uniform", n_md=128, gamma=0.05, skin=0.3)
    inp = synth.inputs(cfg, 1)
    steps = 2
    h = make(cfg, inp)
    obs, dg, dtau, da = lbmd.lbmd_backward(h, steps, 1, lbmd.OBS_DRAG_X)
    o_ref = _oracle_obs(orc, cfg, inp, steps, lbmd.OBS_DRAG_X)
    print(f"ADJ LJ globule obs: GPU {obs:.8e} oracle {o_ref:.8e}")
    assert abs(obs - o_ref) <= 1e-4 * abs(o_ref)
    _check("LJ globule 5k 64^3 2 steps", dict(gamma=dg, tau=dtau, force_amp=da), orc, cfg, inp, steps,
           lbmd.OBS_DRAG_X, fd_rel=dict(gamma=1e-5, tau=1e-5, force_amp=1e-3))


@pytest.mark.parametrize("lj", [0.0, 1.0])
def test_state_gradient_matches_oracle_directional_derivative(orc, lj):
    """The adjoint of the whole step with respect to the initial state
    (lbmd_backward_state: populations, positions, velocities) against the FP64
    oracle's central difference along random directions: <grad, delta> =
    d/de obs(state + e delta). Exercises every reverse operator together (the
    transposed pull, the collision's Jacobian, interpolation and spread with
    their weight gradients, the reverse substeps with the force Hessian)."""
    cfg, inp = _case(lj_eps=lj, n_md=16 if lj == 0.0 else 128, n_atoms=30 if lj == 0.0 else 40,
                     seed=4 if lj == 0.0 else 7, v_scale=0.02 if lj == 0.0 else 0.0)
    steps = 4 if lj == 0.0 else 2
    h = make(cfg, inp)
    obs, gf, gx, gv = lbmd.lbmd_backward_state(h, steps, 2, lbmd.OBS_DRAG_X)
    topo = orc.Topology(inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"])
    f0 = orc.equilibrium(inp["rho"].astype(np.float32).astype(np.float64),
                         inp["u"].astype(np.float32).astype(np.float64))
    x0, v0 = inp["x"], inp["v"].astype(np.float32).astype(np.float64)

    def oobs(f, x, v):
        return orc.run(cfg, topo, f, x, v, steps)[3][:, 0].mean()

    rng = np.random.default_rng(8)
    W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)[:, None]
    # The oracle's central differences converge (to < 1e-5) at these steps
    # along each direction; along the combined one only for the harmonic chain.
    eps = 1e-4 if lj == 0.0 else 1e-5
    for which in (("f", "x", "v", "all") if lj == 0.0 else ("f", "x", "v")):
        df = 1e-3 * W * rng.standard_normal(f0.shape) if which in ("f", "all") else np.zeros_like(f0)
        dx = 1e-2 * rng.standard_normal(x0.shape) if which in ("x", "all") else np.zeros_like(x0)
        dv = 1e-2 * rng.standard_normal(v0.shape) if which in ("v", "all") else np.zeros_like(v0)
        pred = (gf.astype(np.float64) * df).sum() + (gx.astype(np.float64) * dx).sum() + (gv * dv).sum()

        def cd(e):
            return (oobs(f0 + e * df, x0 + e * dx, v0 + e * dv) - oobs(f0 - e * df, x0 - e * dx, v0 - e * dv)) / (2 * e)

        d1, d2 = cd(eps), cd(eps / 2)
        ref = (4 * d2 - d1) / 3
        err = abs(pred - ref) / abs(ref)
        print(f"ADJ state lj={lj} along {which}: adjoint {pred:.8e} oracle FD {ref:.8e} rel err {err:.2e} "
              f"(FD convergence {abs(d2 - d1) / abs(ref):.1e})")
        assert abs(d2 - d1) < 1e-5 * abs(ref)
        assert err <= 1e-3, (which, pred, ref)
