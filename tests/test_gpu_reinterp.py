"""GPU re-interpolated coupling (the fluid velocity taken at the atom's
current position at every half-kick, each substep's friction impulse spread
with the weights of that position) against the FP64 oracle's reading R17:
teacher-forced parity of the 500-bead chain with the literal gamma, exact
momentum balance, and the single atom in a linear shear field, where the
re-interpolated and the frozen coupling differ by the velocity gradient the
atom crosses."""
import numpy as np
import pytest

from paper_2305_05025_gb300 import build, lbmd, synth
from gpu_helpers import make, oracle_start, teacher_forced

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbmd.lib()


@pytest.mark.parametrize("gamma", [0.5, 0.05])
def test_reinterpolated_chain_teacher_forced(orc, gamma):
    cfg = synth.workload("chain500_lattice32", n_md=128, gamma=gamma, skin=0.3, reinterp=1)
    inp = synth.inputs(cfg, 1)
    worst, done = teacher_forced(orc, cfg, inp, 10, f"reinterp gamma {gamma}")
    assert done == 10
    for k, r in worst.items():
        assert r <= 1.0, (k, r)


def test_reinterpolated_momentum_balance():
    """sum f c + sum m v grows by exactly N g per step with the per-substep
    spread (FP64 sums of the FP32 state). gamma 0.05: at 0.5 the explicit
    exchange of this chain goes unstable within 20 steps in the oracle too.
    Its fastest beads cross more than one node in some steps (1.7 at most in
    the oracle), so the nodes beyond the frozen region are exercised."""
    cfg = synth.workload("chain500_lattice32", n_md=128, gamma=0.05, skin=0.3, reinterp=1, forcing="uniform",
                         force_amp=1e-5, force_dir=1)
    inp = synth.inputs(cfg, 1)
    h = make(cfg, inp)
    m0, pf0, pa0 = lbmd.lbmd_get_stats(h)
    lbmd.lbmd_step(h, 20)
    m1, pf1, pa1 = lbmd.lbmd_get_stats(h)
    N = 32 ** 3
    dP = (pf1 + pa1) - (pf0 + pa0)
    expect = np.array([0.0, 20 * N * 1e-5, 0.0])
    print("reinterp: mass drift", m1 - m0, "momentum error", dP - expect, "atom momentum change", pa1 - pa0)
    # FP32 rounding of 19 populations per node-step, summed over 20 steps of
    # 32^3 nodes: a random walk of about 1e-5.
    assert abs(m1 - m0) < 1e-4
    assert np.abs(dP - expect).max() < 1e-4 * np.abs(pa1 - pa0).max() + 1e-5


@pytest.mark.parametrize("store", ["f32", "f16"])
def test_fast_atoms_beyond_the_frozen_region(orc, store):
    """Atoms that cross up to 2.6 nodes within one step, some through the
    periodic faces: the substeps take the velocities of the nodes the
    interpolation did not freeze (it froze the stencil and one node of
    margin) from the step's populations and add those nodes to the step's
    touched list. Positions and velocities agree with the oracle, which holds
    every node velocity, and so does the lattice after the step: the impulse
    spread onto the far nodes reached the collision."""
    n = 12
    cfg = dict(synth._COMMON, nx=n, ny=n, nz=n, tau=0.8, gamma=0.05, n_md=64, lj_eps=0.0, reinterp=1, store=store)
    rng = np.random.default_rng(17)
    u = 0.02 * rng.standard_normal((3, n ** 3))
    x = np.array([[0.4, 11.7, 5.5, 3.2], [5.0, 0.3, 11.8, 6.6], [6.1, 4.4, 0.2, 11.5]])
    v = np.array([[-2.1, 2.6, 0.3, -1.2], [1.7, -0.2, 2.4, 1.9], [-0.5, -2.2, -1.8, 2.3]])
    na = x.shape[1]
    inp = dict(rho=np.ones(n ** 3), u=u, x=x, v=v, mass=np.ones(na), bonds=np.zeros((0, 2), np.int32),
               bond_k=np.zeros(0), bond_r0=np.zeros(0))
    h = make(cfg, inp)
    m0, pf0, pa0 = lbmd.lbmd_get_stats(h)
    lbmd.lbmd_step(h, 1)
    lbmd.lbmd_check(h)
    s = lbmd.lbmd_get_fields(h, f=True, x=True, v=True)
    m1, pf1, pa1 = lbmd.lbmd_get_stats(h)
    f0, x0, v0, topo = oracle_start(orc, cfg, inp)
    fo, xo, vo, _ = orc.run(cfg, topo, f0, x0, v0, 1)
    assert np.abs(xo - x).max() > 2.0  # beyond the one-node margin
    ev = np.abs(s["v"] - vo).max() / np.abs(vo).max()
    ex = np.abs(s["x"] - xo).max()
    ef = np.abs(s["f"] - fo).max()
    print(f"fast atoms ({store}): v rel err {ev:.2e}, x err {ex:.2e}, f err {ef:.2e}, "
          f"momentum change {(pf1 + pa1) - (pf0 + pa0)}")
    if store == "f32":
        assert ev < 1e-5 and ex < 1e-5 and ef < 1e-6
    else:  # 16-bit storage: the populations the velocities come from carry its rounding
        assert ev < 1e-3 and ex < 1e-4 and ef < 1e-4
    # The coupling's whole effect on the lattice (against gamma = 0) is
    # 5e-3, most of it on nodes beyond the margin: far above the error.
    fg, _, _, _ = orc.run(dict(cfg, gamma=0.0), topo, f0, x0, v0, 1)
    assert np.abs(fo - fg).max() > 50 * ef
    # Momentum balance, up to the storage's rounding of the populations: the
    # kicked nodes carry delta f ~ 0.02, whose FP16 step (scaled by 2^10) is
    # ~1.5e-5 per population.
    assert np.abs((pf1 + pa1) - (pf0 + pa0)).max() < (1e-5 if store == "f32" else 5e-4)


@pytest.mark.parametrize("reinterp", [0, 1])
def test_single_atom_in_shear(orc, reinterp):
    n, S = 8, 1e-3
    cfg = dict(synth._COMMON, nx=n, ny=n, nz=n, tau=0.8, gamma=0.5, n_md=64, lj_eps=0.0, reinterp=reinterp)
    y = (np.arange(n ** 3) // n) % n
    u = np.zeros((3, n ** 3))
    u[0] = S * (y - 4.0)
    inp = dict(rho=np.ones(n ** 3), u=u, x=np.array([[2.3], [4.3], [3.6]]), v=np.array([[0.0], [0.05], [0.0]]),
               mass=np.ones(1), bonds=np.zeros((0, 2), np.int32), bond_k=np.zeros(0), bond_r0=np.zeros(0))
    h = make(cfg, inp)
    lbmd.lbmd_step(h, 1)
    s = lbmd.lbmd_get_fields(h, x=True, v=True)
    topo = orc.Topology(np.ones(1), np.zeros((0, 2)), [], [])
    f0 = orc.equilibrium(np.ones(n ** 3), u.astype(np.float32).astype(np.float64))
    _, xo, vo, _ = orc.run(cfg, topo, f0, inp["x"], inp["v"].astype(np.float32).astype(np.float64), 1)
    # the other coupling, for scale
    _, _, vf, _ = orc.run(dict(cfg, reinterp=1 - reinterp), topo, f0, inp["x"],
                          inp["v"].astype(np.float32).astype(np.float64), 1)
    err = abs(s["v"][0, 0] - vo[0, 0]) / abs(vo[0, 0])
    print(f"shear, reinterp={reinterp}: v_x GPU {s['v'][0, 0]:.9e} oracle {vo[0, 0]:.9e} (other coupling "
          f"{vf[0, 0]:.9e}), rel err {err:.1e}")
    assert err < 1e-5
    assert abs(vf[0, 0] - vo[0, 0]) > 1e3 * abs(s["v"][0, 0] - vo[0, 0])
    assert np.abs(s["x"] - xo).max() < 1e-6


def test_adjoint_refuses_reinterpolation():
    cfg = synth.workload("chain500_lattice32", nx=12, ny=12, nz=12, n_md=16, reinterp=1,
                         chains=[dict(n=20, centre="box", radius=None)])
    inp = synth.inputs(cfg, 1)
    inp["x"] = inp["x"] - inp["x"].mean(1, keepdims=True) + 6.0
    h = make(cfg, inp)
    with pytest.raises(lbmd.LBMDError) as e:
        lbmd.lbmd_backward(h, 2, 1)
    assert e.value.status == lbmd.LBMD_ERR_ARG
