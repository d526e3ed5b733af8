"""GPU screened Coulomb pairs (the force field's electrostatics with a
distance-dependent dielectric and a cutoff, Sec. 2.2) against the FP64
oracle: a charged 500-bead chain, teacher-forced over ten coupled steps
(bound max(1e-5, 3 x the FP32 floor) per field, as the other coupled tests),
the adjoint of a short charged Lennard-Jones chain against the oracle's
converged central differences, and the setter's argument errors."""
import numpy as np
import pytest

from paper_2305_05025_gb300 import build, lbmd, synth
from gpu_helpers import make, rel_linf, teacher_forced

pytestmark = pytest.mark.gpu

COUL = dict(coul_c=0.3, coul_rc=0.9)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbmd.lib()


def _alternating(n):
    return np.where(np.arange(n) % 2 == 0, 1.0, -1.0)


def test_charged_chain_teacher_forced(orc):
    cfg = synth.workload("chain500_lattice32", n_md=128, gamma=0.05, skin=0.3, **COUL)
    inp = dict(synth.inputs(cfg, 1))
    inp["charge"] = _alternating(inp["x"].shape[1])
    worst, done = teacher_forced(orc, cfg, inp, 10, "charged chain")
    assert done == 10
    for k, r in worst.items():
        assert r <= 1.0, (k, r)
    # The charges act: the same chain without them moves differently.
    h0 = make(cfg, dict(inp, charge=None))
    h1 = make(cfg, inp)
    lbmd.lbmd_step(h0, 2)
    lbmd.lbmd_step(h1, 2)
    assert rel_linf(lbmd.lbmd_get_fields(h0, v=True)["v"], lbmd.lbmd_get_fields(h1, v=True)["v"]) > 1e-2


def test_charged_chain_adjoint(orc):
    """The 40-bead Lennard-Jones chain of the adjoint tests with alternating
    charges, two steps: every gradient within 1e-3 of the converged FP64
    central difference."""
    cfg = synth.workload("chain500_lattice32", nx=12, ny=12, nz=12, tau=0.8, gamma=0.5, n_md=128, lj_eps=1.0,
                         forcing="uniform", force_amp=1e-4, force_dir=0, u_sigma=0.005,
                         chains=[dict(n=40, centre="box", radius=None)], **COUL)
    inp = dict(synth.inputs(cfg, 7))
    inp["v"] = np.zeros_like(inp["v"])
    inp["x"] = inp["x"] - inp["x"].mean(1, keepdims=True) + 6.0
    inp["charge"] = _alternating(40)
    h = make(cfg, inp)
    obs, dg, dtau, da = lbmd.lbmd_backward(h, 2, 1, lbmd.OBS_DRAG_X)
    topo = orc.Topology(inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"], charge=inp["charge"])
    f0 = orc.equilibrium(inp["rho"].astype(np.float32).astype(np.float64),
                         inp["u"].astype(np.float32).astype(np.float64))

    def oobs(c):
        return orc.run(c, topo, f0, inp["x"], inp["v"], 2)[3][:, 0].mean()

    assert abs(obs - oobs(cfg)) <= 1e-4 * abs(oobs(cfg))
    for key, got, rel in (("gamma", dg, 1e-5), ("tau", dtau, 1e-5), ("force_amp", da, 1e-3)):
        x0 = cfg[key]
        hh = rel * abs(x0)
        cd = lambda s: (oobs(dict(cfg, **{key: x0 + s})) - oobs(dict(cfg, **{key: x0 - s}))) / (2 * s)
        d1, d2 = cd(hh), cd(hh / 2)
        ref = (4 * d2 - d1) / 3
        err = abs(got - ref) / abs(ref)
        print(f"ADJ charged chain d/d{key}: adjoint {got:.8e} oracle FD {ref:.8e} rel err {err:.2e} "
              f"(FD convergence {abs(d2 - d1) / abs(ref):.1e})")
        assert abs(d2 - d1) < 1e-5 * abs(ref)
        assert err <= 1e-3, (key, got, ref)


def test_charge_setter_errors():
    cfg = synth.workload("chain500_lattice32", n_md=16, **COUL)
    inp = synth.inputs(cfg, 1)
    q = _alternating(500)
    h = lbmd.lbmd_create(cfg, inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"])
    with pytest.raises(lbmd.LBMDError) as e:
        lbmd.lbmd_set_charges(h, q, 0.3, 1.5)  # beyond the Lennard-Jones cutoff (1.0)
    assert e.value.status == lbmd.LBMD_ERR_ARG
    lbmd.lbmd_set_charges(h, q, 0.3, 0.9)
    lbmd.lbmd_set_state(h, rho=inp["rho"].astype(np.float32), u=inp["u"].astype(np.float32), x=inp["x"],
                        v=inp["v"].astype(np.float32))
    with pytest.raises(lbmd.LBMDError) as e:
        lbmd.lbmd_set_charges(h, q, 0.3, 0.9)
    assert e.value.status == lbmd.LBMD_ERR_STATE
