"""Pins of the oracle's thermal noise (the xi_i of the fluctuating lattice
Boltzmann source term S_i = p_i + xi_i, Sec. 2.2): the random-number
generator against its published known answers, the moment basis against
weighted orthogonality, the noise against the exact conservation of mass and
momentum and against its closed-form covariance, and a run against
equipartition (density variance rho0 kT / c_s^2, momentum variance rho0 kT
per node and component)."""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
C = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
              [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1],
              [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]], float)
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def test_philox_known_answers(orc):
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        assert orc.philox4x32_10(v[:4], v[4:6]) == v[6:10]


def test_mode_basis_is_weighted_orthogonal(orc):
    E, b = orc.mode_basis()
    G = (E * W) @ E.T
    assert np.allclose(G, np.diag(b), atol=1e-14)
    assert np.all(b > 0)
    # the conserved modes: density and momentum
    assert np.allclose(E[0], 1.0) and np.allclose(E[1:4], C.T)


def _cfg(**kw):
    d = dict(nx=8, ny=8, nz=8, tau=0.8, rho0=1.0, kT=1e-4, seed=12345)
    d.update(kw)
    return d


def test_noise_carries_no_mass_or_momentum(orc):
    for node, step in ((0, 0), (17, 3), (511, 1 << 33)):
        xi = orc.node_noise(_cfg(), node, step)
        assert abs(xi.sum()) < 1e-18 + 1e-15 * np.abs(xi).max()
        assert np.abs(xi @ C).max() < 1e-15 * np.abs(xi).max() * 4
        assert np.abs(xi).max() > 0


def test_noise_covariance_closed_form(orc):
    """With one relaxation rate for every non-conserved mode the noise
    covariance in population space does not depend on the basis:
    mu (1 - (1 - omega)^2) w_i (delta_ij - w_j (1 + 3 c_i.c_j)), mu = 3 rho0 kT."""
    cfg = _cfg(tau=0.7, kT=2e-4)
    n = 20000
    X = np.array([orc.node_noise(cfg, k, 7) for k in range(n)])
    om = 1 / 0.7
    mu = 3 * 1.0 * 2e-4
    expect = mu * (1 - (1 - om) ** 2) * W[:, None] * (np.eye(19) - W[None, :] * (1 + 3 * C @ C.T))
    got = X.T @ X / n
    # sampling error of a variance estimate: ~ sqrt(2/n) of the diagonal scale
    scale = np.sqrt(np.outer(np.diag(expect), np.diag(expect)))
    assert np.abs(got - expect).max() < 5 * np.sqrt(2 / n) * scale.max()
    assert np.abs(X.mean(0)).max() < 5 * np.sqrt(np.diag(expect).max() / n)
    # different steps and nodes draw different numbers
    assert not np.allclose(orc.node_noise(cfg, 3, 7), orc.node_noise(cfg, 3, 8))
    assert not np.allclose(orc.node_noise(cfg, 3, 7), orc.node_noise(dict(cfg, seed=1), 3, 7))


def test_noise_off_leaves_the_step_deterministic(orc):
    """kT = 0 adds nothing: the step does not depend on the seed; kT > 0 does."""
    rng = np.random.default_rng(5)
    f = orc.equilibrium(np.ones(512), 0.01 * rng.standard_normal((3, 512)))
    topo = orc.Topology(np.zeros(0), np.zeros((0, 2)), [], [])
    none = (np.zeros((3, 0)), np.zeros((3, 0)))
    a = orc.run(_cfg(kT=0.0, seed=1), topo, f, *none, 3)[0]
    b = orc.run(_cfg(kT=0.0, seed=2), topo, f, *none, 3)[0]
    c = orc.run(_cfg(kT=1e-6, seed=2), topo, f, *none, 3)[0]
    assert np.array_equal(a, b)
    assert np.abs(c - a).max() > 1e-6


@pytest.mark.slow
def test_equipartition_of_the_fluctuating_fluid(orc):
    """An 8^3 periodic fluid at rest with noise: after equilibration the
    density fluctuates with variance rho0 kT / c_s^2 and each momentum
    component with rho0 kT (1 - 1/N): total momentum is conserved at zero."""
    cfg = _cfg(tau=1.0, kT=1e-4)
    N = 512
    f = orc.equilibrium(np.ones(N), np.zeros((3, N)))
    topo = orc.Topology(np.zeros(0), np.zeros((0, 2)), [], [])
    f, _, _, _ = orc.run(dict(cfg, step0=0), topo, f, np.zeros((3, 0)), np.zeros((3, 0)), 50)
    rv, jv = [], []
    step = 50
    for _ in range(300):
        f, _, _, _ = orc.run(dict(cfg, step0=step), topo, f, np.zeros((3, 0)), np.zeros((3, 0)), 4)
        step += 4
        rho, j = orc.moments(f)
        rv.append(((rho - 1.0) ** 2).mean())
        jv.append((j ** 2).mean())
    kT = 1e-4
    assert abs(np.mean(rv) / (3 * kT) - 1) < 0.05, np.mean(rv) / (3 * kT)
    assert abs(np.mean(jv) / (kT * (1 - 1 / N)) - 1) < 0.05, np.mean(jv) / kT
