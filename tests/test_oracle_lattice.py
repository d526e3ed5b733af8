"""Pins of the oracle's lattice Boltzmann part (Sec. 2.2, Eqs. 1-2) against what
the mathematics fixes: D3Q19 isotropy, equilibrium and Guo-source moments, the
BGK relaxation factor, the rest state, conservation, and the closed-form
hydrodynamics of the shear wave, Kolmogorov and Poiseuille flows."""
import itertools

import numpy as np
import pytest

EMPTY = np.zeros((3, 0))


def _empty(orc):
    return orc.Topology(np.zeros(0), np.zeros((0, 2)), [], [])


def test_d3q19_set_and_isotropy(orc):
    c, w, opp = orc.lattice()
    assert c.shape == (19, 3)
    # 19 distinct speeds: one at rest, six of length 1, twelve of length sqrt(2).
    assert len({tuple(r) for r in c}) == 19
    norms = (c * c).sum(1)
    assert sorted(np.bincount(norms)) == [1, 6, 12]
    assert np.all(c[opp] == -c)
    d = np.eye(3)
    assert np.isclose(w.sum(), 1.0, rtol=0, atol=1e-15)
    assert np.allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), d / 3, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0, atol=1e-15)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
            + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso4, atol=1e-15)
    # Speeds of the same length share one weight.
    for n in (0, 1, 2):
        assert np.ptp(w[norms == n]) == 0


def test_equilibrium_moments(orc):
    c, _, _ = orc.lattice()
    rng = np.random.default_rng(3)
    n = 50
    rho = 1 + 0.1 * rng.standard_normal(n)
    u = 0.05 * rng.standard_normal((3, n))
    feq = orc.equilibrium(rho, u)
    assert np.allclose(feq.sum(0), rho, rtol=0, atol=1e-14)
    assert np.allclose(np.einsum("in,ia->an", feq, c), rho * u, rtol=0, atol=1e-14)
    # Second moment of the second-order equilibrium: rho/3 delta + rho u u.
    pi = np.einsum("in,ia,ib->abn", feq, c, c)
    ref = np.eye(3)[:, :, None] * rho / 3 + rho * np.einsum("an,bn->abn", u, u)
    assert np.allclose(pi, ref, rtol=0, atol=1e-14)


def test_guo_source_moments(orc):
    c, _, _ = orc.lattice()
    rng = np.random.default_rng(4)
    for tau in (0.55, 0.8, 1.3):
        om = 1 / tau
        u = 0.05 * rng.standard_normal(3)
        F = 1e-3 * rng.standard_normal(3)
        S = orc.guo_source(tau, u, F)
        assert abs(S.sum()) < 1e-17
        assert np.allclose(S @ c, (1 - om / 2) * F, rtol=0, atol=1e-17)
        second = np.einsum("i,ia,ib->ab", S, c, c)
        assert np.allclose(second, (1 - om / 2) * (np.outer(u, F) + np.outer(F, u)), rtol=0, atol=1e-17)


def test_collision_relaxes_nonequilibrium_by_one_minus_omega(orc):
    """Without force the collision keeps rho and j, so f_eq is unchanged and the
    non-equilibrium part must shrink by exactly (1 - omega): this fixes both the
    sign of Eq. (1) and omega = 1/tau."""
    c, _, _ = orc.lattice()
    rng = np.random.default_rng(5)
    for tau in (0.55, 0.8, 1.7):
        rho = np.array([1.02])
        u = 0.03 * rng.standard_normal((3, 1))
        feq = orc.equilibrium(rho, u)[:, 0]
        f = feq + 1e-3 * rng.standard_normal(19)
        out = orc.collide_node(tau, f, np.zeros(3))
        r2, j2 = out.sum(), out @ c
        feq2 = orc.equilibrium(np.array([r2]), (j2 / r2)[:, None])[:, 0]
        assert np.isclose(r2, f.sum(), rtol=0, atol=1e-15)
        assert np.allclose(out - feq2, (1 - 1 / tau) * (f - orc.equilibrium(
            np.array([f.sum()]), ((f @ c) / f.sum())[:, None])[:, 0]), rtol=0, atol=1e-15)


def test_collision_with_force_adds_exactly_F(orc):
    c, _, _ = orc.lattice()
    rng = np.random.default_rng(6)
    f = orc.equilibrium(np.array([1.0]), 0.02 * rng.standard_normal((3, 1)))[:, 0]
    f += 1e-4 * rng.standard_normal(19)
    F = 1e-4 * rng.standard_normal(3)
    out = orc.collide_node(0.7, f, F)
    assert np.isclose(out.sum(), f.sum(), rtol=0, atol=1e-15)
    assert np.allclose(out @ c - f @ c, F, rtol=0, atol=1e-16)


@pytest.mark.parametrize("walls", [0, 1])
def test_rest_state_is_a_fixed_point(orc, walls):
    cfg = dict(nx=4, ny=5, nz=6, tau=0.7, walls_z=walls)
    n = 4 * 5 * 6
    f0 = orc.equilibrium(np.ones(n), np.zeros((3, n)))
    f, _, _, _ = orc.run(cfg, _empty(orc), f0, EMPTY, EMPTY, 25)
    assert np.abs(f - f0).max() < 1e-15


def test_uniform_force_mass_and_momentum(orc):
    """Periodic fluid pushed by a uniform g: mass is constant and the total
    momentum grows by exactly N g per step."""
    g = 2e-5
    cfg = dict(nx=6, ny=4, nz=5, tau=0.9, forcing="uniform", force_amp=g, force_dir=2)
    n = 6 * 4 * 5
    rng = np.random.default_rng(7)
    f = orc.equilibrium(np.ones(n), 0.01 * rng.standard_normal((3, n)))
    r0, j0 = orc.moments(f)
    f, _, _, _ = orc.run(cfg, _empty(orc), f, EMPTY, EMPTY, 40)
    r1, j1 = orc.moments(f)
    assert abs(r1.sum() - r0.sum()) < 1e-12
    dj = j1.sum(1) - j0.sum(1)
    assert np.allclose(dj, [0, 0, 40 * n * g], rtol=1e-12, atol=1e-15)


def _shear_nu(orc, N, tau, steps):
    cfg = dict(nx=1, ny=N, nz=1, tau=tau)
    y = np.arange(N)
    u = np.zeros((3, N))
    u[0] = 1e-4 * np.sin(2 * np.pi * y / N)
    f = orc.equilibrium(np.ones(N), u)
    ts, amps = [], []
    for s in range(steps // 10):
        f, _, _, _ = orc.run(cfg, _empty(orc), f, EMPTY, EMPTY, 10)
        r, j = orc.moments(f)
        ts.append((s + 1) * 10)
        amps.append(2 * np.mean(j[0] / r * np.sin(2 * np.pi * y / N)))
    ts, amps = np.array(ts), np.array(amps)
    k = 2 * np.pi / N
    q = len(ts) // 4
    return -np.polyfit(ts[q:], np.log(amps[q:]), 1)[0] / k ** 2


@pytest.mark.parametrize("tau", [0.55, 0.6, 0.8, 1.0])
def test_shear_wave_decays_at_lattice_viscosity(orc, tau):
    """u_x = U0 sin(2 pi y / N) decays as exp(-nu k^2 t), nu = (tau - 1/2)/3
    (Sec. 2.2: omega = 2/(6 nu + 1)); within 1% at N = 32, second order in k."""
    nu = (tau - 0.5) / 3
    e32 = _shear_nu(orc, 32, tau, 2000) / nu - 1
    e64 = _shear_nu(orc, 64, tau, 8000) / nu - 1
    assert abs(e32) < 0.01
    if tau != 1.0:
        assert 3.5 < e32 / e64 < 4.5


def test_kolmogorov_steady_state(orc):
    """g_x = A sin(k y) drives u_x = A sin(k y) / (rho nu k^2) at steady state,
    up to the O(k^2) lattice correction."""
    N, tau, A = 32, 0.8, 1e-6
    nu = (tau - 0.5) / 3
    cfg = dict(nx=1, ny=N, nz=1, tau=tau, forcing="kolmogorov", force_amp=A, force_dir=0,
               force_wave_axis=1)
    f = orc.equilibrium(np.ones(N), np.zeros((3, N)))
    k = 2 * np.pi / N
    f, _, _, _ = orc.run(cfg, _empty(orc), f, EMPTY, EMPTY, int(25 / (nu * k * k)))
    r, j = orc.moments(f)
    y = np.arange(N)
    g = A * np.sin(k * y)
    u = (j[0] + 0.5 * g) / r
    ref = g / (nu * k * k)
    err = np.abs(u - ref).max() / np.abs(ref).max()
    assert err < 2 * (k ** 2)  # O(k^2): 0.077 at N = 32
    assert err < 0.02


@pytest.mark.parametrize("tau", [0.55, 0.8, 1.0])
def test_poiseuille_between_bounce_back_walls(orc, tau):
    """Walls at z = -1/2 and N - 1/2 (half-way bounce-back) and g_x = A: the
    steady profile is A/(2 nu) (z + 1/2)(N - 1/2 - z). In the bulk the discrete
    second difference equals -A/nu exactly; the profile carries a
    tau-dependent wall slip that vanishes at second order in 1/N."""
    A = 1e-6
    nu = (tau - 0.5) / 3
    errs = []
    for N in (16, 32):
        cfg = dict(nx=1, ny=1, nz=N, tau=tau, walls_z=1, forcing="poiseuille", force_amp=A,
                   force_dir=0)
        f = orc.equilibrium(np.ones(N), np.zeros((3, N)))
        f, _, _, _ = orc.run(cfg, _empty(orc), f, EMPTY, EMPTY, int(20 * N * N / nu / np.pi ** 2) + 500)
        r, j = orc.moments(f)
        u = (j[0] + 0.5 * A) / r
        z = np.arange(N)
        ua = A / (2 * nu) * (z + 0.5) * (N - 0.5 - z)
        d2 = u[2:] - 2 * u[1:-1] + u[:-2]
        assert np.allclose(d2, -A / nu, rtol=1e-6)
        errs.append(np.abs(u - ua).max() / ua.max())
    assert errs[0] < 0.005
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_moments_match_definition_on_random_field(orc):
    c, _, _ = orc.lattice()
    rng = np.random.default_rng(8)
    f = rng.random((19, 30))
    rho, j = orc.moments(f)
    assert np.allclose(rho, f.sum(0), rtol=1e-15)
    assert np.allclose(j, np.einsum("in,ia->an", f, c), rtol=1e-14, atol=1e-15)


def test_streaming_is_a_permutation_with_walls(orc):
    """With tau = 1 and no force the collision maps f to f_eq; a stream is then a
    pure permutation, so the multiset of post-collision values is preserved:
    check it on one step with walls, where bounce-back must put every value
    somewhere."""
    cfg = dict(nx=3, ny=3, nz=4, tau=1.0, walls_z=1)
    n = 36
    rng = np.random.default_rng(9)
    f = orc.equilibrium(np.ones(n) + 0.01 * rng.standard_normal(n), 0.01 * rng.standard_normal((3, n)))
    r, j = orc.moments(f)
    post = orc.equilibrium(r, j / r)  # tau = 1: f* = f_eq
    f2, _, _, _ = orc.run(cfg, _empty(orc), f, EMPTY, EMPTY, 1)
    assert np.allclose(np.sort(f2.ravel()), np.sort(post.ravel()), rtol=0, atol=1e-16)
    assert np.isclose(f2.sum(), f.sum(), rtol=1e-15)
