"""Pins of the oracle's solute and coupling parts (Sec. 2.2: Stokes friction,
trilinear interpolation over the eight nearest nodes, equal and opposite force
on the fluid, lock-step integration) against closed forms, brute force and
conservation laws."""
import numpy as np
import pytest

from paper_2305_05025_gb300 import synth

EMPTY = np.zeros((3, 0))


def _chain_topo(orc, inp):
    return orc.Topology(inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"])


@pytest.fixture(scope="module")
def c1():
    cfg = synth.workload("chain500_lattice32", n_md=128)
    return cfg, synth.inputs(cfg, 1)


def test_lj_closed_forms(orc):
    """Plain 12-6 LJ has its minimum at 2^(1/6) sigma and U(sigma) = 0; the
    shifted-force form has F(rc) = U(rc) = 0. Probed with a two-atom system."""
    sig, eps = 0.4, 1.0
    cfg = dict(nx=16, ny=16, nz=16, tau=1.0, lj_sigma=sig, lj_eps=eps, lj_rcut_over_sigma=2.5)
    topo = orc.Topology(np.ones(2), np.zeros((0, 2)), [], [])
    rc = 2.5 * sig

    def fe(r, rcos=2.5):
        c = dict(cfg, lj_rcut_over_sigma=rcos)
        x = np.array([[5.0, 5.0 + r], [5.0, 5.0], [5.0, 5.0]])
        F, e = orc.forces(c, topo, x)
        return F[0, 1], e  # radial force on atom 1 (positive = repulsive)

    # A long cutoff makes the shift small (|F_LJ(8)| ~ 5e-8): plain-LJ closed
    # forms, against force scales of order 10-100 near sigma.
    f_min, _ = fe(2 ** (1 / 6) * sig, rcos=20.0)
    assert abs(f_min) < 1e-7
    _, e_sig = fe(sig, rcos=20.0)
    assert abs(e_sig) < 1e-6
    # Shifted force: force and energy vanish at the cutoff, and inside it the
    # force equals F_LJ(r) - F_LJ(rc).
    f_c, e_c = fe(rc * (1 - 1e-9))
    assert abs(f_c) < 1e-7 and abs(e_c) < 1e-9
    r = 0.55
    plain = 24 * eps / r * (2 * (sig / r) ** 12 - (sig / r) ** 6)
    plain_c = 24 * eps / rc * (2 * (sig / rc) ** 12 - (sig / rc) ** 6)
    assert np.isclose(fe(r)[0], plain - plain_c, rtol=1e-12)
    # Beyond the cutoff nothing acts.
    assert fe(rc * 1.01) == (0.0, 0.0)


def test_bond_closed_form(orc):
    cfg = dict(nx=16, ny=16, nz=16, tau=1.0, lj_eps=0.0)
    topo = orc.Topology(np.ones(2), np.array([[0, 1]]), [100.0], [0.5])
    x = np.array([[3.0, 3.7], [4.0, 4.0], [5.0, 5.0]])
    F, e = orc.forces(cfg, topo, x)
    assert np.isclose(e, 0.5 * 100 * 0.2 ** 2, rtol=1e-14)
    assert np.allclose(F[:, 0], [100 * 0.2, 0, 0], rtol=1e-14)
    assert np.allclose(F[:, 1], [-100 * 0.2, 0, 0], rtol=1e-14)


def test_forces_are_minus_energy_gradient(orc, c1):
    cfg, inp = c1
    topo = _chain_topo(orc, inp)
    rng = np.random.default_rng(11)
    x = inp["x"] + 0.02 * rng.standard_normal(inp["x"].shape)
    F, _ = orc.forces(cfg, topo, x)
    h = 1e-6
    for a in rng.choice(x.shape[1], 12, replace=False):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[d, a] += h
            xm[d, a] -= h
            g = (orc.forces(cfg, topo, xp)[1] - orc.forces(cfg, topo, xm)[1]) / (2 * h)
            assert abs(-g - F[d, a]) <= 1e-6 * max(1.0, abs(F[d, a]))


def test_cells_equal_brute_force_and_newton_third_law(orc, c1):
    cfg, inp = c1
    topo = _chain_topo(orc, inp)
    F1, e1 = orc.forces(cfg, topo, inp["x"])
    F2, e2 = orc.forces(cfg, topo, inp["x"], brute_force=True)
    assert np.allclose(F1, F2, rtol=1e-12, atol=1e-12)
    assert np.isclose(e1, e2, rtol=1e-13)
    assert np.abs(F1.sum(1)).max() < 1e-10


def test_cell_membership_is_geometric(orc, c1):
    cfg, inp = c1
    x = inp["x"]
    cell, nc = orc.cells(cfg, x)
    L = np.array([cfg["nx"], cfg["ny"], cfg["nz"]], float)
    h = L / nc
    assert np.all(h >= 1.0)  # side >= cutoff + skin
    cz, rem = np.divmod(cell, nc[0] * nc[1])
    cy, cx = np.divmod(rem, nc[0])
    xw = np.mod(x, L[:, None])
    for d, c in enumerate((cx, cy, cz)):
        assert np.all(xw[d] >= c * h[d] - 1e-12) and np.all(xw[d] < (c + 1) * h[d] + 1e-12)


def test_neighbour_counts_equal_brute_force(orc, c1):
    cfg, inp = c1
    x = inp["x"]
    counts = orc.neighbour_counts(cfg, x)
    L = np.array([cfg["nx"], cfg["ny"], cfg["nz"]], float)[:, None, None]
    d = x[:, :, None] - x[:, None, :]
    d -= L * np.round(d / L)
    r2 = (d * d).sum(0)
    np.fill_diagonal(r2, np.inf)
    assert np.array_equal(counts, (r2 < 1.0).sum(1))
    assert np.array_equal(counts, orc.neighbour_counts(cfg, x, brute_force=True))


def test_interpolation_reproduces_linear_fields(orc):
    """Trilinear weights are a partition of unity and exact for fields linear
    inside the stencil."""
    N = 12
    cfg = dict(nx=N, ny=N, nz=N, tau=1.0)
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    a = np.array([0.3, -0.2, 0.1])
    B = np.array([[0.01, 0.02, -0.03], [0.0, 0.04, 0.01], [-0.02, 0.01, 0.03]])
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()]).astype(float)
    u = a[:, None] + B @ pos
    rng = np.random.default_rng(12)
    xa = rng.uniform(1.0, N - 2.0, size=(3, 40))
    U = orc.interp(cfg, u, xa)
    assert np.allclose(U, a[:, None] + B @ xa, rtol=0, atol=1e-14)
    ones = orc.interp(cfg, np.ones((3, N ** 3)), rng.uniform(-30, 30, size=(3, 40)))
    assert np.allclose(ones, 1.0, rtol=0, atol=1e-15)


def test_spread_is_transpose_of_interpolation(orc):
    N = 7
    cfg = dict(nx=N, ny=N + 1, nz=N - 1, tau=1.0)
    n = N * (N + 1) * (N - 1)
    rng = np.random.default_rng(13)
    xa = rng.uniform(-10, 20, size=(3, 25))
    u = rng.standard_normal((3, n))
    J = rng.standard_normal((3, 25))
    lhs = np.sum(orc.interp(cfg, u, xa) * J)
    rhs = np.sum(u * orc.spread(cfg, xa, J))
    assert np.isclose(lhs, rhs, rtol=1e-13)


def test_atom_on_node_spreads_everything_there(orc):
    cfg = dict(nx=5, ny=5, nz=5, tau=1.0)
    G = orc.spread(cfg, np.array([[2.0], [3.0], [-1.0]]), np.array([[1.0], [2.0], [3.0]]))
    k = (4 * 5 + 3) * 5 + 2
    assert np.allclose(G[:, k], [1, 2, 3])
    assert np.count_nonzero(G) == 3


@pytest.mark.parametrize("n_md", [1, 4, 32])
def test_single_atom_first_step_drag(orc, n_md):
    """One atom at rest in a uniform flow u0 (no forces): every half-kick of the
    Verlet substeps relaxes u0 - v by (1 - gamma/(2 n_md)), so the impulse after
    one LB step is m u0 [1 - (1 - gamma/(2 n_md m))^(2 n_md)] exactly; the
    fluid loses the same momentum."""
    gamma, u0 = 0.5, 1e-3
    cfg = dict(nx=4, ny=4, nz=4, tau=0.8, gamma=gamma, n_md=n_md)
    n = 64
    u = np.zeros((3, n))
    u[0] = u0
    f = orc.equilibrium(np.ones(n), u)
    topo = orc.Topology(np.ones(1), np.zeros((0, 2)), [], [])
    x = np.array([[1.3], [2.1], [0.7]])
    f2, x2, v2, obs = orc.run(cfg, topo, f, x, np.zeros((3, 1)), 1)
    J = u0 * (1 - (1 - gamma / (2 * n_md)) ** (2 * n_md))
    assert np.isclose(obs[0, 0], J, rtol=1e-13)
    assert np.isclose(v2[0, 0], J, rtol=1e-13)
    r0, j0 = orc.moments(f)
    r2, j2 = orc.moments(f2)
    assert np.isclose(j2[0].sum() - j0[0].sum(), -J, rtol=1e-10)


def test_single_atom_reaches_common_velocity(orc):
    """Momentum is shared until atom and fluid move together at
    V = P / (sum rho + m)."""
    cfg = dict(nx=4, ny=4, nz=4, tau=0.8, gamma=0.5, n_md=4)
    n = 64
    u = np.zeros((3, n))
    u[0] = 1e-3
    f = orc.equilibrium(np.ones(n), u)
    topo = orc.Topology(np.ones(1), np.zeros((0, 2)), [], [])
    x = np.array([[1.3], [2.1], [0.7]])
    v = np.array([[0.0], [2e-4], [0.0]])
    r, j = orc.moments(f)
    P = j.sum(1) + v[:, 0]
    f2, x2, v2, _ = orc.run(cfg, topo, f, x, v, 2400)
    V = P / (r.sum() + 1.0)
    r2, j2 = orc.moments(f2)
    # Sound waves excited by the moving atom die out slowly; after 2400 steps
    # the residual is below 1e-5 of |V|.
    assert np.allclose(v2[:, 0], V, rtol=0, atol=2e-9)
    assert np.allclose(j2 / r2, V[:, None], rtol=0, atol=2e-8)


def test_coupled_step_conserves_mass_and_total_momentum(orc, c1):
    """Total momentum sum f c + sum m v changes by exactly sum_x g per step: the
    atom receives the drag impulse and the fluid its opposite (Sec. 2.2)."""
    cfg, inp = c1
    cfg = dict(cfg, nx=16, ny=16, nz=16, gamma=0.05, forcing="uniform", force_amp=1e-5)
    inp = synth.inputs(dict(cfg, chains=[dict(n=120, centre="box", radius=None)]), 2)
    topo = _chain_topo(orc, inp)
    rng = np.random.default_rng(14)
    u = 0.01 * rng.standard_normal((3, 16 ** 3))
    f = orc.equilibrium(np.ones(16 ** 3), u)
    v = 0.1 * rng.standard_normal(inp["x"].shape)
    r0, j0 = orc.moments(f)
    P0 = j0.sum(1) + v.sum(1)
    steps = 6
    f2, x2, v2, obs = orc.run(cfg, topo, f, inp["x"], v, steps)
    r1, j1 = orc.moments(f2)
    P1 = j1.sum(1) + v2.sum(1)
    assert abs(r1.sum() - r0.sum()) < 1e-11
    assert np.allclose(P1 - P0, [steps * 16 ** 3 * 1e-5, 0, 0], rtol=0, atol=1e-11)
    assert np.abs(obs[:, :3]).max() > 1e-4  # the coupling did act


def test_verlet_harmonic_dimer_second_order(orc):
    """Without drag a harmonic dimer oscillates with omega = sqrt(2k/m); the
    velocity-Verlet error after a fixed time falls by ~4 when the substep
    halves."""
    k, r0, A = 100.0, 0.5, 0.1
    topo = orc.Topology(np.ones(2), np.array([[0, 1]]), [k], [r0])
    x = np.array([[4.0, 4.0 + r0 + A], [4.0, 4.0], [4.0, 4.0]])
    w = np.sqrt(2 * k)
    errs = []
    for n_md in (32, 64, 128):
        cfg = dict(nx=8, ny=8, nz=8, tau=1.0, gamma=0.0, n_md=n_md, lj_eps=0.0)
        f = orc.equilibrium(np.ones(512), np.zeros((3, 512)))
        _, x2, _, _ = orc.run(cfg, topo, f, x, np.zeros((3, 2)), 3)
        r = x2[0, 1] - x2[0, 0]
        errs.append(abs(r - (r0 + A * np.cos(w * 3.0))))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5
    assert errs[2] < 3e-3


def test_wall_stencil_is_rejected(orc):
    cfg = dict(nx=4, ny=4, nz=4, tau=1.0, walls_z=1)
    with pytest.raises(ValueError):
        orc.interp(cfg, np.zeros((3, 64)), np.array([[1.0], [1.0], [3.5]]))


def _static_obs(orc, x, mass):
    """obs of one oracle step in which nothing can move: fluid at rest, atoms
    at rest, no Lennard-Jones, no bonds, so x after the step is x exactly and
    obs[3] is the squared radius of gyration of x itself."""
    n = 16 ** 3
    cfg = dict(nx=16, ny=16, nz=16, tau=0.8, gamma=0.5, n_md=4, lj_eps=0.0)
    f = orc.equilibrium(np.ones(n), np.zeros((3, n)))
    topo = orc.Topology(np.asarray(mass, float), np.zeros((0, 2)), [], [])
    _, x2, _, obs = orc.run(cfg, topo, f, x, np.zeros_like(x), 1)
    assert np.array_equal(x2, x)
    return obs[0, 3]


def test_radius_of_gyration_two_unequal_beads(orc):
    """Two beads of masses m1, m2 a distance d apart: about the mass-weighted
    centre, R_g^2 = m1 m2 d^2 / (m1 + m2)^2 (an unweighted centre or an
    unweighted average would give d^2/4)."""
    m1, m2, d = 0.7, 1.9, 1.3
    rng = np.random.default_rng(21)
    e = rng.standard_normal(3)
    e /= np.linalg.norm(e)
    c = np.array([7.2, 8.1, 6.6])
    x = np.stack([c, c + d * e], axis=1)
    assert np.isclose(_static_obs(orc, x, [m1, m2]), m1 * m2 * d * d / (m1 + m2) ** 2, rtol=1e-12)


@pytest.mark.parametrize("masses", ["equal", "alternating"])
def test_radius_of_gyration_ring(orc, masses):
    """n beads on a circle of radius R in a tilted plane: R_g^2 = R^2 whether
    the masses are equal or alternate (either way the centre of mass is the
    circle's centre); unwrapped positions past the box edge count as they are."""
    n, R = 12, 2.5
    rng = np.random.default_rng(22)
    a, b = np.linalg.qr(rng.standard_normal((3, 2)))[0].T
    phi = 2 * np.pi * np.arange(n) / n
    c = np.array([15.5, 0.3, 8.0])  # the ring crosses y = 0
    x = c[:, None] + R * (np.cos(phi)[None, :] * a[:, None] + np.sin(phi)[None, :] * b[:, None])
    mass = np.ones(n) if masses == "equal" else np.where(np.arange(n) % 2 == 0, 0.6, 1.8)
    assert np.isclose(_static_obs(orc, x, mass), R * R, rtol=1e-12)


def test_radius_of_gyration_is_translation_invariant(orc, c1):
    _, inp = c1
    x = inp["x"][:, :60]
    mass = np.random.default_rng(23).uniform(0.5, 2.0, 60)
    r1 = _static_obs(orc, x, mass)
    r2 = _static_obs(orc, x + np.array([[3.25], [-1.5], [0.75]]), mass)
    assert np.isclose(r1, r2, rtol=1e-12)
    # and equals the mass-weighted definition written out here
    cm = (x * mass).sum(1) / mass.sum()
    assert np.isclose(r1, (mass * ((x - cm[:, None]) ** 2).sum(0)).sum() / mass.sum(), rtol=1e-12)


@pytest.mark.parametrize("m", [0.5, 2.5])
def test_single_atom_drag_with_mass(orc, m):
    """The friction gamma (u - v) is a force (gamma in mass per time): an atom
    of mass m relaxes u0 - v by (1 - gamma/(2 n_md m)) per half-kick, so its
    impulse after one step is m u0 [1 - (1 - gamma/(2 n_md m))^(2 n_md)]; a
    per-mass friction rate would drop the m inside."""
    gamma, u0, n_md = 0.5, 1e-3, 8
    cfg = dict(nx=4, ny=4, nz=4, tau=0.8, gamma=gamma, n_md=n_md)
    u = np.zeros((3, 64))
    u[0] = u0
    f = orc.equilibrium(np.ones(64), u)
    topo = orc.Topology(np.array([m]), np.zeros((0, 2)), [], [])
    _, _, v2, obs = orc.run(cfg, topo, f, np.array([[1.3], [2.1], [0.7]]), np.zeros((3, 1)), 1)
    vexp = u0 * (1 - (1 - gamma / (2 * n_md * m)) ** (2 * n_md))
    assert np.isclose(v2[0, 0], vexp, rtol=1e-13)
    assert np.isclose(obs[0, 0], m * vexp, rtol=1e-13)


def test_total_momentum_with_unequal_masses(orc):
    """sum f c + sum m v is conserved with random masses in [0.5, 2] (no body
    force): the fluid receives exactly the impulse the atoms lose."""
    cfg = dict(synth._COMMON, nx=12, ny=12, nz=12, tau=0.8, gamma=0.5, n_md=128,
               chains=[dict(n=80, centre="box", radius=None)])
    inp = synth.inputs(cfg, 3)
    rng = np.random.default_rng(24)
    mass = rng.uniform(0.5, 2.0, inp["x"].shape[1])
    topo = orc.Topology(mass, inp["bonds"], inp["bond_k"], inp["bond_r0"])
    u = 0.01 * rng.standard_normal((3, 12 ** 3))
    f = orc.equilibrium(np.ones(12 ** 3), u)
    v = 0.05 * rng.standard_normal(inp["x"].shape)
    _, j0 = orc.moments(f)
    P0 = j0.sum(1) + (mass * v).sum(1)
    f2, _, v2, _ = orc.run(cfg, topo, f, inp["x"], v, 4)
    _, j1 = orc.moments(f2)
    P1 = j1.sum(1) + (mass * v2).sum(1)
    assert np.allclose(P1, P0, rtol=0, atol=1e-12)
    assert np.abs((mass * (v2 - v)).sum(1)).max() > 1e-4  # the coupling moved momentum


def _two(orc, r, q1, q2, bonded=False, **kw):
    cfg = dict(nx=16, ny=16, nz=16, tau=1.0, lj_eps=0.0, coul_c=0.7, coul_rc=1.0)
    cfg.update(kw)
    b = np.array([[0, 1]]) if bonded else np.zeros((0, 2))
    topo = orc.Topology(np.ones(2), b, [0.0] if bonded else [], [0.5] if bonded else [], charge=[q1, q2])
    x = np.array([[5.0, 5.0 + r], [5.0, 5.0], [5.0, 5.0]])
    F, e = orc.forces(cfg, topo, x)
    return F, e


def test_coulomb_pair_closed_form(orc):
    """Energy C q1 q2 / r^2 (dielectric eps_r r), shifted-force at the cutoff:
    radial force 2 C q1 q2 (1/r^3 - 1/rc^3); like charges repel."""
    C, rc = 0.7, 1.0
    for r, q1, q2 in ((0.5, 1.0, 1.0), (0.8, 1.0, -1.0), (0.3, -0.5, 2.0)):
        F, e = _two(orc, r, q1, q2)
        f = 2 * C * q1 * q2 * (1 / r ** 3 - 1 / rc ** 3)
        assert np.isclose(F[0, 1], f, rtol=1e-13) and np.isclose(F[0, 0], -f, rtol=1e-13)
        u = C * q1 * q2 * (1 / r ** 2 - 1 / rc ** 2) + (r - rc) * 2 * C * q1 * q2 / rc ** 3
        assert np.isclose(e, u, rtol=1e-12)
    F, _ = _two(orc, 0.5, 1.0, 1.0)
    assert F[0, 1] > 0  # repulsion pushes atom 1 (at larger x) further out
    F, e = _two(orc, 1.0 * (1 - 1e-9), 1.0, 1.0)
    assert abs(F[0, 1]) < 1e-7 and abs(e) < 1e-9
    assert _two(orc, 1.01, 1.0, 1.0)[1] == 0.0
    # bonded pairs carry no Coulomb (a bond of zero stiffness leaves nothing)
    F, e = _two(orc, 0.5, 1.0, 1.0, bonded=True)
    assert np.abs(F).max() == 0.0 and e == 0.0


def test_coulomb_forces_are_minus_energy_gradient(orc, c1):
    """A charged chain (alternating +-1, LJ and bonds on): F = -grad U by
    central differences, and the forces sum to zero (Newton's third law)."""
    cfg, inp = c1
    cfg = dict(cfg, coul_c=0.3, coul_rc=0.9)
    q = np.where(np.arange(inp["x"].shape[1]) % 2 == 0, 1.0, -1.0)
    topo = orc.Topology(inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"], charge=q)
    rng = np.random.default_rng(12)
    x = inp["x"] + 0.02 * rng.standard_normal(inp["x"].shape)
    F, _ = orc.forces(cfg, topo, x)
    F0, _ = orc.forces(cfg, orc.Topology(inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"]), x)
    assert np.abs(F - F0).max() > 1e-2  # the charges act
    assert np.abs(F.sum(1)).max() < 1e-9 * np.abs(F).max()
    h = 1e-6
    for a in rng.choice(x.shape[1], 12, replace=False):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[d, a] += h
            xm[d, a] -= h
            g = (orc.forces(cfg, topo, xp)[1] - orc.forces(cfg, topo, xm)[1]) / (2 * h)
            assert abs(-g - F[d, a]) <= 1e-6 * max(1.0, abs(F[d, a]))


def test_coulomb_cutoff_beyond_lennard_jones_is_rejected(orc):
    cfg = dict(nx=8, ny=8, nz=8, tau=1.0, coul_c=1.0, coul_rc=1.5)
    topo = orc.Topology(np.ones(2), np.zeros((0, 2)), [], [], charge=[1.0, -1.0])
    f = orc.equilibrium(np.ones(512), np.zeros((3, 512)))
    with pytest.raises(ValueError):
        orc.run(cfg, topo, f, np.array([[2.0, 2.5], [2.0, 2.0], [2.0, 2.0]]), np.zeros((3, 2)), 1)


def _shear_step(orc, n_md, reinterp, S=1e-3, gamma=0.5, y0=4.3, vx0=0.0, vy0=0.05):
    """One coupled step of one atom (m = 1, no forces) in a node velocity
    field u_x = S (y - 4) (linear between the nodes it visits, so trilinear
    interpolation is exact), u_y = u_z = 0. Returns (v_x, v_y, y) after it."""
    n = 8
    cfg = dict(nx=n, ny=n, nz=n, tau=0.8, gamma=gamma, n_md=n_md, reinterp=int(reinterp))
    y = (np.arange(n ** 3) // n) % n
    u = np.zeros((3, n ** 3))
    u[0] = S * (y - 4.0)
    f = orc.equilibrium(np.ones(n ** 3), u)
    topo = orc.Topology(np.ones(1), np.zeros((0, 2)), [], [])
    _, x2, v2, _ = orc.run(cfg, topo, f, np.array([[2.3], [y0], [3.6]]), np.array([[vx0], [vy0], [0.0]]), 1)
    return v2[0, 0], v2[1, 0], x2[1, 0]


@pytest.mark.parametrize("reinterp", [False, True])
def test_coupling_converges_to_its_ode(orc, reinterp):
    """Over one LB step the node velocities are frozen, so as n_md grows the
    atom follows dv/dt = gamma (U - v) with U = S (y(t) - 4) e_x when the
    velocity is re-interpolated at the current position, or U = S (y0 - 4) e_x
    when it is held at the step's start. Closed forms (t = 1, m = 1):
    v_y = v0 e^-g, y = y0 + v0 (1 - e^-g)/g, and
    re-interpolated: v_x = S (y0 - 4 + v0/g)(1 - e^-g) - S v0 e^-g;
    frozen:          v_x = S (y0 - 4)(1 - e^-g).
    The half-kicks take the friction at the velocity they start from (the
    second at v^(s+1/2)), which makes the velocity-dependent part first order:
    the error halves per doubling of n_md, towards each coupling's own ODE."""
    S, g, y0, v0 = 1e-3, 0.5, 4.3, 0.05
    e = np.exp(-g)
    vy = v0 * e
    yy = y0 + v0 * (1 - e) / g
    vx = S * (y0 - 4 + v0 / g) * (1 - e) - S * v0 * e if reinterp else S * (y0 - 4) * (1 - e)
    errs = []
    for n_md in (8, 16, 32, 64):
        gx, gy, gyy = _shear_step(orc, n_md, reinterp)
        errs.append(max(abs(gx - vx) / abs(vx), abs(gy - vy) / abs(vy), abs(gyy - yy) / abs(yy)))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(1.9 < r < 2.1 for r in ratios), (errs, ratios)
    assert errs[-1] < 2e-3
    # The two couplings differ by the velocity gradient seen along the path.
    fx, _, _ = _shear_step(orc, 64, not reinterp)
    assert abs(fx - vx) > 10 * errs[-1] * abs(vx)


def test_reinterpolated_coupling_conserves_momentum(orc, c1):
    cfg, inp = c1
    cfg = dict(cfg, nx=16, ny=16, nz=16, gamma=0.5, reinterp=1)
    inp = synth.inputs(dict(cfg, chains=[dict(n=120, centre="box", radius=None)]), 2)
    topo = _chain_topo(orc, inp)
    rng = np.random.default_rng(15)
    f = orc.equilibrium(np.ones(16 ** 3), 0.01 * rng.standard_normal((3, 16 ** 3)))
    v = 0.1 * rng.standard_normal(inp["x"].shape)
    r0, j0 = orc.moments(f)
    f2, x2, v2, obs = orc.run(cfg, topo, f, inp["x"], v, 4)
    r1, j1 = orc.moments(f2)
    assert abs(r1.sum() - r0.sum()) < 1e-11
    assert np.allclose(j1.sum(1) + v2.sum(1), j0.sum(1) + v.sum(1), rtol=0, atol=1e-12)
    f3, x3, v3, _ = orc.run(dict(cfg, reinterp=0), topo, f, inp["x"], v, 4)
    assert np.abs(v3 - v2).max() > 1e-6  # the option changes the dynamics
