"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and
the benchmark.

This module holds geometry and random numbers only, none of the method's
arithmetic: velocity fields are handed out as (rho, u) and each side builds its
own equilibrium populations from them.

The paper's systems (a 53k-atom glycosylated spike trimer in a 19.2 nm cubic
box, Sec. 2.1) rest on PDB structures and force-field files that are not
available here. Self-avoiding bead chains with harmonic bonds stand in for the
protein, with matching atom counts and compactness.

Every generator draws from ``numpy.random.Generator(PCG64(seed))``.
"""
import math

import numpy as np

# Workloads, named by what they are. Keys are the ones both the C-ABI
# parameter block and the oracle understand.
_COMMON = dict(rho0=1.0, gamma=0.5, n_md=32, lj_eps=1.0, lj_sigma=0.4, lj_rcut_over_sigma=2.5,
               skin=0.0, forcing="none", force_amp=0.0, force_dir=0, force_wave_axis=1,
               walls_z=0, store="f32", bond_k=100.0, bond_r0=0.5, mass=1.0)

WORKLOADS = {
    # Periodic 32^3, tau 0.8, Gaussian velocity noise 0.01, one 500-bead chain.
    "chain500_lattice32": dict(_COMMON, nx=32, ny=32, nz=32, tau=0.8, u_sigma=0.01,
                               chains=[dict(n=500, centre="box", radius=None)], steps=100),
    # Periodic 128^3, tau 0.6, Kolmogorov forcing 1e-5, 20k-bead globule r = 20.
    "globule20k_lattice128": dict(_COMMON, nx=128, ny=128, nz=128, tau=0.6, u_sigma=0.0,
                                  forcing="kolmogorov", force_amp=1e-5, force_dir=0,
                                  force_wave_axis=1,
                                  chains=[dict(n=20000, centre="box", radius=20.0)], steps=1000),
    # Periodic 256^3, tau 0.55, noise 0.005, trimer of three 20k-bead globules.
    "trimer60k_lattice256": dict(_COMMON, nx=256, ny=256, nz=256, tau=0.55, u_sigma=0.005,
                                 chains="trimer", steps=200),
    # 64^3, tau 0.8, uniform forcing 1e-5 along x, 5k-bead globule r = 12.
    "chain5k_lattice64_uniform": dict(_COMMON, nx=64, ny=64, nz=64, tau=0.8, u_sigma=0.0,
                                      forcing="uniform", force_amp=1e-5,
                                      chains=[dict(n=5000, centre="box", radius=12.0)],
                                      steps=200, ckpt_every=20),
    # 512^3 z-channel, bounce-back walls, Poiseuille forcing 1e-6, ten globules.
    "channel10x20k_lattice512": dict(_COMMON, nx=512, ny=512, nz=512, tau=0.8, u_sigma=0.0,
                                     forcing="poiseuille", force_amp=1e-6, walls_z=1,
                                     chains="grid10", steps=500),
    # The same ten globules in a shallower 256 x 256 x 64 channel: the solute
    # of the 512^3 channel on a lattice 32x smaller (profiling of the solute
    # kernels on a few GB of device memory).
    "channel10x20k_lattice256x256x64": dict(_COMMON, nx=256, ny=256, nz=64, tau=0.8, u_sigma=0.0,
                                            forcing="poiseuille", force_amp=1e-6, walls_z=1,
                                            chains="grid10", steps=500),
    # A z-channel small enough for the oracle that still takes the 512^3
    # channel's code path: more than 65,536 atoms, a box side above 166 (the
    # coarse pair-search grid), walls, and two flat chains whose stencils touch
    # the first and the last fluid plane pair (z = 0.5 and z = nz - 1.5).
    "channel4x17k_lattice176x48x48": dict(_COMMON, nx=176, ny=48, nz=48, tau=0.8, u_sigma=0.0,
                                          forcing="poiseuille", force_amp=1e-6, walls_z=1,
                                          chains="channel4", steps=2),
}


def workload(name, **overrides):
    cfg = dict(WORKLOADS[name])
    cfg.update(overrides)
    cfg["name"] = name
    return cfg


def velocity_field(shape, sigma, seed, rho0=1.0):
    """rho = rho0 everywhere; u i.i.d. N(0, sigma^2) per node and component with
    the mean of each component removed. Returns rho (N,) and u (3, N), node
    index (z * ny + y) * nx + x."""
    nx, ny, nz = shape
    n = nx * ny * nz
    rho = np.full(n, rho0, dtype=np.float64)
    if sigma == 0.0:
        return rho, np.zeros((3, n))
    g = np.random.Generator(np.random.PCG64(seed))
    u = g.normal(0.0, sigma, size=(3, n))
    u -= u.mean(axis=1, keepdims=True)
    return rho, u


class _Grid:
    """Hash grid for excluded-volume checks in a periodic box; cell sides
    divide the box exactly so keys wrap cleanly."""

    def __init__(self, box, h):
        self.box = np.asarray(box, dtype=np.float64)
        self.n = [max(1, int(math.floor(self.box[d] / h))) for d in range(3)]
        self.h = [self.box[d] / self.n[d] for d in range(3)]
        self.cells = {}
        self.pts = []

    def key(self, p):
        return tuple(int(math.floor(p[d] / self.h[d])) % self.n[d] for d in range(3))

    def add(self, p):
        k = self.key(p)
        self.cells.setdefault(k, []).append(len(self.pts))
        self.pts.append(np.array(p))

    def pop(self):
        p = self.pts.pop()
        self.cells[self.key(p)].pop()

    def near(self, p):
        k = self.key(p)
        seen = set()
        out = []
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    kk = ((k[0] + dx) % self.n[0], (k[1] + dy) % self.n[1], (k[2] + dz) % self.n[2])
                    if kk in seen:
                        continue
                    seen.add(kk)
                    lst = self.cells.get(kk)
                    if lst:
                        out.extend(lst)
        return out


def _min_image(d, box):
    return d - box * np.round(d / box)


def self_avoiding_chain(n, seed, start, box, step=0.5, exclude=0.4, radius=None,
                        centre=None, grid=None, trials=32, max_rounds=64, planar=False):
    """Self-avoiding random walk of n beads with fixed step length: each new
    bead is placed at a uniformly random direction from the previous one and
    rejected when it comes within `exclude` of any earlier bead (minimum image,
    periodic box) or, if `radius` is given, leaves the sphere of that radius
    around `centre`. planar=True keeps the walk in the plane z = start z and
    directed along +x (directions drawn in the half plane x > 0, so the walk
    never traps itself). Dead ends are left by backtracking a few beads.
    Returns unwrapped positions (3, n)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    box = np.asarray(box, dtype=np.float64)
    if grid is None:
        grid = _Grid(box, max(step + exclude, 1.0))
    base = len(grid.pts)
    pos = [np.asarray(start, dtype=np.float64)]
    grid.add(np.mod(pos[0], box))
    fails = 0
    while len(pos) < n:
        prev = pos[-1]
        placed = False
        for _ in range(max_rounds):
            dirs = rng.normal(size=(trials, 3))
            if planar:
                dirs[:, 2] = 0.0
                dirs[:, 0] = np.abs(dirs[:, 0])
            dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
            cand = prev[None, :] + step * dirs
            ok = np.ones(trials, dtype=bool)
            if radius is not None:
                ok &= np.linalg.norm(cand - np.asarray(centre)[None, :], axis=1) <= radius
            idx = grid.near(np.mod(prev, box))
            if idx:
                pts = np.array([grid.pts[i] for i in idx])
                d = _min_image(np.mod(cand, box)[:, None, :] - pts[None, :, :], box)
                ok &= (np.einsum("tkd,tkd->tk", d, d) >= exclude * exclude).all(axis=1)
            good = np.nonzero(ok)[0]
            if good.size:
                p = cand[good[0]]
                pos.append(p)
                grid.add(np.mod(p, box))
                placed = True
                break
        if not placed:
            fails += 1
            if fails > 1000:
                raise RuntimeError("self-avoiding walk is stuck")
            back = min(len(pos) - 1, 8)
            for _ in range(back):
                pos.pop()
                grid.pop()
    assert len(grid.pts) - base == n
    return np.array(pos).T.copy()


def _chain_bonds(offset, n):
    i = np.arange(n - 1, dtype=np.int64) + offset
    return np.stack([i, i + 1], axis=1)


def _contacts(x, owner, cut):
    """Cross-chain bead pairs closer than `cut` (brute force over a cell hash)."""
    pts = x.T
    h = cut
    cells = {}
    for a, p in enumerate(pts):
        cells.setdefault(tuple(np.floor(p / h).astype(int)), []).append(a)
    pairs = []
    for a, p in enumerate(pts):
        k = tuple(np.floor(p / h).astype(int))
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for b in cells.get((k[0] + dx, k[1] + dy, k[2] + dz), ()):
                        if b > a and owner[b] != owner[a]:
                            r = np.linalg.norm(pts[a] - pts[b])
                            if r < cut:
                                pairs.append((a, b, r))
    return pairs


def solute(cfg, seed):
    """Positions (3, Na), velocities (3, Na, zero), masses, bonds (Nb, 2),
    bond stiffness and rest lengths for a workload."""
    box = np.array([cfg["nx"], cfg["ny"], cfg["nz"]], dtype=np.float64)
    centre = box / 2.0
    step, excl = cfg["bond_r0"], cfg["lj_sigma"]
    chains = cfg["chains"]
    xs, bonds, k, r0, owner = [], [], [], [], []
    grid = _Grid(box, max(step + excl, 1.0))
    if chains == "trimer":
        side = 38.0
        R = side / math.sqrt(3.0)
        centres = [centre + R * np.array([math.cos(a), math.sin(a), 0.0])
                   for a in (math.pi / 2, math.pi / 2 + 2 * math.pi / 3, math.pi / 2 + 4 * math.pi / 3)]
        specs = [dict(n=20000, c=c, radius=20.0) for c in centres]
    elif chains == "grid10":
        specs = [dict(n=20000, c=np.array([(i + 0.5) * box[0] / 5, (j + 0.5) * box[1] / 2, box[2] / 2]),
                      radius=20.0) for j in range(2) for i in range(5)]
    elif chains == "channel4":
        # Four 17k-bead globules (radius 19.5) along x in the mid-plane, and two
        # flat 300-bead walks at z = 0.5 and z = nz - 1.5 next to the walls.
        specs = [dict(n=17000, c=np.array([(i + 0.5) * box[0] / 4, box[1] / 2, box[2] / 2]), radius=19.5)
                 for i in range(4)]
        specs += [dict(n=300, c=np.array([box[0] / 8, box[1] / 2, z]), radius=None, planar=True)
                  for z in (0.5, box[2] - 1.5)]
    else:
        specs = [dict(n=c["n"], c=centre if c["centre"] == "box" else np.asarray(c["centre"]),
                      radius=c["radius"]) for c in chains]
    off = 0
    for ci, s in enumerate(specs):
        x = self_avoiding_chain(s["n"], seed * 1000 + ci, s["c"], box, step=step, exclude=excl,
                                radius=s["radius"], centre=s["c"], grid=grid, planar=s.get("planar", False))
        xs.append(x)
        bonds.append(_chain_bonds(off, s["n"]))
        k.append(np.full(s["n"] - 1, cfg["bond_k"]))
        r0.append(np.full(s["n"] - 1, cfg["bond_r0"]))
        owner.append(np.full(s["n"], ci))
        off += s["n"]
    x = np.concatenate(xs, axis=1)
    bonds = np.concatenate(bonds)
    k = np.concatenate(k)
    r0 = np.concatenate(r0)
    owner = np.concatenate(owner)
    if chains == "trimer":
        # Inter-chain contacts: a harmonic bond at its current length for every
        # cross-chain pair closer than 1.0.
        pairs = _contacts(x, owner, 1.0)
        if pairs:
            pb = np.array([(a, b) for a, b, _ in pairs], dtype=np.int64)
            bonds = np.concatenate([bonds, pb])
            k = np.concatenate([k, np.full(len(pairs), cfg["bond_k"])])
            r0 = np.concatenate([r0, np.array([r for _, _, r in pairs])])
    na = x.shape[1]
    return dict(x=x, v=np.zeros((3, na)), mass=np.full(na, cfg["mass"]), bonds=bonds.astype(np.int32),
                bond_k=k, bond_r0=r0)


def inputs(cfg, seed=1, atoms=True):
    """Complete seeded input set for a workload: rho, u node fields plus the
    solute (empty when atoms=False or the workload has none)."""
    rho, u = velocity_field((cfg["nx"], cfg["ny"], cfg["nz"]), cfg.get("u_sigma", 0.0), seed,
                            cfg.get("rho0", 1.0))
    out = dict(rho=rho, u=u)
    if atoms and cfg.get("chains"):
        out.update(solute(cfg, seed))
    else:
        out.update(x=np.zeros((3, 0)), v=np.zeros((3, 0)), mass=np.zeros(0),
                   bonds=np.zeros((0, 2), np.int32), bond_k=np.zeros(0), bond_r0=np.zeros(0))
    return out
