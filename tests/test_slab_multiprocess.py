"""The z-slab decomposition of the coupled step (paper_2305_05025_gb300.slab)
on two gloo ranks on CPU, against the single-rank FP64 oracle:

- the lattice: each rank collides its own planes (the oracle's per-node
  collision), exchanges the populations that cross its faces into ghost
  planes, and pull-streams locally; after six steps the gathered lattice
  equals the oracle's whole-lattice run bit for bit;
- the coupling across a face: atoms in the top plane of a slab interpolate
  from the plane above (exchanged) and spread onto it (the reverse halo):
  equal to the oracle's interpolation and spread over the whole lattice;
- ownership and ghosts: every atom has one owner; the ghosts of a rank are
  the other ranks' atoms within the pair-list radius of its slab.

The per-rank compute here is the oracle's (test infrastructure): what is
under test is the decomposition's plan and exchanges."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
              [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1],
              [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
NX, NY, NZ = 12, 10, 16
CFG = dict(nx=NX, ny=NY, nz=NZ, tau=0.8, forcing="kolmogorov", force_amp=1e-4, force_dir=0, force_wave_axis=1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _initial():
    import oracle

    rng = np.random.default_rng(21)
    u = 0.01 * rng.standard_normal((3, NX * NY * NZ))
    return oracle.equilibrium(np.ones(NX * NY * NZ), u)


def _rank(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    import oracle
    from paper_2305_05025_gb300 import slab

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle.build.build_oracle()
    ranges = slab.slab_ranges(NZ, world)
    z0, z1 = ranges[rank]
    nzl = z1 - z0

    # --- lattice: collide own planes, exchange crossing populations, pull
    f = _initial().reshape(19, NZ, NY, NX)[:, z0:z1].copy()
    g = oracle.body_force(CFG).reshape(3, NZ, NY, NX)[:, z0:z1]
    for _ in range(6):
        post = np.zeros((19, nzl + 2, NY, NX))
        for z in range(nzl):
            for y in range(NY):
                for x in range(NX):
                    post[:, z + 1, y, x] = oracle.collide_node(CFG["tau"], f[:, z, y, x], g[:, z, y, x])
        post = slab.exchange_crossing(torch.from_numpy(post), rank, world).numpy()
        for i in range(19):
            cx, cy, cz = C[i]
            src = post[i, 1 - cz:1 - cz + nzl]
            f[i] = np.roll(np.roll(src, cy, axis=1), cx, axis=2)
    got = [torch.zeros(19, r[1] - r[0], NY, NX, dtype=torch.float64) for r in ranges]
    dist.all_gather(got, torch.from_numpy(f))

    # --- coupling across the face: atoms in the slab's top plane
    rng = np.random.default_rng(5)
    ufield = 0.01 * rng.standard_normal((3, NZ, NY, NX))
    xa = np.stack([rng.uniform(0, NX, 6), rng.uniform(0, NY, 6), rng.uniform(z1 - 1, z1, 6)])
    Ja = rng.standard_normal((3, 6))
    ext = np.zeros((3, nzl + 1, NY, NX))
    ext[:, :nzl] = ufield[:, z0:z1]
    ext = slab.exchange_above(torch.from_numpy(ext), rank, world).numpy()
    loc = dict(CFG, nz=nzl + 1)
    xl = xa - np.array([[0.0], [0.0], [z0]])
    U = oracle.interp(loc, ext.reshape(3, -1), xl)
    Gext = oracle.spread(loc, xl, Ja).reshape(3, nzl + 1, NY, NX)
    G = slab.reverse_halo(torch.from_numpy(Gext), rank, world).numpy()
    Gs = [torch.zeros(3, r[1] - r[0], NY, NX, dtype=torch.float64) for r in ranges]
    dist.all_gather(Gs, torch.from_numpy(G))
    xs = [torch.zeros(3, 6, dtype=torch.float64) for _ in range(world)]
    Js = [torch.zeros(3, 6, dtype=torch.float64) for _ in range(world)]
    Us = [torch.zeros(3, 6, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(xs, torch.from_numpy(xa))
    dist.all_gather(Js, torch.from_numpy(Ja))
    dist.all_gather(Us, torch.from_numpy(U))
    if rank == 0:
        q.put(dict(f=torch.cat(got, 1).numpy(), G=torch.cat(Gs, 1).numpy(), x=np.concatenate([t.numpy() for t in xs], 1),
                   J=np.concatenate([t.numpy() for t in Js], 1), U=np.concatenate([t.numpy() for t in Us], 1),
                   ufield=ufield))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_slabs_equal_the_whole_lattice(orc):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    topo = orc.Topology(np.zeros(0), np.zeros((0, 2)), [], [])
    fo, _, _, _ = orc.run(CFG, topo, _initial(), np.zeros((3, 0)), np.zeros((3, 0)), 6)
    assert np.array_equal(res["f"].reshape(19, -1), fo)
    Uo = orc.interp(CFG, res["ufield"].reshape(3, -1), res["x"])
    assert np.array_equal(res["U"], Uo)
    Go = orc.spread(CFG, res["x"], res["J"])
    assert np.allclose(res["G"].reshape(3, -1), Go, rtol=0, atol=1e-14)
    assert np.abs(Go.reshape(3, NZ, NY, NX)[:, [0, 8]]).max() > 0  # contributions landed on the faces


def test_ownership_and_ghosts():
    import sys

    sys.path.insert(0, ROOT)
    from paper_2305_05025_gb300 import slab

    rng = np.random.default_rng(3)
    nz, world, width = 40, 3, 1.3
    z = rng.uniform(-5, 45, 2000)
    ranges = slab.slab_ranges(nz, world)
    assert ranges == [(0, 14), (14, 27), (27, 40)]
    owner = slab.atom_owner(z, ranges, nz)
    zw = z % nz
    for r, (a, b) in enumerate(ranges):
        assert np.array_equal(owner == r, (zw >= a) & (zw < b))
    for r, (a, b) in enumerate(ranges):
        gh = set(slab.ghost_atoms(z, r, ranges, nz, width).tolist())
        # brute force: periodic distance from zw to the interval [a, b)
        expect = set()
        for i, v in enumerate(zw):
            if owner[i] == r:
                continue
            dist_ = min((a - v) % nz, (v - b) % nz)
            if dist_ <= width:
                expect.add(i)
        assert gh == expect, r


def _migrate_rank(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    from paper_2305_05025_gb300 import slab

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nz, n, width = 24, 3000, 1.1
    rng = np.random.default_rng(11)
    x_all = rng.uniform(-30, 30, (3, n))
    v_all = rng.standard_normal((3, n))
    ranges = slab.slab_ranges(nz, world)
    mine = slab.atom_owner(x_all[2], ranges, nz) == rank
    ids = np.nonzero(mine)[0]
    # One step of motion: every atom moves by less than one plane.
    step = rng.uniform(-0.9, 0.9, (3, n))
    x_new = x_all + step
    got_ids, got_x, got_v = slab.migrate_atoms(ids, x_new[:, ids], v_all[:, ids], rank, ranges, nz)
    gh_ids, gh_x = slab.exchange_ghosts(got_ids, got_x, rank, ranges, nz, width)
    q.put((rank, got_ids, got_x, got_v, gh_ids, gh_x))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_atom_migration_and_ghost_exchange(world):
    """After one step of motion each rank holds exactly the atoms its slab
    owns (none lost, none twice, positions and velocities carried), and the
    ghost positions it receives are the other ranks' atoms within the list
    radius of its slab (brute force over all atoms)."""
    import sys

    sys.path.insert(0, ROOT)
    from paper_2305_05025_gb300 import slab

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_migrate_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r, *rest = q.get(timeout=300)
        res[r] = rest
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    nz, n, width = 24, 3000, 1.1
    rng = np.random.default_rng(11)
    x_all = rng.uniform(-30, 30, (3, n))
    v_all = rng.standard_normal((3, n))
    x_new = x_all + rng.uniform(-0.9, 0.9, (3, n))
    ranges = slab.slab_ranges(nz, world)
    owner = slab.atom_owner(x_new[2], ranges, nz)
    seen = np.concatenate([res[r][0] for r in range(world)])
    assert np.array_equal(np.sort(seen), np.arange(n))
    for r in range(world):
        ids, xr, vr, gh_ids, gh_x = res[r]
        assert np.array_equal(ids, np.nonzero(owner == r)[0])
        assert np.array_equal(xr, x_new[:, ids]) and np.array_equal(vr, v_all[:, ids])
        expect = slab.ghost_atoms(x_new[2], r, ranges, nz, width)
        assert np.array_equal(np.sort(gh_ids), np.sort(expect)), r
        order = np.argsort(gh_ids)
        assert np.array_equal(gh_x[:, order], x_new[:, np.sort(gh_ids)])
