"""Host-side plan of a z-slab decomposition of the coupled step over ranks
(one GPU each; the paper's own runs decompose the box over CPU ranks,
Sec. 2.2). Each rank owns a slab of whole z planes and the atoms whose
position lies in it; per step it exchanges with its two neighbours:

- the post-collision populations that cross its faces (the 5 speeds with
  c_z = +1 leave through the upper face, the 5 with c_z = -1 through the
  lower one) into a ghost plane on each side, so the pull of the dense
  lattice kernel finds them there;
- the populations of the plane just above the slab (the interpolation
  stencil of an atom in the slab's top plane reaches it);
- the coupling force its atoms spread onto that plane (the reverse halo:
  summed into the owner's plane);
- the positions of atoms within the pair-list radius of a face, at every
  substep, and the atoms that left the slab, once per step.

This module holds the partition, the index plans and the exchanges over
torch.distributed (gloo or NCCL), on tensors the caller provides. It
computes nothing of the method itself: the per-rank compute is the
library's step on the rank's slab.
"""
import numpy as np

# D3Q19 speeds with c_z = +1 and -1 (the ABI order: 5, 11, 14, 15, 18 have
# c_z = +1; 6, 12, 13, 16, 17 have c_z = -1).
UP = (5, 11, 14, 15, 18)
DOWN = (6, 12, 13, 16, 17)


def slab_ranges(nz, world):
    """[(z0, z1)] per rank: contiguous slabs of whole planes, the first
    nz % world ranks one plane thicker."""
    if world < 1 or nz < world:
        raise ValueError("need 1 <= world <= nz")
    base, extra = divmod(nz, world)
    out, z = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


def neighbours(rank, world):
    """(lower, upper) neighbour ranks on the periodic ring of slabs."""
    return (rank - 1) % world, (rank + 1) % world


def atom_owner(z, ranges, nz):
    """Owning rank of each atom: the slab holding floor(z) wrapped into the box."""
    zc = np.floor(np.asarray(z, np.float64)).astype(np.int64) % nz
    bounds = np.array([r[1] for r in ranges])
    return np.searchsorted(bounds, zc, side="right")


def ghost_atoms(z, rank, ranges, nz, width):
    """Atoms owned by other ranks that lie within `width` of this rank's slab
    [z0, z1) along z (periodic): the atoms whose positions a rank needs for
    the pair forces of its own atoms (width = pair-list radius)."""
    z = np.asarray(z, np.float64) % nz
    z0, z1 = ranges[rank]
    # distance from the slab interval on the ring
    below = (z0 - z) % nz  # how far below z0
    above = (z - z1) % nz  # how far at or above z1
    near = (below <= width) | (above <= width)
    owner = atom_owner(z, ranges, nz)
    return np.nonzero(near & (owner != rank))[0]


def exchange_crossing(post, rank, world, group=None):
    """Fills the two ghost planes of a rank's post-collision populations
    post (19, nz_local + 2, ny, nx): ghost plane 0 receives, for the speeds
    UP, the lower neighbour's last interior plane; ghost plane nz_local + 1
    receives, for the speeds DOWN, the upper neighbour's first interior
    plane. After it, the pull of every interior node finds its populations
    locally. A torch tensor on the device of the process group's backend."""
    import torch.distributed as dist

    lo, hi = neighbours(rank, world)
    nzl = post.shape[1] - 2
    up_send = post[list(UP), nzl].contiguous()  # to the upper neighbour's ghost plane 0
    down_send = post[list(DOWN), 1].contiguous()  # to the lower neighbour's top ghost plane
    up_recv = torch_empty_like(up_send)
    down_recv = torch_empty_like(down_send)
    # distinct tags: with two ranks both neighbours are the same peer
    ops = [dist.P2POp(dist.isend, up_send, hi, group, 1), dist.P2POp(dist.irecv, up_recv, lo, group, 1),
           dist.P2POp(dist.isend, down_send, lo, group, 2), dist.P2POp(dist.irecv, down_recv, hi, group, 2)]
    for r in dist.batch_isend_irecv(ops):
        r.wait()
    post[list(UP), 0] = up_recv
    post[list(DOWN), nzl + 1] = down_recv
    return post


def exchange_above(planes, rank, world, group=None):
    """planes (C, nz_local + 1, ny, nx): fills plane nz_local (the one above
    the slab) with the upper neighbour's first plane, for any per-node field
    (populations for the interpolation stencils of the top plane's atoms)."""
    import torch.distributed as dist

    lo, hi = neighbours(rank, world)
    nzl = planes.shape[1] - 1
    send = planes[:, 0].contiguous()
    recv = torch_empty_like(send)
    ops = [dist.P2POp(dist.isend, send, lo, group), dist.P2POp(dist.irecv, recv, hi, group)]
    for r in dist.batch_isend_irecv(ops):
        r.wait()
    planes[:, nzl] = recv
    return planes


def reverse_halo(G, rank, world, group=None):
    """G (C, nz_local + 1, ny, nx): the coupling force a rank's atoms spread,
    its last plane lying on the upper neighbour's first plane. Sends that
    plane up and adds the plane received from below into the first plane;
    returns the interior planes (C, nz_local, ny, nx)."""
    import torch.distributed as dist

    lo, hi = neighbours(rank, world)
    nzl = G.shape[1] - 1
    send = G[:, nzl].contiguous()
    recv = torch_empty_like(send)
    ops = [dist.P2POp(dist.isend, send, hi, group), dist.P2POp(dist.irecv, recv, lo, group)]
    for r in dist.batch_isend_irecv(ops):
        r.wait()
    out = G[:, :nzl].clone()
    out[:, 0] += recv
    return out


def torch_empty_like(t):
    import torch

    return torch.empty_like(t)


def _exchange_rows(send_lo, send_hi, rank, world, group=None, tag=0):
    """Sends the float64 row block send_lo (k, m_lo) to the lower neighbour
    and send_hi (k, m_hi) to the upper one; returns the blocks received from
    the lower and the upper neighbour. Counts go first, so the blocks may
    have any length (0 included)."""
    import torch
    import torch.distributed as dist

    lo, hi = neighbours(rank, world)
    k = send_lo.shape[0]
    n_out = [torch.tensor([send_lo.shape[1]], dtype=torch.int64), torch.tensor([send_hi.shape[1]], dtype=torch.int64)]
    n_in = [torch.zeros(1, dtype=torch.int64), torch.zeros(1, dtype=torch.int64)]
    ops = [dist.P2POp(dist.isend, n_out[0], lo, group, tag + 1), dist.P2POp(dist.irecv, n_in[1], hi, group, tag + 1),
           dist.P2POp(dist.isend, n_out[1], hi, group, tag + 2), dist.P2POp(dist.irecv, n_in[0], lo, group, tag + 2)]
    for r in dist.batch_isend_irecv(ops):
        r.wait()
    r_lo = torch.zeros((k, int(n_in[0])), dtype=torch.float64)
    r_hi = torch.zeros((k, int(n_in[1])), dtype=torch.float64)
    ops = []
    if send_lo.shape[1]:
        ops.append(dist.P2POp(dist.isend, send_lo.contiguous(), lo, group, tag + 3))
    if r_hi.shape[1]:
        ops.append(dist.P2POp(dist.irecv, r_hi, hi, group, tag + 3))
    if send_hi.shape[1]:
        ops.append(dist.P2POp(dist.isend, send_hi.contiguous(), hi, group, tag + 4))
    if r_lo.shape[1]:
        ops.append(dist.P2POp(dist.irecv, r_lo, lo, group, tag + 4))
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()
    return r_lo, r_hi


def migrate_atoms(ids, x, v, rank, ranges, nz, group=None):
    """Once per step: the atoms a rank holds whose position left its slab go
    to the neighbour that now owns them (an atom moves far less than a slab
    per step, so only the two neighbours can be the new owner). ids (n,)
    global atom indices, x (3, n) unwrapped FP64 positions, v (3, n); returns
    the rank's atoms after the exchange, in the same layout, sorted by id."""
    import torch

    world = len(ranges)
    if world == 1:
        order = np.argsort(ids, kind="stable")
        return ids[order], x[:, order], v[:, order]
    lo, hi = neighbours(rank, world)
    owner = atom_owner(x[2], ranges, nz)
    stay = owner == rank
    if not np.all(stay | (owner == lo) | (owner == hi)):
        raise ValueError("an atom moved past a neighbouring slab in one step")
    pack = lambda m: torch.from_numpy(np.vstack([ids[m][None].astype(np.float64), x[:, m], v[:, m]]))
    # With two ranks both neighbours are the same rank: send everything leaving once.
    to_lo = (owner == lo) & ~stay
    to_hi = (owner == hi) & ~stay & ~to_lo
    r_lo, r_hi = _exchange_rows(pack(to_lo), pack(to_hi), rank, world, group, tag=10)
    got = np.hstack([np.vstack([ids[stay][None].astype(np.float64), x[:, stay], v[:, stay]]), r_lo.numpy(), r_hi.numpy()])
    order = np.argsort(got[0], kind="stable")
    got = got[:, order]
    return got[0].astype(np.int64), got[1:4], got[4:7]


def exchange_ghosts(ids, x, rank, ranges, nz, width, group=None):
    """Every substep: the positions of this rank's atoms within `width` (the
    pair-list radius) of its lower and upper faces go to the neighbour on that
    side; returns (ghost ids, ghost positions) received, the other ranks'
    atoms within `width` of this slab (those ghost_atoms names). Slabs are
    assumed thicker than `width`, so only the neighbours hold ghosts."""
    import torch

    world = len(ranges)
    if world == 1:
        return np.zeros(0, np.int64), np.zeros((3, 0))
    lo, hi = neighbours(rank, world)
    z0, z1 = ranges[rank]
    zw = np.asarray(x[2], np.float64) % nz
    near_lo = (zw - z0) % nz <= width  # within width above the lower face
    near_hi = (z1 - zw) % nz <= width  # within width below the upper face
    pack = lambda m: torch.from_numpy(np.vstack([ids[m][None].astype(np.float64), x[:, m]]))
    if world == 2:  # one neighbour on both sides: send the union once
        r_lo, r_hi = _exchange_rows(pack(near_lo | near_hi), pack(np.zeros_like(near_lo)), rank, world, group, tag=20)
    else:
        r_lo, r_hi = _exchange_rows(pack(near_lo), pack(near_hi), rank, world, group, tag=20)
    got = np.hstack([r_lo.numpy(), r_hi.numpy()])
    return got[0].astype(np.int64), got[1:4]
