"""Multirate study of the lock-step coupling (Sec. 2.2: one LB step per MD
step; here n_md velocity-Verlet substeps per LB step): on the 500-bead
harmonic chain (no Lennard-Jones, so trajectories do not diverge
chaotically), the atom velocities after two coupled steps for
n_md = 8..128, for the frozen and the re-interpolated coupling, against each
coupling's own n_md = 512 result, next to the difference between the two
couplings. Printed as a table (the record of the study). Both couplings
converge at second order in the substep (errors fall ~4x per doubling from
n_md = 16; n_md = 8 is unstable: the bond frequency sqrt(2k/m) = 14 times
dt_md exceeds 2), and on this stiff chain the substep error at n_md = 128
(~2e-2) is still larger than the gap between the couplings (~8e-3): the
substep count, more than the choice of coupling, sets the accuracy here."""
import numpy as np

from paper_2305_05025_gb300 import synth


def _run(orc, inp, n_md, reinterp):
    cfg = synth.workload("chain500_lattice32", n_md=n_md, gamma=0.5, lj_eps=0.0, reinterp=int(reinterp),
                         nx=24, ny=20, nz=28)
    topo = orc.Topology(inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"])
    f0 = orc.equilibrium(inp["rho"], inp["u"])
    _, x, v, _ = orc.run(cfg, topo, f0, inp["x"], inp["v"], 2)
    return v


def test_multirate_convergence(orc):
    cfg = synth.workload("chain500_lattice32", lj_eps=0.0, nx=24, ny=20, nz=28)
    inp = dict(synth.inputs(cfg, 2))
    rng = np.random.default_rng(3)
    inp["v"] = 0.05 * rng.standard_normal(inp["v"].shape)
    inp["x"] = inp["x"] - inp["x"].mean(1, keepdims=True) + np.array([[12.0], [10.0], [14.0]])
    ref = {r: _run(orc, inp, 512, r) for r in (False, True)}
    scale = np.abs(ref[False]).max()
    gap = np.abs(ref[True] - ref[False]).max() / scale
    rows = []
    for n_md in (8, 16, 32, 64, 128):
        e = [np.abs(_run(orc, inp, n_md, r) - ref[r]).max() / scale for r in (False, True)]
        rows.append((n_md, e[0], e[1]))
    print("\nmultirate (harmonic chain500, 2 steps, gamma 0.5): rel. L-inf velocity error vs n_md = 512")
    print("n_md  frozen      reinterp    (frozen vs reinterp at 512: %.3e)" % gap)
    for n_md, a, b in rows:
        print(f"{n_md:4d}  {a:.3e}   {b:.3e}")
    assert rows[0][1] > 1.0 and rows[0][2] > 1.0  # n_md = 8: unstable
    for i in range(1, len(rows) - 1):
        for c in (1, 2):
            assert 3.0 < rows[i][c] / rows[i + 1][c] < 5.0, rows
    assert 0.1 * rows[-1][1] < gap < rows[-1][1]
