"""FP64 CPU oracle of one coupled lattice-Boltzmann / MD step.

Follows Sec. 2.2 of Lauricella et al. (arXiv 2305.05025): the BGK lattice
Boltzmann equation with a source term (Eq. 1), its moments (Eq. 2), Stokes
friction between atoms and fluid with trilinear interpolation over the eight
nearest nodes, the equal and opposite force returned to the fluid, and lock-step
time integration. The arithmetic lives in ``lbmd_oracle.c``; this module only
marshals numpy arrays.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may import this package. It imports nothing from the
CUDA path and the CUDA path imports nothing from it.

parity unpinned: the exact multi-step trajectory of the Lennard-Jones chain
(chaotic in general) has no closed form; it is pinned only through its parts
(each sub-operator below has a pin in ``tests/test_oracle_*.py``).
"""
import ctypes as C
import os

import numpy as np

from .build import LIB, build_oracle

Q = 19
_FORCING = {"none": 0, "uniform": 1, "kolmogorov": 2, "poiseuille": 3}


class _Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("tau", C.c_double), ("rho0", C.c_double), ("gamma", C.c_double),
                ("n_md", C.c_int),
                ("lj_eps", C.c_double), ("lj_sigma", C.c_double), ("lj_rcut", C.c_double),
                ("cell_min", C.c_double),
                ("forcing", C.c_int), ("force_amp", C.c_double),
                ("force_dir", C.c_int), ("force_wave_axis", C.c_int),
                ("walls_z", C.c_int), ("brute_force", C.c_int),
                ("kT", C.c_double), ("seed", C.c_uint64), ("step0", C.c_int64),
                ("coul_c", C.c_double), ("coul_rc", C.c_double), ("reinterp", C.c_int)]


class _Topology(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("mass", C.POINTER(C.c_double)),
                ("n_bonds", C.c_int), ("bonds", C.POINTER(C.c_int32)),
                ("bond_k", C.POINTER(C.c_double)), ("bond_r0", C.POINTER(C.c_double)),
                ("charge", C.POINTER(C.c_double))]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            build_oracle()
        _lib = C.CDLL(LIB)
        _lib.orc_run.restype = C.c_int
        _lib.orc_forces.restype = C.c_int
        _lib.orc_interp.restype = C.c_int
        _lib.orc_spread.restype = C.c_int
        _lib.orc_neighbour_counts.restype = C.c_int
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def params(cfg, brute_force=False):
    """Builds the oracle's parameter block from a workload description (a dict
    with the keys of ``paper_2305_05025_gb300.synth`` configs)."""
    forcing = cfg.get("forcing", "none")
    forcing = _FORCING[forcing] if isinstance(forcing, str) else int(forcing)
    rcut = float(cfg.get("lj_sigma", 0.4)) * float(cfg.get("lj_rcut_over_sigma", 2.5))
    return _Params(int(cfg["nx"]), int(cfg["ny"]), int(cfg["nz"]),
                   float(cfg["tau"]), float(cfg.get("rho0", 1.0)), float(cfg.get("gamma", 0.5)),
                   int(cfg.get("n_md", 32)),
                   float(cfg.get("lj_eps", 1.0)), float(cfg.get("lj_sigma", 0.4)), rcut,
                   rcut + float(cfg.get("skin", 0.0)),
                   forcing, float(cfg.get("force_amp", 0.0)),
                   int(cfg.get("force_dir", 0)), int(cfg.get("force_wave_axis", 1)),
                   int(cfg.get("walls_z", 0)), int(bool(brute_force)),
                   float(cfg.get("kT", 0.0)), int(cfg.get("seed", 0)), int(cfg.get("step0", 0)),
                   float(cfg.get("coul_c", 0.0)), float(cfg.get("coul_rc", rcut)),
                   int(cfg.get("reinterp", 0)))


class Topology:
    """Holds contiguous copies of the atom topology for the C call."""

    def __init__(self, mass, bonds, bond_k, bond_r0, charge=None):
        self.mass = np.ascontiguousarray(mass, dtype=np.float64)
        self.charge = None if charge is None else np.ascontiguousarray(charge, dtype=np.float64)
        self.bonds = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 2))
        self.bond_k = np.ascontiguousarray(bond_k, dtype=np.float64)
        self.bond_r0 = np.ascontiguousarray(bond_r0, dtype=np.float64)
        if self.bonds.size == 0:
            self.bonds = np.zeros((1, 2), np.int32)
            self.nb = 0
        else:
            self.nb = self.bonds.shape[0]
        if self.bond_k.size == 0:
            self.bond_k = np.zeros(1)
            self.bond_r0 = np.zeros(1)
        self.s = _Topology(len(self.mass), _d(self.mass), self.nb, _i(self.bonds),
                           _d(self.bond_k), _d(self.bond_r0),
                           None if self.charge is None else _d(self.charge))


def lattice():
    c = np.zeros(3 * Q, np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, np.int32)
    lib().orc_lattice(_i(c), _d(w), _i(opp))
    return c.reshape(Q, 3), w, opp


def equilibrium(rho, u):
    rho = np.ascontiguousarray(rho, dtype=np.float64).ravel()
    n = rho.size
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(3, n)
    feq = np.zeros((Q, n))
    lib().orc_equilibrium(C.c_int64(n), _d(rho), _d(u), _d(feq))
    return feq


def moments(f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    n = f.shape[1]
    rho = np.zeros(n)
    j = np.zeros((3, n))
    lib().orc_moments(C.c_int64(n), _d(f), _d(rho), _d(j))
    return rho, j


def guo_source(tau, u, F):
    u = np.ascontiguousarray(u, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    S = np.zeros(Q)
    lib().orc_guo_source(C.c_double(tau), _d(u), _d(F), _d(S))
    return S


def collide_node(tau, f, F):
    f = np.ascontiguousarray(f, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(Q)
    lib().orc_collide_node(C.c_double(tau), _d(f), _d(F), _d(out))
    return out


def philox4x32_10(ctr, key):
    """Philox4x32-10 block of the 4-word counter and 2-word key."""
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    out = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, out)
    return [int(v) for v in out]


def mode_basis():
    """D3Q19 moment basis E (19 modes x 19 speeds) and norms b_k = sum w E^2."""
    E = np.zeros((Q, Q))
    b = np.zeros(Q)
    lib().orc_mode_basis(_d(E), _d(b))
    return E, b


def node_noise(cfg, node, step):
    """The thermal noise xi (19,) the oracle adds at a node and step."""
    p = params(cfg)
    xi = np.zeros(Q)
    lib().orc_node_noise(C.byref(p), C.c_int64(int(node)), C.c_int64(int(step)), _d(xi))
    return xi


def body_force(cfg):
    p = params(cfg)
    n = p.nx * p.ny * p.nz
    g = np.zeros((3, n))
    lib().orc_body_force(C.byref(p), _d(g))
    return g


def interp(cfg, ufield, x):
    p = params(cfg)
    ufield = np.ascontiguousarray(ufield, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    na = x.shape[1]
    U = np.zeros((3, na))
    err = lib().orc_interp(C.byref(p), _d(ufield), na, _d(x), _d(U))
    if err:
        raise ValueError(f"orc_interp failed ({err})")
    return U


def spread(cfg, x, J):
    p = params(cfg)
    x = np.ascontiguousarray(x, dtype=np.float64)
    J = np.ascontiguousarray(J, dtype=np.float64)
    G = np.zeros((3, p.nx * p.ny * p.nz))
    err = lib().orc_spread(C.byref(p), x.shape[1], _d(x), _d(J), _d(G))
    if err:
        raise ValueError(f"orc_spread failed ({err})")
    return G


def forces(cfg, topo, x, brute_force=False):
    p = params(cfg, brute_force)
    x = np.ascontiguousarray(x, dtype=np.float64)
    F = np.zeros_like(x)
    e = C.c_double(0.0)
    err = lib().orc_forces(C.byref(p), C.byref(topo.s), _d(x), _d(F), C.byref(e))
    if err:
        raise ValueError(f"orc_forces failed ({err})")
    return F, e.value


def cells(cfg, x):
    p = params(cfg)
    x = np.ascontiguousarray(x, dtype=np.float64)
    cell_of = np.zeros(x.shape[1], np.int32)
    nc = np.zeros(3, np.int32)
    lib().orc_cells(C.byref(p), x.shape[1], _d(x), _i(cell_of), _i(nc))
    return cell_of, nc


def neighbour_counts(cfg, x, brute_force=False):
    p = params(cfg, brute_force)
    x = np.ascontiguousarray(x, dtype=np.float64)
    counts = np.zeros(x.shape[1], np.int32)
    err = lib().orc_neighbour_counts(C.byref(p), x.shape[1], _d(x), _i(counts))
    if err:
        raise ValueError(f"orc_neighbour_counts failed ({err})")
    return counts


def run(cfg, topo, f, x, v, n_steps, brute_force=False):
    """Advances (f, x, v) by n_steps coupled steps; returns new copies and the
    per-step observables (n_steps, 4): drag impulse on the atoms (x, y, z) and
    the squared radius of gyration after the step."""
    p = params(cfg, brute_force)
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    v = np.array(v, dtype=np.float64, order="C", copy=True)
    obs = np.zeros((max(n_steps, 1), 4))
    err = lib().orc_run(C.byref(p), C.byref(topo.s), _d(f), _d(x), _d(v), int(n_steps), _d(obs))
    if err:
        raise ValueError(f"orc_run failed ({err})")
    return f, x, v, obs[:n_steps]
