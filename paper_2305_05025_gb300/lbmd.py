"""ctypes binding of liblbmd.so (the C ABI declared in include/lbmd.h).

Argument marshalling only: every step of the coupled LB-MD update runs in the
library's CUDA kernels. Inputs may be numpy arrays (host, on_device=0) or CUDA
torch tensors (device, on_device=1); outputs come back as numpy arrays unless
device tensors are requested. There is no CPU fallback: if the library is
missing or no GPU is present the calls raise.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

Q = 19

LBMD_OK, LBMD_ERR_ARG, LBMD_ERR_ALLOC, LBMD_ERR_CUDA, LBMD_ERR_NONFINITE, LBMD_ERR_CELL, LBMD_ERR_STATE = range(7)
STATUS_NAMES = {0: "LBMD_OK", 1: "LBMD_ERR_ARG", 2: "LBMD_ERR_ALLOC", 3: "LBMD_ERR_CUDA",
                4: "LBMD_ERR_NONFINITE", 5: "LBMD_ERR_CELL", 6: "LBMD_ERR_STATE"}
STORES = {"f32": 0, "f16": 1, "bf16": 2}
FORCING = {"none": 0, "uniform": 1, "kolmogorov": 2, "poiseuille": 3}
OBS_DRAG_X, OBS_RG2 = 0, 1


class LBMDError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class lbmd_params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("tau", C.c_double), ("rho0", C.c_double), ("gamma", C.c_double), ("dt", C.c_double),
                ("n_md", C.c_int),
                ("lj_eps", C.c_double), ("lj_sigma", C.c_double), ("lj_rcut_over_sigma", C.c_double),
                ("skin", C.c_double),
                ("forcing", C.c_int), ("force_amp", C.c_double), ("force_dir", C.c_int),
                ("force_wave_axis", C.c_int), ("walls_z", C.c_int), ("store", C.c_int),
                ("deterministic", C.c_int), ("check_every", C.c_int)]


def params_from(cfg):
    """lbmd_params from a workload description (keys of synth.WORKLOADS)."""
    forcing = cfg.get("forcing", "none")
    store = cfg.get("store", "f32")
    return lbmd_params(int(cfg["nx"]), int(cfg["ny"]), int(cfg["nz"]),
                       float(cfg["tau"]), float(cfg.get("rho0", 1.0)), float(cfg.get("gamma", 0.5)), 1.0,
                       int(cfg.get("n_md", 32)),
                       float(cfg.get("lj_eps", 1.0)), float(cfg.get("lj_sigma", 0.4)),
                       float(cfg.get("lj_rcut_over_sigma", 2.5)), float(cfg.get("skin", 0.0)),
                       FORCING[forcing] if isinstance(forcing, str) else int(forcing),
                       float(cfg.get("force_amp", 0.0)), int(cfg.get("force_dir", 0)),
                       int(cfg.get("force_wave_axis", 1)), int(cfg.get("walls_z", 0)),
                       STORES[store] if isinstance(store, str) else int(store),
                       int(cfg.get("deterministic", 0)), int(cfg.get("check_every", 0)))


_lib = None


def lib():
    """Loads liblbmd.so from the package directory (built by build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing: build it with paper_2305_05025_gb300.build.build() "
                               "(or __graft_entry__.build())")
        L = C.CDLL(_build.LIB)
        vp, ip, i32p = C.c_void_p, C.c_int, C.POINTER(C.c_int32)
        dp = C.POINTER(C.c_double)
        L.lbmd_create.argtypes = [C.POINTER(lbmd_params), ip, dp, ip, i32p, dp, dp, vp, C.POINTER(vp)]
        L.lbmd_set_state.argtypes = [vp, vp, vp, vp, vp, vp, ip]
        L.lbmd_step.argtypes = [vp, ip]
        L.lbmd_get_fields.argtypes = [vp, vp, vp, vp, vp, vp, ip]
        L.lbmd_save_state.argtypes = [vp, vp, vp, vp, ip]
        L.lbmd_load_state.argtypes = [vp, vp, vp, vp, ip]
        L.lbmd_get_stats.argtypes = [vp, dp, dp, dp]
        L.lbmd_check.argtypes = [vp]
        L.lbmd_cell_list.argtypes = [vp, vp, vp, vp, ip]
        L.lbmd_set_physics.argtypes = [vp, C.c_double, C.c_double, C.c_double]
        L.lbmd_set_timing_events.argtypes = [vp, vp, vp]
        L.lbmd_set_md_timing_events.argtypes = [vp, vp, vp]
        L.lbmd_set_thermal.argtypes = [vp, C.c_double, C.c_uint64]
        L.lbmd_set_charges.argtypes = [vp, vp, C.c_double, C.c_double]
        L.lbmd_set_reinterpolation.argtypes = [vp, ip]
        L.lbmd_analysis_begin.argtypes = [vp, ip, vp, vp, ip]
        L.lbmd_analysis_frame.argtypes = [vp, dp, dp]
        L.lbmd_analysis_result.argtypes = [vp, vp, vp, vp, ip]
        L.lbmd_backward.argtypes = [vp, ip, ip, ip, dp, dp, dp, dp]
        L.lbmd_backward_state.argtypes = [vp, ip, ip, ip, dp, vp, vp, vp, ip]
        L.lbmd_last_error.argtypes = [vp]
        L.lbmd_last_error.restype = C.c_char_p
        L.lbmd_destroy.argtypes = [vp]
        L.lbmd_destroy.restype = None
        for name in ("lbmd_create", "lbmd_set_state", "lbmd_step", "lbmd_get_fields", "lbmd_get_stats",
                     "lbmd_check", "lbmd_cell_list", "lbmd_set_physics", "lbmd_set_timing_events", "lbmd_set_md_timing_events",
                     "lbmd_analysis_begin", "lbmd_analysis_frame", "lbmd_analysis_result", "lbmd_set_thermal", "lbmd_set_charges",
                     "lbmd_set_reinterpolation", "lbmd_backward_state",
                     "lbmd_backward", "lbmd_version"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(h, status):
    if status != LBMD_OK:
        raise LBMDError(status, lbmd_last_error(h))


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype, shape, keep):
    """Device pointer of a CUDA tensor, or host pointer of a contiguous numpy
    copy (kept alive in `keep`). Returns (pointer, on_device)."""
    if a is None:
        return None, None
    if _is_torch(a):
        import torch

        tdt = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if not a.is_cuda or a.dtype != tdt or not a.is_contiguous() or a.numel() != int(np.prod(shape)):
            raise ValueError(f"expected a contiguous CUDA {tdt} tensor with {int(np.prod(shape))} elements")
        keep.append(a)
        return C.c_void_p(a.data_ptr()), 1
    arr = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    if arr.size != int(np.prod(shape)):
        raise ValueError(f"expected {int(np.prod(shape))} elements, got {arr.size}")
    keep.append(arr)
    return arr.ctypes.data_as(C.c_void_p), 0


def lbmd_last_error(h):
    msg = lib().lbmd_last_error(h)
    return msg.decode() if msg else ""


def _current_stream():
    try:
        import torch

        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return C.c_void_p(0)


class Handle:
    """Owns an lbmd_t; carries the sizes the marshalling needs."""

    def __init__(self, ptr, params, n_atoms):
        self.ptr = ptr
        self.params = params
        self.n_atoms = n_atoms
        self.N = params.nx * params.ny * params.nz

    @property
    def _as_parameter_(self):
        return self.ptr

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                lib().lbmd_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


def lbmd_create(params, mass=None, bonds=None, bond_k=None, bond_r0=None, stream=None):
    """params: lbmd_params or a workload dict. Topology arrays are host arrays."""
    if not isinstance(params, lbmd_params):
        params = params_from(params)
    mass = np.ascontiguousarray(np.zeros(0) if mass is None else mass, dtype=np.float64)
    bonds = np.ascontiguousarray(np.zeros((0, 2)) if bonds is None else bonds, dtype=np.int32).reshape(-1)
    nb = bonds.size // 2
    bond_k = np.ascontiguousarray(np.zeros(0) if bond_k is None else bond_k, dtype=np.float64)
    bond_r0 = np.ascontiguousarray(np.zeros(0) if bond_r0 is None else bond_r0, dtype=np.float64)
    out = C.c_void_p()
    st = _current_stream() if stream is None else C.c_void_p(stream)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    status = lib().lbmd_create(C.byref(params), len(mass), dp(mass), nb,
                               bonds.ctypes.data_as(C.POINTER(C.c_int32)), dp(bond_k), dp(bond_r0), st,
                               C.byref(out))
    if status != LBMD_OK:
        raise LBMDError(status, lbmd_last_error(None))
    return Handle(out, params, len(mass))


def lbmd_set_state(h, f=None, rho=None, u=None, x=None, v=None):
    keep = []
    N, na = h.N, h.n_atoms
    pf, d1 = _ptr(f, np.float32, (Q, N), keep)
    pr, d2 = _ptr(rho, np.float32, (N,), keep)
    pu, d3 = _ptr(u, np.float32, (3, N), keep)
    px, d4 = _ptr(x, np.float64, (3, na), keep)
    pv, d5 = _ptr(v, np.float32, (3, na), keep)
    flags = {d for d in (d1, d2, d3, d4, d5) if d is not None}
    if len(flags) > 1:
        raise ValueError("mix of host and device inputs")
    on_dev = flags.pop() if flags else 0
    _check(h, lib().lbmd_set_state(h, pf, pr, pu, px, pv, on_dev))


def lbmd_step(h, n_steps=1):
    _check(h, lib().lbmd_step(h, int(n_steps)))


def lbmd_get_fields(h, f=False, rho=False, u=False, x=False, v=False, out=None):
    """Returns a dict of numpy arrays for the requested fields; with `out`
    (a dict of preallocated CUDA tensors) fills those on the device instead."""
    N, na = h.N, h.n_atoms
    keep = []
    if out is not None:
        ptrs = {}
        for name, dt, shape in (("f", np.float32, (Q, N)), ("rho", np.float32, (N,)), ("u", np.float32, (3, N)),
                                ("x", np.float64, (3, na)), ("v", np.float32, (3, na))):
            p, _ = _ptr(out.get(name), dt, shape, keep)
            ptrs[name] = p
        _check(h, lib().lbmd_get_fields(h, ptrs["f"], ptrs["rho"], ptrs["u"], ptrs["x"], ptrs["v"], 1))
        return out
    res = {}
    if f:
        res["f"] = np.zeros((Q, N), np.float32)
    if rho:
        res["rho"] = np.zeros(N, np.float32)
    if u:
        res["u"] = np.zeros((3, N), np.float32)
    if x:
        res["x"] = np.zeros((3, na), np.float64)
    if v:
        res["v"] = np.zeros((3, na), np.float32)
    p = lambda k: res[k].ctypes.data_as(C.c_void_p) if k in res else None
    _check(h, lib().lbmd_get_fields(h, p("f"), p("rho"), p("u"), p("x"), p("v"), 0))
    return res


def _pop_dtype(h):
    """Element type of the handle's population storage (the raw snapshot)."""
    return np.float32 if h.params.store == STORES["f32"] else np.uint16


def lbmd_save_state(h, out=None):
    """Raw snapshot (pop in the storage format, x, v) as numpy arrays; with
    `out` (a dict of CUDA tensors "pop" (float32 or int16/uint16-sized), "x",
    "v") fills those on the device."""
    N, na = h.N, h.n_atoms
    if out is not None:
        keep = []
        pop = out["pop"]
        if not (_is_torch(pop) and pop.is_cuda and pop.is_contiguous()
                and pop.numel() * pop.element_size() == Q * N * np.dtype(_pop_dtype(h)).itemsize):
            raise ValueError("pop: a contiguous CUDA tensor of 19*N storage elements")
        px, _ = _ptr(out.get("x"), np.float64, (3, na), keep)
        pv, _ = _ptr(out.get("v"), np.float32, (3, na), keep)
        _check(h, lib().lbmd_save_state(h, C.c_void_p(pop.data_ptr()), px, pv, 1))
        return out
    res = {"pop": np.zeros((Q, N), _pop_dtype(h)), "x": np.zeros((3, na), np.float64), "v": np.zeros((3, na), np.float32)}
    p = lambda k: res[k].ctypes.data_as(C.c_void_p)
    _check(h, lib().lbmd_save_state(h, p("pop"), p("x") if na else None, p("v") if na else None, 0))
    return res


def lbmd_load_state(h, pop, x=None, v=None):
    """Restores a snapshot of lbmd_save_state (numpy arrays, or CUDA tensors
    for all three)."""
    N, na = h.N, h.n_atoms
    keep = []
    if _is_torch(pop):
        if not (pop.is_cuda and pop.is_contiguous()
                and pop.numel() * pop.element_size() == Q * N * np.dtype(_pop_dtype(h)).itemsize):
            raise ValueError("pop: a contiguous CUDA tensor of 19*N storage elements")
        pp, dp_ = C.c_void_p(pop.data_ptr()), 1
        keep.append(pop)
    else:
        arr = np.ascontiguousarray(np.asarray(pop, dtype=_pop_dtype(h)))
        if arr.size != Q * N:
            raise ValueError(f"expected {Q * N} elements, got {arr.size}")
        keep.append(arr)
        pp, dp_ = arr.ctypes.data_as(C.c_void_p), 0
    px, d1 = _ptr(x, np.float64, (3, na), keep)
    pv, d2 = _ptr(v, np.float32, (3, na), keep)
    if any(d is not None and d != dp_ for d in (d1, d2)):
        raise ValueError("mix of host and device inputs")
    _check(h, lib().lbmd_load_state(h, pp, px, pv, dp_))


def lbmd_get_stats(h):
    m = C.c_double()
    pf = (C.c_double * 3)()
    pa = (C.c_double * 3)()
    _check(h, lib().lbmd_get_stats(h, C.byref(m), pf, pa))
    return m.value, np.array(pf[:]), np.array(pa[:])


def lbmd_check(h):
    _check(h, lib().lbmd_check(h))


def lbmd_cell_list(h):
    na = h.n_atoms
    cell = np.zeros(max(na, 1), np.int32)
    neigh = np.zeros(max(na, 1), np.int32)
    nc = np.zeros(3, np.int32)
    v = lambda a: a.ctypes.data_as(C.c_void_p)
    _check(h, lib().lbmd_cell_list(h, v(cell), v(neigh), v(nc), 0))
    return cell[:na], neigh[:na], nc


def lbmd_set_physics(h, gamma, tau, force_amp):
    _check(h, lib().lbmd_set_physics(h, float(gamma), float(tau), float(force_amp)))
    h.params.gamma, h.params.tau, h.params.force_amp = float(gamma), float(tau), float(force_amp)


def lbmd_set_charges(h, charge, coul_c=0.0, coul_rc=1.0):
    """Screened Coulomb pairs (see include/lbmd.h); charge None turns them off.
    Call before lbmd_set_state."""
    keep = []
    p, _ = (None, None) if charge is None else _ptr(np.asarray(charge, np.float64), np.float64, (h.n_atoms,), keep)
    _check(h, lib().lbmd_set_charges(h, p, float(coul_c), float(coul_rc)))


def lbmd_set_reinterpolation(h, on=True):
    """Fluid velocity re-interpolated at every substep (see include/lbmd.h)."""
    _check(h, lib().lbmd_set_reinterpolation(h, int(bool(on))))


def lbmd_set_thermal(h, kT, seed=0):
    """Thermal noise of the fluid: kT > 0 turns it on (see include/lbmd.h)."""
    _check(h, lib().lbmd_set_thermal(h, float(kT), int(seed) & 0xFFFFFFFFFFFFFFFF))


def lbmd_set_timing_events(h, ev_start=None, ev_stop=None):
    """ev_start/ev_stop: torch.cuda.Event(enable_timing=True) or raw cudaEvent_t
    handles; None restores the library's own events."""
    def raw(e):
        if e is None:
            return None
        return C.c_void_p(e.cuda_event if hasattr(e, "cuda_event") else int(e))
    _check(h, lib().lbmd_set_timing_events(h, raw(ev_start), raw(ev_stop)))


def lbmd_set_md_timing_events(h, ev_start=None, ev_stop=None):
    """Events around the substep kernels of the next step launches (see
    lbmd_set_timing_events)."""
    def raw(e):
        if e is None:
            return None
        return C.c_void_p(e.cuda_event if hasattr(e, "cuda_event") else int(e))
    _check(h, lib().lbmd_set_md_timing_events(h, raw(ev_start), raw(ev_stop)))


def lbmd_backward(h, n_steps, ckpt_every, observable=OBS_DRAG_X):
    """Returns (observable, d/dgamma, d/dtau, d/dforce_amp)."""
    vals = [C.c_double() for _ in range(4)]
    _check(h, lib().lbmd_backward(h, int(n_steps), int(ckpt_every), int(observable),
                                  C.byref(vals[0]), C.byref(vals[1]), C.byref(vals[2]), C.byref(vals[3])))
    return vals[3].value, vals[0].value, vals[1].value, vals[2].value


def lbmd_analysis_begin(h, sel=None, x_ref=None, max_frames=1):
    """Starts a trajectory analysis of the atoms `sel` (None: all) against the
    reference x_ref (3, n_sel) (None: their current positions)."""
    keep = []
    n = h.n_atoms if sel is None else len(sel)
    ps, _ = (None, None) if sel is None else _ptr(np.asarray(sel, np.int32), np.int32, (n,), keep)
    pr, _ = (None, None) if x_ref is None else _ptr(np.asarray(x_ref, np.float64), np.float64, (3, n), keep)
    _check(h, lib().lbmd_analysis_begin(h, int(n), ps, pr, int(max_frames)))
    h.ana_n = n


def lbmd_analysis_frame(h):
    """Returns (R_g^2 of all atoms, RMSD of the selection after superposition)."""
    rg2, rmsd = C.c_double(), C.c_double()
    _check(h, lib().lbmd_analysis_frame(h, C.byref(rg2), C.byref(rmsd)))
    return rg2.value, rmsd.value


def lbmd_analysis_result(h, cov=True):
    """Returns (mean displacement (3, n), RMSF (n,), covariance (3n, 3n) FP32 or None)."""
    n = h.ana_n
    mean = np.zeros((3, n))
    rmsf = np.zeros(n)
    c = np.zeros((3 * n, 3 * n), np.float32) if cov else None
    p = lambda a: None if a is None else a.ctypes.data_as(C.c_void_p)
    _check(h, lib().lbmd_analysis_result(h, p(mean), p(rmsf), p(c), 0))
    return mean, rmsf, c


def lbmd_backward_state(h, n_steps, ckpt_every, observable=OBS_DRAG_X):
    """Returns (observable, d obs/d f0 (19, N), d obs/d x0 (3, n), d obs/d v0 (3, n))."""
    obs = C.c_double()
    gf = np.zeros((Q, h.N), np.float32)
    gx = np.zeros((3, h.n_atoms), np.float32)
    gv = np.zeros((3, h.n_atoms), np.float32)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    _check(h, lib().lbmd_backward_state(h, int(n_steps), int(ckpt_every), int(observable), C.byref(obs), p(gf),
                                        p(gx), p(gv), 0))
    return obs.value, gf, gx, gv


def lbmd_destroy(h):
    if h.ptr:
        lib().lbmd_destroy(h.ptr)
        h.ptr = None


def lbmd_version():
    return lib().lbmd_version()


def observable_function():
    """torch.autograd.Function over a differentiable rollout: forward runs
    lbmd_backward (observable and its gradients in one pass, the state ends
    advanced by n_steps), backward scales the stored gradients. Usage:
    LBMDObservable.apply(gamma, tau, force_amp, handle, n_steps, ckpt_every,
    observable) with 0-d float64 tensors for the three parameters."""
    import torch

    class LBMDObservable(torch.autograd.Function):
        @staticmethod
        def forward(ctx, gamma, tau, force_amp, handle, n_steps, ckpt_every, observable):
            lbmd_set_physics(handle, float(gamma), float(tau), float(force_amp))
            obs, dg, dt, da = lbmd_backward(handle, n_steps, ckpt_every, observable)
            ctx.save_for_backward(torch.tensor([dg, dt, da], dtype=torch.float64))
            return torch.tensor(obs, dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad):
            (d,) = ctx.saved_tensors
            return grad * d[0], grad * d[1], grad * d[2], None, None, None, None

    return LBMDObservable
