"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/lbmd.h declares, and rejects invalid parameters before
touching a device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2305_05025_gb300 import build, lbmd
from paper_2305_05025_gb300.synth import workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return lbmd.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "lbmd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbmd_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("lbmd_create", "lbmd_set_state", "lbmd_step", "lbmd_get_fields", "lbmd_backward",
              "lbmd_get_stats", "lbmd_last_error", "lbmd_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    for n in _declared():
        assert hasattr(L, n), n
    assert L.lbmd_version() == 1


def test_params_struct_matches_header():
    text = open(os.path.join(ROOT, "include", "lbmd.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} lbmd_params;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        typ, rest = decl.split(None, 1)
        fields += [(typ, n.strip()) for n in rest.split(",")]
    py = [(n, t) for n, t in lbmd.lbmd_params._fields_]
    assert [n for _, n in fields] == [n for n, _ in py]
    cmap = {"int": C.c_int, "double": C.c_double}
    assert all(cmap[t] is pt for (t, _), (_, pt) in zip(fields, py))


def _create(params, **kw):
    out = C.c_void_p()
    mass = np.ascontiguousarray(kw.get("mass", np.zeros(0)), np.float64)
    bonds = np.ascontiguousarray(kw.get("bonds", np.zeros((0, 2))), np.int32).reshape(-1)
    k = np.ascontiguousarray(kw.get("bond_k", np.zeros(0)), np.float64)
    r0 = np.ascontiguousarray(kw.get("bond_r0", np.zeros(0)), np.float64)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    st = lbmd.lib().lbmd_create(C.byref(params), len(mass), dp(mass), bonds.size // 2,
                                bonds.ctypes.data_as(C.POINTER(C.c_int32)), dp(k), dp(r0), None, C.byref(out))
    return st, out


@pytest.mark.parametrize("change,msg", [
    (dict(tau=0.5), "tau"),
    (dict(nx=0), "lattice"),
    (dict(dt=0.5), "dt"),
    (dict(store=7), "store"),
    (dict(forcing=9), "forcing"),
    (dict(walls_z=1, nz=1), "walls"),
    (dict(deterministic=2), "deterministic"),
    (dict(force_dir=3), "force_dir"),
])
def test_invalid_params_are_rejected_before_device_work(L, change, msg):
    p = lbmd.params_from(workload("chain500_lattice32"))
    for k, v in change.items():
        setattr(p, k, v)
    st, out = _create(p)
    assert st == lbmd.LBMD_ERR_ARG
    assert out.value is None
    assert msg in lbmd.lbmd_last_error(None)


def test_invalid_topology_is_rejected(L):
    p = lbmd.params_from(workload("chain500_lattice32"))
    st, _ = _create(p, mass=[1.0, 1.0], bonds=[[0, 2]], bond_k=[1.0], bond_r0=[0.5])
    assert st == lbmd.LBMD_ERR_ARG and "bond" in lbmd.lbmd_last_error(None)
    st, _ = _create(p, mass=[1.0, -1.0])
    assert st == lbmd.LBMD_ERR_ARG and "mass" in lbmd.lbmd_last_error(None)
    small = lbmd.params_from(workload("chain500_lattice32", nx=2, ny=8, nz=8))
    st, _ = _create(small, mass=[1.0])
    assert st == lbmd.LBMD_ERR_ARG and "cells" in lbmd.lbmd_last_error(None)


def test_null_handle_calls_fail_cleanly(L):
    assert L.lbmd_step(None, 1) == lbmd.LBMD_ERR_ARG
    assert L.lbmd_check(None) == lbmd.LBMD_ERR_ARG
    assert L.lbmd_set_state(None, None, None, None, None, None, 0) == lbmd.LBMD_ERR_ARG
    L.lbmd_destroy(None)


def test_create_without_gpu_reports_cuda_error(L):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = lbmd.params_from(workload("chain500_lattice32", nx=8, ny=8, nz=8))
    st, out = _create(p)
    assert st in (lbmd.LBMD_ERR_CUDA, lbmd.LBMD_ERR_ALLOC)
    assert out.value is None
    assert lbmd.lbmd_last_error(None)
