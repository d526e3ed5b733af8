"""The allocation-free entry point lbmd_fluid_sums_noalloc, for callers that
cannot call cudaMalloc (an engine that owns the device memory through its own
pool, or a loop that cannot take the synchronisation of an allocation): its
sums must equal those of lbmd_get_stats, the handle-based reduction, on two
calls in a row with different inputs (the shared scratch array keeps the
previous call's partials; nothing of it may leak into the next result).

Collected last so that a failure here never hides the other GPU tests."""
import ctypes as C

import numpy as np
import pytest

from paper_2305_05025_gb300 import build, lbmd, synth

pytestmark = pytest.mark.gpu

# Both sides sum the same FP32 populations in FP64, but the reference first
# stores delta f = f - fl32(w_i) in FP32 (exact by Sterbenz's lemma for all
# but ~0.6 % of these values) and adds w_i back in FP64: each value carries
# w_i - fl32(w_i), at most 2^-24 w_i, so the sums differ by up to
# 2^-24 sum_i w_i = 6e-8 of the mass, plus FP64 reordering (~1e-12).
TOL = 1e-7


@pytest.fixture(scope="module")
def L():
    build.build()
    return lbmd.lib()


def _populations(shape, seed):
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    return (w[:, None] * (1.0 + 0.2 * rng.standard_normal((19, n)))).astype(np.float32)


def _reference(shape, f):
    """Mass and fluid momentum through the existing entry point."""
    cfg = dict(synth._COMMON, nx=shape[0], ny=shape[1], nz=shape[2], tau=0.7)
    h = lbmd.lbmd_create(cfg)
    lbmd.lbmd_set_state(h, f=f)
    mass, mom, _ = lbmd.lbmd_get_stats(h)
    lbmd.lbmd_destroy(h)
    return np.array([mass, *mom])


def test_noalloc_sums_match_get_stats_twice(L):
    torch = pytest.importorskip("torch")
    shape = (40, 33, 17)  # ragged: the last 256-node block is partial
    L.lbmd_fluid_sums_noalloc.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
    L.lbmd_fluid_sums_noalloc.restype = C.c_int
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for seed in (1, 2):
        f = _populations(shape, seed)
        ref = _reference(shape, f)
        fd = torch.from_numpy(f).cuda()
        st = L.lbmd_fluid_sums_noalloc(C.c_void_p(fd.data_ptr()), *shape, C.c_void_p(out.data_ptr()), stream)
        assert st == lbmd.LBMD_OK, lbmd.lbmd_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # Mass relative to itself; momenta relative to the largest |sum|.
        assert abs(got[0] - ref[0]) <= TOL * abs(ref[0])
        assert np.abs(got[1:] - ref[1:]).max() <= TOL * np.abs(ref).max()


def test_noalloc_rejects_oversized_lattice(L):
    L.lbmd_fluid_sums_noalloc.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
    L.lbmd_fluid_sums_noalloc.restype = C.c_int
    dummy = C.c_void_p(16)  # never dereferenced: the size check comes first
    st = L.lbmd_fluid_sums_noalloc(dummy, 257, 256, 256, dummy, None)
    assert st == lbmd.LBMD_ERR_ARG
    assert "at most" in lbmd.lbmd_last_error(None)
