"""GPU trajectory analyses (lbmd_analysis_*: radius of gyration, RMSD after
optimal superposition, RMSF, covariance of the fluctuations -- the analyses of
the paper's Sec. 3) against the FP64 oracle of oracle/analysis.py, evaluated
on the same frames: the CUDA path's own positions, read back after each step.

Tolerances: R_g^2 and RMSD are FP64 sums (masses held in FP32 on the device:
1e-6 relative); the stored frames are FP32 displacements, so the mean
displacement, RMSF and covariance carry FP32 rounding of the displacements
(1e-5 relative to the largest entry)."""
import numpy as np
import pytest

from oracle import analysis
from paper_2305_05025_gb300 import build, lbmd, synth
from gpu_helpers import make

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbmd.lib()


def _run(cfg, inp, sel, T, x_ref=None):
    h = make(cfg, inp)
    lbmd.lbmd_analysis_begin(h, sel, x_ref, max_frames=T)
    frames, got = [], []
    x0 = lbmd.lbmd_get_fields(h, x=True)["x"]
    for _ in range(T):
        lbmd.lbmd_step(h, 1)
        got.append(lbmd.lbmd_analysis_frame(h))
        frames.append(lbmd.lbmd_get_fields(h, x=True)["x"])
    return h, x0, frames, np.array(got)


def test_analysis_matches_oracle_on_the_chain():
    cfg = synth.workload("chain500_lattice32", n_md=128, gamma=0.05, skin=0.3)
    inp = dict(synth.inputs(cfg, 1))
    inp["mass"] = np.random.default_rng(41).uniform(0.5, 2.0, inp["x"].shape[1])
    sel = np.arange(0, 500, 3)  # 167 atoms: 501 coordinates, a ragged last tile
    T = 21                      # not a multiple of the 16-frame chunk
    h, x0, frames, got = _run(cfg, inp, sel, T)
    ref = x0[:, sel]
    for t, x in enumerate(frames):
        rg2 = analysis.radius_gyration2(x, inp["mass"])
        _, rmsd = analysis.superpose(x[:, sel], ref)
        assert abs(got[t, 0] - rg2) <= 1e-6 * rg2, (t, got[t, 0], rg2)
        assert abs(got[t, 1] - rmsd) <= 1e-6 * rmsd + 1e-9, (t, got[t, 1], rmsd)
    assert got[-1, 1] > 1e-2  # the chain did move
    mean, rmsf, cov = lbmd.lbmd_analysis_result(h)
    o_rmsd, o_mean, o_rmsf, o_cov = analysis.trajectory([x[:, sel] for x in frames], ref)
    print("analysis: max rmsd", o_rmsd.max(), "max rmsf", o_rmsf.max(), "max |cov|", np.abs(o_cov).max())
    assert np.abs(mean - o_mean).max() <= 1e-5 * np.abs(o_mean).max()
    assert np.abs(rmsf - o_rmsf).max() <= 1e-5 * o_rmsf.max()
    assert np.abs(cov - o_cov).max() <= 1e-5 * np.abs(o_cov).max()
    # Principal components: the leading eigenvalues agree.
    w, _ = analysis.principal_components(cov.astype(np.float64))
    wo, _ = analysis.principal_components(o_cov)
    assert np.allclose(w[:5], wo[:5], rtol=1e-4)
    # More frames than reserved are refused.
    with pytest.raises(lbmd.LBMDError) as e:
        lbmd.lbmd_analysis_frame(h)
    assert e.value.status == lbmd.LBMD_ERR_ARG


def test_rigid_motion_of_the_reference_has_zero_rmsd():
    """The reference given explicitly as a rotated and shifted copy of the
    starting positions: a frame taken before any step has RMSD zero (the
    superposition undoes the rigid motion), and after one step the RMSD is
    the oracle's for the new positions."""
    cfg = synth.workload("chain500_lattice32", n_md=128, gamma=0.05, skin=0.3)
    inp = synth.inputs(cfg, 2)
    rng = np.random.default_rng(42)
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    R = np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                  [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                  [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])
    ref = R @ inp["x"] + np.array([[3.0], [-40.0], [7.5]])
    h = make(cfg, inp)
    lbmd.lbmd_analysis_begin(h, None, ref, max_frames=2)
    rg2, rmsd = lbmd.lbmd_analysis_frame(h)
    assert rmsd < 1e-6
    assert np.isclose(rg2, analysis.radius_gyration2(inp["x"], inp["mass"]), rtol=1e-6)
    lbmd.lbmd_step(h, 1)
    x1 = lbmd.lbmd_get_fields(h, x=True)["x"]
    _, rmsd1 = lbmd.lbmd_analysis_frame(h)
    assert np.isclose(rmsd1, analysis.superpose(x1, ref)[1], rtol=1e-6)
    mean, rmsf, _ = lbmd.lbmd_analysis_result(h, cov=False)
    _, o_mean, o_rmsf, _ = analysis.trajectory([inp["x"], x1], ref)
    assert np.abs(rmsf - o_rmsf).max() <= 1e-5 * o_rmsf.max()


def test_analysis_argument_errors():
    cfg = synth.workload("chain500_lattice32", n_md=128, gamma=0.05, skin=0.3)
    inp = synth.inputs(cfg, 1)
    h = make(cfg, inp)
    with pytest.raises(lbmd.LBMDError) as e:
        lbmd.lbmd_analysis_frame(h)
    assert e.value.status == lbmd.LBMD_ERR_STATE
    with pytest.raises(lbmd.LBMDError) as e:
        lbmd.lbmd_analysis_begin(h, [0, 500], None, 4)
    assert e.value.status == lbmd.LBMD_ERR_ARG
    lbmd.lbmd_analysis_begin(h, [7], None, 1)  # one atom: superposition is a translation
    assert lbmd.lbmd_analysis_frame(h)[1] < 1e-6
    lat = lbmd.lbmd_create(dict(synth._COMMON, nx=8, ny=8, nz=8, tau=0.7))
    lbmd.lbmd_set_state(lat, rho=np.ones(512, np.float32), u=np.zeros((3, 512), np.float32))
    with pytest.raises(lbmd.LBMDError) as e:
        lbmd.lbmd_analysis_begin(lat, None, None, 1)
    assert e.value.status == lbmd.LBMD_ERR_ARG
