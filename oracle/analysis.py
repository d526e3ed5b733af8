"""Oracle of the solute observables: the trajectory analyses of the paper's
Sec. 3 (root-mean-square deviation from the starting structure after optimal
superposition, radius of gyration, per-atom root-mean-square fluctuation, and
the covariance matrix whose eigenvectors are the principal components),
applied to the synthetic chains.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may import this module. Plain FP64 numpy; each
function is the definition written out, with numpy.linalg as the library step
(the SVD of the superposition, the eigendecomposition of the covariance).

Readings (the paper names the analyses but not their conventions):
 - The superposition is unweighted (every selected atom counts the same) and
   a proper rotation (det +1) plus a translation, fitted onto the reference
   structure: the Kabsch least-squares problem.
 - RMSF and the covariance are taken over the superposed frames; the
   covariance is the population covariance (1/T), coordinates flattened
   structure-of-arrays (component d of selected atom i at d*n + i).
 - R_g^2 is mass weighted over all atoms, about the centre of mass.
"""
import numpy as np


def radius_gyration2(x, mass):
    """sum_a m_a |x_a - c|^2 / sum_a m_a, c the centre of mass; x (3, n)."""
    x = np.asarray(x, np.float64)
    m = np.asarray(mass, np.float64)
    c = (x * m).sum(1) / m.sum()
    return float((m * ((x - c[:, None]) ** 2).sum(0)).sum() / m.sum())


def superpose(x, ref):
    """Kabsch: the rotation R (det +1) and translation minimising
    sum_i |R (x_i - xbar) + refbar - ref_i|^2. Returns the superposed copy of x
    (3, n) and the RMSD after superposition."""
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    xc = x - x.mean(1, keepdims=True)
    rbar = ref.mean(1, keepdims=True)
    rc = ref - rbar
    H = xc @ rc.T  # 3x3 correlation sum_i x_i ref_i^T
    U, S, Vt = np.linalg.svd(H)
    d = np.sign(np.linalg.det(Vt.T @ U.T))
    D = np.diag([1.0, 1.0, d])
    R = Vt.T @ D @ U.T
    fitted = R @ xc + rbar
    rmsd = float(np.sqrt(((fitted - ref) ** 2).sum() / x.shape[1]))
    return fitted, rmsd


def trajectory(frames, ref):
    """frames: sequence of (3, n) selected positions. Returns the per-frame
    RMSD after superposition, the mean superposed displacement from ref
    (3, n), the per-atom RMSF (n,) and the covariance (3n, 3n) of the
    superposed coordinates."""
    ref = np.asarray(ref, np.float64)
    fitted, rmsd = [], []
    for x in frames:
        f, r = superpose(x, ref)
        fitted.append(f)
        rmsd.append(r)
    Y = np.stack([f.reshape(-1) for f in fitted])  # (T, 3n), component-major
    mean = Y.mean(0)
    Yc = Y - mean
    cov = Yc.T @ Yc / Y.shape[0]
    n = ref.shape[1]
    rmsf = np.sqrt(np.diag(cov).reshape(3, n).sum(0))
    return np.array(rmsd), (mean - ref.reshape(-1)).reshape(3, n), rmsf, cov


def principal_components(cov):
    """Eigenvalues (descending) and eigenvectors (columns) of the covariance."""
    w, v = np.linalg.eigh(cov)
    order = np.argsort(w)[::-1]
    return w[order], v[:, order]
