"""Accuracy measures of a sampler's output (Sec. 5.1): how close a run's posterior approximation is
to the truth, to the data and to other runs. Host-side statistics of the particles and evidence
estimates that the library returns; none of the sampler's arithmetic runs here.

rel_err        Eq. RelErr: weighted l1 distance of the posterior mean to the true coefficients,
               weights sqrt(lambda_k) (each coefficient by its share of the KL expansion)
rel_misfit     Eq. RelMisfit: |Gamma^-1/2 (y - G(mean))|^2 / |Gamma^-1/2 y|^2 on the finest level,
               from the potential Phi(mean) = 1/2 |Gamma^-1/2 (y - G(mean))|^2
ks_distance    Kolmogorov-Smirnov distance sup_x |F_a(x) - F_b(x)| of two equally weighted samples
               (the paper compares marginals of theta_1..theta_3 between runs)
rel_err_evid   |log Z - log Z_ref| / |log Z_ref|, Z_ref the geometric mean of reference estimates
               (log Z_ref the mean of their logarithms)
"""
import numpy as np


def rel_err(mean, theta_true, lam):
    """Eq. RelErr with Lambda^1/2 = sqrt(lam) (the KL eigenvalues of the coefficients)."""
    w = np.sqrt(np.asarray(lam, dtype=np.float64))
    t = np.asarray(theta_true, dtype=np.float64)
    return float(np.sum(w * np.abs(np.asarray(mean, dtype=np.float64) - t)) / np.sum(w * np.abs(t)))


def rel_misfit(phi_at_mean, y, sigma):
    """Eq. RelMisfit for Gamma = sigma^2 I, from Phi at the posterior mean on the finest level."""
    y = np.asarray(y, dtype=np.float64) / sigma
    return float(2.0 * phi_at_mean / np.dot(y, y))


def ks_distance(a, b):
    """Two-sample Kolmogorov-Smirnov distance of equally weighted samples a and b."""
    a = np.sort(np.asarray(a, dtype=np.float64).ravel())
    b = np.sort(np.asarray(b, dtype=np.float64).ravel())
    if a.size == 0 or b.size == 0:
        raise ValueError("empty sample")
    x = np.concatenate([a, b])
    Fa = np.searchsorted(a, x, side="right") / a.size
    Fb = np.searchsorted(b, x, side="right") / b.size
    return float(np.max(np.abs(Fa - Fb)))


def log_z_ref(log_zs):
    """Logarithm of the geometric mean of the evidence estimates exp(log_zs)."""
    return float(np.mean(np.asarray(log_zs, dtype=np.float64)))


def rel_err_evid(log_z, ref):
    """|log Z - log Z_ref| / |log Z_ref| for each estimate log_z."""
    return np.abs(np.asarray(log_z, dtype=np.float64) - ref) / abs(ref)


def pairwise_ks(runs_a, runs_b=None):
    """KS distances of all pairs (one run of a, one of b) per coordinate: runs are [J][m] samples
    of m marginals. With runs_b None, the pairs within runs_a (each unordered pair once), the
    base value of a method's scatter. Returns (mean [m], standard deviation [m], pairs)."""
    A = [np.asarray(r, dtype=np.float64) for r in runs_a]
    if runs_b is None:
        pairs = [(A[i], A[j]) for i in range(len(A)) for j in range(i + 1, len(A))]
    else:
        B = [np.asarray(r, dtype=np.float64) for r in runs_b]
        pairs = [(x, z) for x in A for z in B]
    if not pairs:
        raise ValueError("no pairs")
    m = A[0].shape[1]
    d = np.array([[ks_distance(x[:, k], z[:, k]) for k in range(m)] for x, z in pairs])
    return d.mean(axis=0), d.std(axis=0), len(pairs)
