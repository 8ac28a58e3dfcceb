"""Statistical acceptance rules shared by the parity and accuracy tests."""
import numpy as np


def combined_z(m1, se1, m2, se2):
    """z_i = (m1 - m2) / sqrt(se1^2 + se2^2); zero-variance pairs that agree give 0."""
    den = np.sqrt(np.asarray(se1) ** 2 + np.asarray(se2) ** 2)
    diff = np.asarray(m1) - np.asarray(m2)
    with np.errstate(divide="ignore", invalid="ignore"):
        z = np.where(den > 0, diff / np.where(den > 0, den, 1.0), np.where(diff == 0, 0.0, np.inf))
    return z


def four_se_rule(z, k=4.0):
    """Agreement within k combined standard errors, read for many points at once:
    at most max(2, 3 N 6.3e-5) points beyond k (6.3e-5 is the two-sided normal
    tail at 4 sigma) and a mean z within k / sqrt(N)."""
    z = np.asarray(z, dtype=np.float64)
    n = z.size
    outliers = int(np.sum(np.abs(z) > k))
    allowed = max(2, int(3 * n * 6.3e-5))
    mean_ok = abs(float(np.mean(z[np.isfinite(z)]))) <= k / np.sqrt(n)
    return outliers <= allowed and mean_ok and np.all(np.isfinite(z)), outliers, float(np.mean(z))


def normalised_rms(est, exact):
    """||est - exact||_2 / ||exact||_2 over the evaluation points."""
    est = np.asarray(est, dtype=np.float64)
    exact = np.asarray(exact, dtype=np.float64)
    return float(np.linalg.norm(est - exact) / np.linalg.norm(exact))
