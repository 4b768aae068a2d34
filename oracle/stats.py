"""Oracle: distribution and convergence statistics (test infrastructure only).

* per-output moments (mean, variance, skewness) of exit-state samples;
* the 1-D Wasserstein-1 distance W1(a, b) = integral |F_a(x) - F_b(x)| dx,
  which for equal sample sizes is mean |sort(a) - sort(b)|;
* the cell-averaged run-to-run standard deviation of Eq. 12,
  sigma_bar(N) = (1/N_cells) sum_i sqrt( (1/(K-1)) sum_k (phi_i^k - phi_bar_i)^2 ).
"""
import numpy as np


def moments(a):
    a = np.asarray(a, dtype=np.float64)
    mu = a.mean()
    var = a.var()
    skew = np.mean((a - mu) ** 3) / var ** 1.5 if var > 0 else 0.0
    return mu, var, skew


def w1(a, b):
    a = np.sort(np.asarray(a, dtype=np.float64))
    b = np.sort(np.asarray(b, dtype=np.float64))
    if a.size == b.size:
        return float(np.mean(np.abs(a - b)))
    xs = np.sort(np.concatenate([a, b]))
    fa = np.searchsorted(a, xs[:-1], side="right") / a.size
    fb = np.searchsorted(b, xs[:-1], side="right") / b.size
    return float(np.sum(np.abs(fa - fb) * np.diff(xs)))


def sigma_bar(runs):
    """runs: [K, n_cells] flux estimates from K independent runs."""
    runs = np.asarray(runs, dtype=np.float64)
    K = runs.shape[0]
    mean = runs.mean(axis=0)
    sd = np.sqrt(np.sum((runs - mean) ** 2, axis=0) / (K - 1))
    return float(sd.mean())
