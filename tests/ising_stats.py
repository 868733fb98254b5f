"""Estimators of the Ising application test's observables (Sec. 2, Table 1):
internal energy per spin e = -<E>/N and specific heat C_V = beta^2 (<E^2> -
<E>^2) / N, from the sums of E and E^2 over bins of measurements.

Both come from the pooled sums of the whole run, so C_V carries no bias from
short bins (averaging per-bin variances biases C_V low by O(tau / bin
length)); their errors are jackknife errors over the bins, which must be
long against the autocorrelation time or independent (separate chains)."""
import numpy as np


def e_cv(sum_e, sum_e2, n, n_sites, beta):
    mE = sum_e / n
    mE2 = sum_e2 / n
    return -mE / n_sites, beta * beta * (mE2 - mE * mE) / n_sites


def jackknife_e_cv(sum_e_bins, sum_e2_bins, n_bins, n_sites, beta):
    """((e, de), (cv, dcv)) from per-bin sums of E, E^2 and measurement counts."""
    sE = np.asarray(sum_e_bins, dtype=np.float64)
    sE2 = np.asarray(sum_e2_bins, dtype=np.float64)
    n = np.asarray(n_bins, dtype=np.float64)
    B = len(n)
    e_all, cv_all = e_cv(sE.sum(), sE2.sum(), n.sum(), n_sites, beta)
    e_j, cv_j = e_cv(sE.sum() - sE, sE2.sum() - sE2, n.sum() - n, n_sites, beta)
    de = np.sqrt((B - 1) / B * np.sum((e_j - e_j.mean()) ** 2))
    dcv = np.sqrt((B - 1) / B * np.sum((cv_j - cv_j.mean()) ** 2))
    return (e_all, de), (cv_all, dcv)


def binned_library_run(R, h, bins, sweep_bin):
    """Runs `bins` bins on a library Ising handle (sweep_bin(h) advances one
    bin with one measurement per sweep or round) and returns the per-bin
    sums of E, E^2 and the measurement counts, from the accumulators."""
    prev = R.ising_observables(h)
    sE, sE2, nb = [], [], []
    for _ in range(bins):
        sweep_bin(h)
        cur = R.ising_observables(h)
        nb.append(cur["n_meas"] - prev["n_meas"])
        sE.append(cur["acc"][0] - prev["acc"][0])
        sE2.append(cur["acc"][1] - prev["acc"][1])
        prev = cur
    return sE, sE2, nb
