"""The estimators of e and C_V (tests/ising_stats.py) against what the
mathematics fixes: for a linear estimator the jackknife error over equal
bins is the standard error of the bin means, exactly; on independent normal
samples the pooled variance and its jackknife error match the known values."""
import numpy as np

from ising_stats import e_cv, jackknife_e_cv


def test_jackknife_of_the_mean_is_the_standard_error_of_bin_means():
    rng = np.random.default_rng(3)
    B, n, N, beta = 37, 500, 64, 0.4
    E = rng.normal(-100.0, 7.0, size=(B, n))
    (e, de), _ = jackknife_e_cv(E.sum(1), (E**2).sum(1), np.full(B, n), N, beta)
    bin_e = -E.mean(1) / N
    assert abs(e - bin_e.mean()) < 1e-12
    assert abs(de - bin_e.std(ddof=1) / np.sqrt(B)) < 1e-12 * abs(de) + 1e-15


def test_pooled_variance_of_independent_normals():
    rng = np.random.default_rng(4)
    B, n, N, beta, sd = 50, 4000, 16, 0.5, 3.0
    E = rng.normal(10.0, sd, size=(B, n))
    _, (cv, dcv) = jackknife_e_cv(E.sum(1), (E**2).sum(1), np.full(B, n), N, beta)
    want = beta * beta * sd * sd / N
    # var of the sample variance of m normals: 2 sd^4 / (m - 1)
    m = B * n
    dcv_want = beta * beta * sd * sd * np.sqrt(2.0 / (m - 1)) / N
    assert abs(cv - want) < 5 * dcv
    assert 0.7 < dcv / dcv_want < 1.3
    # the pooled estimate is the plain one over all samples
    _, cv_all = e_cv(E.sum(), (E**2).sum(), m, N, beta)
    assert abs(cv - cv_all) < 1e-12
