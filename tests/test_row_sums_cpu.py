"""The mathematics behind the closed-form row sums of the posterior (the device sums each grid
row of the cut ellipse in closed form): along a row the weights are a Gaussian sampled at the
integers, whose sum and mean over all integers follow from Poisson summation, and the FP64
oracle's brute-force grid sums must agree with that closed form where the box edges are far.
No GPU: NumPy and the oracle only."""
import numpy as np
import pytest

import oracle


def _direct(a, mu):
    j = np.arange(np.floor(mu) - 200, np.floor(mu) + 201)
    w = np.exp(-a * (j - mu) ** 2)
    return w.sum(), (w * j).sum() / w.sum()


def _poisson(a, mu):
    """Sum over all integers j of exp(-a (j - mu)^2) and its mean, first Poisson term kept."""
    q = np.exp(-np.pi ** 2 / a)
    den = 1.0 + 2.0 * q * np.cos(2 * np.pi * mu)
    return np.sqrt(np.pi / a) * den, mu - 2 * np.pi / a * q * np.sin(2 * np.pi * mu) / den


@pytest.mark.parametrize("a", [0.074, 0.5, 1.0, 1.386])
def test_full_line_sum_and_mean(a):
    """Up to -Cq = 2 (a = 2 ln 2 = 1.386, the narrowest rows the row kernel takes) the first
    Poisson term leaves the second, of order q^4 < 7e-13: relative in the sum, and (4 pi / a)
    q^4 < 5e-12 columns in the mean."""
    rng = np.random.default_rng(int(a * 1000))
    for mu in rng.uniform(-5, 130, 40):
        s, m = _direct(a, mu)
        ps, pm = _poisson(a, mu)
        assert abs(ps - s) <= 2e-12 * s
        assert abs(pm - m) <= 5e-12


def test_poisson_term_matters_for_narrow_rows():
    """Without the first term the mean of a row 0.6 columns wide is off by ~3e-3 columns, and
    with a row 2.6 columns wide (the 1080p grid) by less than 1e-50: the term is kept only
    where it is above 1e-14."""
    a = 1.386
    mu = 40.3
    _, m = _direct(a, mu)
    assert abs(m - mu) > 1e-3
    q_wide = np.exp(-np.pi ** 2 / 0.074)
    assert q_wide < 1e-50


def test_oracle_separable_posterior_mean_equals_closed_form():
    """With orthogonal mixing columns the posterior factorises, and along HbO2 the oracle's
    posterior mean over the grid nodes, far from the box edges, is the sampled Gaussian's mean
    in closed form (first Poisson term included): a pin of the oracle's discrete sums that a
    continuous-mean shortcut, a dropped node or a shifted index would fail."""
    sigma, a0, b1 = 0.02, 0.02, 0.01
    A = np.array([[a0, 0.0], [0.0, b1], [0.0, 0.0]])
    h0 = np.sqrt(2.0) * sigma / a0 * 1.2      # (a0 h0)^2 / (2 sigma^2) = 1.44: rows ~0.6 nodes wide
    n0 = 101
    grid = dict(n0=n0, n1=41, lo0=0.0, hi0=h0 * (n0 - 1), lo1=0.0, hi1=100.0, sigma_l=sigma)
    acoef = (a0 * h0) ** 2 / (2 * sigma ** 2)
    for mu_nodes in (50.0, 50.13, 50.37, 49.71):
        yb = A @ np.array([mu_nodes * h0, 50.0])
        got = oracle.posterior_mean(yb, A, grid)
        _, m = _poisson(acoef, mu_nodes)
        assert abs(got[0] / h0 - m) <= 1e-9, (mu_nodes, got[0] / h0, m)
        if abs(np.sin(2 * np.pi * mu_nodes)) > 0.3:
            assert abs(got[0] / h0 - mu_nodes) > 1e-4   # the continuous mean alone would not do
