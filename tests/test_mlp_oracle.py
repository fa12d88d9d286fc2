"""Pins of the FP64 reference of the learned stand-in (oracle/mlp.py), on the CPU."""
import numpy as np
import pytest

from oracle import mlp
from paper_1706_07263_gb300 import synth

RNG = np.random.default_rng(7)


def _setup(n=64):
    A = synth.make_mixing(3).A
    grid = dict(n0=128, n1=128, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)
    nm = mlp.norm_for(A, grid)
    c = np.stack([RNG.uniform(-10, 160, n), RNG.uniform(-10, 110, n)], 1)
    ybar = c @ A.T + RNG.normal(0, 0.01, (n, 3))
    target = np.clip(c + RNG.normal(0, 1, c.shape), [0, 0], [150, 100])
    params = RNG.normal(0, 0.3, mlp.NPARAMS)
    return A, grid, nm, ybar, target, params


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.concatenate([RNG.normal(0, 1, 4000), RNG.normal(0, 1e3, 1000), [0.0, -0.0, 1.0, 1.00390625, 1.01171875]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), ref)


def test_gelu_closed_forms():
    assert mlp.gelu(0.0) == 0.0
    assert mlp.gelu_grad(0.0) == pytest.approx(0.5, abs=1e-15)
    assert mlp.gelu(1.0) == pytest.approx(0.8413447460685429, rel=1e-14)  # Phi(1)
    assert mlp.gelu(10.0) == pytest.approx(10.0, rel=1e-15)
    assert abs(mlp.gelu(-10.0)) < 1e-20
    z = np.linspace(-4, 4, 81)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), atol=1e-8)


def test_input_transform_maps_the_box_to_plus_minus_four():
    A, grid, nm, *_ = _setup()
    for c, want in (([75.0, 50.0], [0, 0]), ([0.0, 0.0], [-4, -4]), ([150.0, 100.0], [4, 4]), ([150.0, 0.0], [4, -4])):
        x = nm["T"] @ (A @ np.array(c)) + nm["t0"]
        np.testing.assert_allclose(x, [want[0], want[1], 0.0], atol=1e-9)
    off = np.cross(A[:, 0], A[:, 1])
    x = nm["T"] @ (A @ np.array([75.0, 50.0]) + 0.02 * off / np.linalg.norm(off)) + nm["t0"]
    np.testing.assert_allclose(x, [0, 0, 1.0], atol=1e-9)       # sigma_l = 0.02 off the range of A
    np.testing.assert_allclose(nm["Ap"] @ A, np.eye(2), atol=1e-10)
    # posterior standard deviation of an untruncated Gaussian likelihood with identity noise
    np.testing.assert_allclose(nm["osc"] ** 2, np.diag(0.02 ** 2 * np.linalg.inv(A.T @ A)), rtol=1e-12)


def test_gradient_matches_finite_differences():
    _, _, nm, ybar, target, params = _setup()
    _, g = mlp.loss_and_grad(params, nm, ybar, target, exact=True)
    idx = np.concatenate([RNG.choice(mlp.NPARAMS, 60, replace=False), np.arange(mlp.OFF_B3, mlp.NPARAMS)])
    h = 1e-6
    for i in idx:
        p1, p2 = params.copy(), params.copy()
        p1[i] += h
        p2[i] -= h
        num = (mlp.loss_and_grad(p1, nm, ybar, target, exact=True)[0] -
               mlp.loss_and_grad(p2, nm, ybar, target, exact=True)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, num, g[i])


def test_output_bias_only_network_has_closed_form_loss_and_gradient():
    _, _, nm, ybar, target, _ = _setup()
    params = np.zeros(mlp.NPARAMS)
    params[mlp.OFF_B3:] = [0.25, -0.5]          # exact in BF16
    loss, g = mlp.loss_and_grad(params, nm, ybar, target)
    t = (target - mlp.baseline(nm, ybar)) / nm["osc"]
    e = params[mlp.OFF_B3:] - t
    assert loss == pytest.approx(np.mean(e * e), rel=1e-14)
    np.testing.assert_allclose(g[mlp.OFF_B3:], 2 * e.sum(axis=0) / e.size, rtol=1e-13)
    np.testing.assert_array_equal(g[:mlp.OFF_W3], 0.0)   # zero weights: nothing flows back


def _edge_setup():
    A = synth.make_mixing(3).A
    grid = dict(n0=128, n1=128, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)
    return A, grid, mlp.norm_for(A, grid)


@pytest.mark.parametrize("c,axis,side", [([75.0, 2.0], 1, "lo"), ([75.0, -8.0], 1, "lo"), ([75.0, 97.0], 1, "hi"),
                                         ([146.0, 50.0], 0, "hi"), ([3.0, 50.0], 0, "lo"),
                                         ([-12.0, 50.0], 0, "lo")])
def test_baseline_is_the_mean_of_a_gaussian_cut_by_one_edge(c, axis, side):
    """Near one edge (the others many standard deviations away) the baseline is the mean of
    N(c_ls, S) truncated to that edge's side: the marginal along the edge's axis is a
    truncated normal (scipy.stats.truncnorm), and the other coordinate follows it through the
    regression S_01 / S_aa -- inside, at and outside the edge."""
    from scipy.stats import truncnorm
    A, grid, nm = _edge_setup()
    c = np.array(c)
    S = nm["S"]
    s = np.sqrt(S[axis, axis])
    lo, hi = (nm["lo"][axis], np.inf) if side == "lo" else (-np.inf, nm["hi"][axis])
    m = truncnorm.mean((lo - c[axis]) / s, (hi - c[axis]) / s, loc=c[axis], scale=s)
    want = c + S[:, axis] / S[axis, axis] * (m - c[axis])
    got = mlp.baseline(nm, (A @ c)[None])[0]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-8)


def test_baseline_is_the_least_squares_point_deep_inside():
    A, grid, nm = _edge_setup()
    c = np.array([[75.0, 50.0], [60.0, 45.0], [90.0, 55.0]])
    np.testing.assert_allclose(mlp.baseline(nm, c @ A.T), c, rtol=0, atol=1e-10)


def test_baseline_is_the_fine_grid_limit_of_the_posterior_near_one_edge():
    """The grid posterior (the oracle's, FP64) near one edge converges to the baseline as the
    grid is refined: halving the node spacing halves the difference (the edge node's weight
    is an O(h) term), and on the finer grid it is a small fraction of a standard deviation.
    A wrong sign or scale of an edge's shift would not converge."""
    import oracle
    A, _, nm = _edge_setup()
    for c in ([75.0, 2.0], [75.0, -8.0], [146.0, 50.0]):
        y = (A @ np.array(c))[None]
        diffs = []
        for n0, n1 in ((601, 401), (1201, 801)):
            grid = dict(n0=n0, n1=n1, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)
            diffs.append(np.abs(mlp.baseline(nm, y)[0] - oracle.posterior_mean(y, A, grid)[0]))
        ratio = diffs[0] / diffs[1]
        assert np.all((ratio > 1.8) & (ratio < 2.2)), (c, ratio)
        assert np.all(diffs[1] < 0.05 * nm["osc"]), (c, diffs[1])
