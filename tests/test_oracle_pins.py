"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test fixes one step of the method by something independent of the
oracle's code: the matrix the paper prints (Eq. 2), textbook basis functions
of the orthonormal Haar wavelet, a library solver (NumPy / SciPy), closed
forms (limits, truncated-normal means, least-squares recovery), invariants
(perfect reconstruction, Parseval, symmetry) and brute force on tiny inputs.
The last group plants mistakes in a copy of the oracle source and checks that
some pin catches each one.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1706_07263_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(1234)


def _grid(n0=5, n1=7, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma=0.02):
    return dict(n0=n0, n1=n1, lo0=lo0, hi0=hi0, lo1=lo1, hi1=hi1, sigma_l=sigma)


def _A(seed=0):
    return synth.make_mixing(seed).A


# --------------------------------------------------------------------------------------------
# log-attenuation (Eq. 8's -log; floor reading for zero / negative intensities)
# --------------------------------------------------------------------------------------------
def test_log_atten_u8_all_codes():
    codes = np.arange(256, dtype=np.uint8)
    frame = np.stack([codes, codes[::-1], codes], axis=-1).reshape(16, 16, 3)
    y = oracle.log_atten(frame)
    I = np.maximum(frame.astype(np.float64) / 255.0, 1.0 / 255.0)
    np.testing.assert_allclose(y, -np.log(I), rtol=0, atol=1e-15)


def test_log_atten_f32_floor_and_overexposure():
    frame = np.array([[[0.5, 1.0, 1.25], [0.0, -0.1, 1e-7]]], dtype=np.float32)
    y = oracle.log_atten(frame)
    I = np.maximum(frame.astype(np.float64), 1e-6)
    np.testing.assert_allclose(y, -np.log(I), rtol=1e-15)
    assert y[0, 0, 2] < 0  # intensities above 1 give negative attenuation, not clamped


def test_pad_edge_matches_numpy_pad():
    x = RNG.normal(size=(5, 7, 3))
    np.testing.assert_array_equal(oracle.pad_edge(x, 8, 8), np.pad(x, ((0, 3), (0, 1), (0, 0)), mode="edge"))


# --------------------------------------------------------------------------------------------
# Haar transform (Eq. 1-2, Eq. 4)
# --------------------------------------------------------------------------------------------
def test_one_level_reproduces_printed_matrix():
    """Transforming each unit window yields the columns of H as printed in Eq. 2."""
    H_paper = np.loadtxt(os.path.join(GOLDEN, "haar_matrix_eq2.txt"))
    got = np.zeros((4, 4))
    for i in range(4):
        win = np.zeros((2, 2, 1))
        win.flat[i] = 1.0   # window order (x,y), (x,y+1), (x+1,y), (x+1,y+1)
        bands = oracle.haar_level(win)
        got[i] = [b[0, 0, 0] for b in bands]
    # row i = unit vector e_i times H = row i of H
    np.testing.assert_array_equal(got, H_paper)


def _basis_coefficients(x, levels):
    """Textbook orthonormal 2D Haar basis: at level l the low-pass function is
    2^-l on a 2^l x 2^l block, and each directional function is +-2^-l with the
    sign pattern of its quadrants (top/bottom, diagonal, left/right).  The
    coefficients are plain inner products; no recursion is used."""
    h, w = x.shape[:2]
    ll_n = None
    det = []
    for l in range(1, levels + 1):
        b = 1 << l
        half = b // 2
        sgn_rows = np.where(np.arange(b) < half, 1.0, -1.0)
        sgn_cols = np.where(np.arange(b) < half, 1.0, -1.0)
        pats = [np.outer(sgn_rows, np.ones(b)),        # [1, 1, -1, -1]: rows differ
                np.outer(sgn_rows, sgn_cols),          # [1, -1, -1, 1]: diagonal
                np.outer(np.ones(b), sgn_cols)]        # [1, -1, 1, -1]: columns differ
        bands = [np.zeros((h // b, w // b, x.shape[2])) for _ in range(3)]
        for r in range(h // b):
            for c in range(w // b):
                blk = x[r * b:(r + 1) * b, c * b:(c + 1) * b]
                for k in range(3):
                    bands[k][r, c] = np.tensordot(pats[k], blk, axes=([0, 1], [0, 1])) / b
        det.append(bands)
        if l == levels:
            ll_n = x.reshape(h // b, b, w // b, b, x.shape[2]).sum(axis=(1, 3)) / b
    return ll_n, det


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_haar_forward_equals_basis_inner_products(levels):
    x = RNG.normal(size=(16, 24, 3))
    ll, det = oracle.haar_forward(x, levels)
    ll_ref, det_ref = _basis_coefficients(x, levels)
    np.testing.assert_allclose(ll, ll_ref, atol=1e-12)
    for l in range(levels):
        for k in range(3):
            np.testing.assert_allclose(det[l][k], det_ref[l][k], atol=1e-12)


@pytest.mark.parametrize("levels", [1, 2, 4])
def test_haar_perfect_reconstruction_and_parseval(levels):
    x = RNG.normal(size=(32, 48, 3))
    ll, det = oracle.haar_forward(x, levels)
    np.testing.assert_allclose(oracle.haar_inverse(ll, det), x, atol=1e-13)
    energy = np.sum(ll ** 2) + sum(np.sum(b ** 2) for d in det for b in d)
    np.testing.assert_allclose(energy, np.sum(x ** 2), rtol=1e-13)


def test_haar_constant_image():
    x = np.full((16, 16, 2), 0.7)
    ll, det = oracle.haar_forward(x, 3)
    np.testing.assert_allclose(ll, 0.7 * 8, rtol=1e-15)
    for d in det:
        for b in d:
            assert np.abs(b).max() < 1e-15


# --------------------------------------------------------------------------------------------
# Tikhonov operator (Eq. 5)
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("relative", [True, False])
def test_tikhonov_matches_linear_solve(relative):
    A = _A(3)
    lam = 1e-3 if relative else 1e-6
    M, gamma = oracle.tikhonov_operator(A, lam, relative)
    if relative:
        assert gamma == pytest.approx(lam * np.trace(A.T @ A) / 2, rel=1e-15)
    else:
        assert gamma == lam
    ys = RNG.normal(size=(3, 10))
    ref = np.linalg.solve(A.T @ A + gamma * np.eye(2), A.T @ ys)
    np.testing.assert_allclose(M @ ys, ref, rtol=1e-12, atol=1e-12)


def test_tikhonov_limits_to_pseudoinverse_and_recovers_noiseless():
    A = _A(1)
    M, _ = oracle.tikhonov_operator(A, 1e-14, True)
    np.testing.assert_allclose(M, np.linalg.pinv(A), rtol=1e-9)
    c = np.array([63.0, 21.0])
    np.testing.assert_allclose(M @ (A @ c), c, rtol=1e-9)


# --------------------------------------------------------------------------------------------
# Posterior mean on the grid (Section 2, Bayesian estimation on the low pass)
# --------------------------------------------------------------------------------------------
def test_posterior_brute_force_with_library_pdf():
    """5x7 grid, weights from scipy's multivariate normal pdf (an independent route)."""
    stats = pytest.importorskip("scipy.stats")
    A = _A(0)
    g = _grid(5, 7, sigma=0.05)
    c0 = np.linspace(0, 150, 5)
    c1 = np.linspace(0, 100, 7)
    for _ in range(5):
        yb = A @ np.array([RNG.uniform(0, 150), RNG.uniform(0, 100)]) + RNG.normal(0, 0.02, 3)
        P = np.array([[stats.multivariate_normal.pdf(yb, mean=A @ [a, b], cov=0.05 ** 2 * np.eye(3))
                       for b in c1] for a in c0])
        ref = np.array([(P.sum(axis=1) @ c0), (P.sum(axis=0) @ c1)]) / P.sum()
        np.testing.assert_allclose(oracle.posterior_mean(yb, A, g), ref, rtol=1e-10)


def test_posterior_wide_sigma_gives_grid_centroid():
    A = _A(2)
    yb = A @ np.array([10.0, 90.0])
    np.testing.assert_allclose(oracle.posterior_mean(yb, A, _grid(64, 64, sigma=1e6)), [75.0, 50.0], rtol=1e-8)


def test_posterior_narrow_sigma_gives_nearest_node():
    A = _A(4)
    n0, n1 = 17, 13
    nodes = np.array([[a, b] for a in np.linspace(0, 150, n0) for b in np.linspace(0, 100, n1)])
    for _ in range(10):
        yb = A @ np.array([RNG.uniform(0, 150), RNG.uniform(0, 100)])
        d2 = np.sum((yb[None, :] - nodes @ A.T) ** 2, axis=1)
        order = np.argsort(d2)
        if d2[order[1]] - d2[order[0]] < 1e-6:
            continue
        got = oracle.posterior_mean(yb, A, _grid(n0, n1, sigma=1e-4))
        np.testing.assert_allclose(got, nodes[order[0]], atol=1e-9)


def test_posterior_fine_grid_recovers_least_squares_point():
    """A Gaussian well inside the box, sampled on a fine lattice, has its
    discrete mean at the continuous mean, i.e. the least-squares solution."""
    A = _A(3)
    c_true = np.array([70.0, 45.0])
    yb = A @ c_true
    c_ls = np.linalg.lstsq(A, yb, rcond=None)[0]
    got = oracle.posterior_mean(yb, A, _grid(301, 201, sigma=0.003))
    np.testing.assert_allclose(got, c_ls, atol=1e-6)


def test_posterior_truncated_gaussian_at_box_edge():
    """Orthogonal columns make the posterior separable; along HbO2 it is a
    normal of sd sigma/|a| truncated at the box edge, whose mean SciPy knows."""
    stats = pytest.importorskip("scipy.stats")
    a, b, sigma = 0.02, 0.01, 0.02
    A = np.array([[a, 0.0], [0.0, b], [0.0, 0.0]])
    mu = 0.5                       # uM, just inside the lower edge
    sd = sigma / a                 # 1 uM
    yb = A @ np.array([mu, 50.0])
    h = 0.005
    g = _grid(2001, 11, lo0=0.0, hi0=10.0, sigma=sigma)
    got = oracle.posterior_mean(yb, A, g)
    ref = stats.truncnorm.mean((0.0 - mu) / sd, (10.0 - mu) / sd, loc=mu, scale=sd)
    assert abs(got[0] - ref) < h   # lattice sum vs integral: O(h) at the truncation edge


def test_posterior_axis_swap_symmetry():
    A = _A(1)
    yb = A @ np.array([40.0, 80.0]) + 0.01
    g = _grid(33, 21, 0.0, 150.0, 0.0, 100.0, sigma=0.03)
    g_sw = _grid(21, 33, 0.0, 100.0, 0.0, 150.0, sigma=0.03)
    got = oracle.posterior_mean(yb, A, g)
    got_sw = oracle.posterior_mean(yb, A[:, ::-1], g_sw)
    np.testing.assert_allclose(got, got_sw[::-1], rtol=1e-12)


# --------------------------------------------------------------------------------------------
# Whole estimator
# --------------------------------------------------------------------------------------------
def _frame(seed, H, W, fmt="f32", noise=0.005):
    mix = synth.make_mixing(seed)
    fr = synth.make_frame(seed, H, W, mix.A, 4, 3.0, 8.0, noise, fmt)
    return mix.A, fr


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_identity_all_tikhonov_equals_per_pixel_operator(levels):
    """With Tikhonov on every coefficient the pipeline is linear and H is
    orthonormal, so it must equal M applied to each pixel's log-attenuation."""
    A, fr = _frame(5, 24, 40)
    g = _grid(8, 8)
    out = oracle.estimate(fr.rgb, A, g, levels, 1e-3, lowpass="tikhonov")
    M, _ = oracle.tikhonov_operator(A, 1e-3, True)
    y = -np.log(np.maximum(fr.rgb.astype(np.float64), 1e-6))
    conc = y @ M.T
    np.testing.assert_allclose(out["hbo2"], conc[..., 0], rtol=1e-11, atol=1e-9)
    np.testing.assert_allclose(out["hb"], conc[..., 1], rtol=1e-11, atol=1e-9)


@pytest.mark.parametrize("levels", [1, 3])
def test_identity_bayes_low_pass_plus_per_pixel_details(levels):
    """Bayes on the low pass: conc(p) = M y(p) + (posterior(B) - M ybar(B)) on each 2^n block B."""
    A, fr = _frame(6, 32, 48)
    g = _grid(16, 12, sigma=0.05)
    out = oracle.estimate(fr.rgb, A, g, levels, 1e-3)
    M, _ = oracle.tikhonov_operator(A, 1e-3, True)
    y = -np.log(np.maximum(fr.rgb.astype(np.float64), 1e-6))
    b = 1 << levels
    ybar = y.reshape(32 // b, b, 48 // b, b, 3).mean(axis=(1, 3))
    post = oracle.posterior_mean(ybar, A, g)
    np.testing.assert_allclose(out["ybar_ll"], ybar, atol=1e-13)
    np.testing.assert_allclose(out["conc_ll"], post * b, rtol=1e-12)
    corr = np.repeat(np.repeat(post - ybar @ M.T, b, axis=0), b, axis=1)
    conc = y @ M.T + corr
    np.testing.assert_allclose(out["hbo2"], conc[..., 0], rtol=1e-11, atol=1e-9)
    np.testing.assert_allclose(out["hb"], conc[..., 1], rtol=1e-11, atol=1e-9)


def test_levels_zero_is_per_pixel_posterior():
    A, fr = _frame(7, 6, 5)
    g = _grid(9, 9, sigma=0.05)
    out = oracle.estimate(fr.rgb, A, g, 0, 1e-3)
    y = -np.log(np.maximum(fr.rgb.astype(np.float64), 1e-6))
    post = oracle.posterior_mean(y, A, g)
    np.testing.assert_allclose(out["hbo2"], post[..., 0], rtol=1e-13)
    np.testing.assert_allclose(out["hb"], post[..., 1], rtol=1e-13)


def test_ragged_size_equals_explicit_edge_padding():
    A, fr = _frame(8, 13, 22)
    g = _grid(10, 10, sigma=0.05)
    out = oracle.estimate(fr.rgb, A, g, 2, 1e-3)
    padded = np.pad(fr.rgb, ((0, 3), (0, 2), (0, 0)), mode="edge")
    outp = oracle.estimate(padded, A, g, 2, 1e-3)
    for k in ("hbo2", "hb", "thb", "so2"):
        np.testing.assert_allclose(out[k], outp[k][:13, :22], rtol=1e-14, atol=1e-13)


def test_noiseless_constant_patch_recovers_node():
    """A constant frame whose concentration lies on a grid node: zero details,
    a sharp posterior on that node, so the output is the node itself up to the
    float32 rounding of the input intensities (bounded through |M|)."""
    A = _A(1)
    n0, n1 = 31, 21
    c_star = np.array([np.linspace(0, 150, n0)[12], np.linspace(0, 100, n1)[7]])
    I = np.exp(-(A @ c_star)).astype(np.float32)
    frame = np.broadcast_to(I, (16, 16, 3)).copy()
    spacing = np.linalg.norm(A @ np.array([150 / 30, 0.0]))
    g = _grid(n0, n1, sigma=0.25 * spacing)
    out = oracle.estimate(frame, A, g, 2, 1e-3)
    M, _ = oracle.tikhonov_operator(A, 1e-3, True)
    bound = np.abs(M).sum() * 2.0 ** -24 * 3
    np.testing.assert_allclose(out["hbo2"], c_star[0], atol=bound + 1e-6)
    np.testing.assert_allclose(out["hb"], c_star[1], atol=bound + 1e-6)
    np.testing.assert_allclose(out["thb"], c_star.sum(), atol=2 * bound + 1e-6)
    np.testing.assert_allclose(out["so2"], c_star[0] / c_star.sum(), atol=1e-6)


def test_thb_so2_definitions():
    A, fr = _frame(9, 16, 16, noise=0.05)
    out = oracle.estimate(fr.rgb, A, _grid(8, 8, sigma=0.05), 1, 1e-3)
    np.testing.assert_array_equal(out["thb"], out["hbo2"] + out["hb"])
    pos = out["thb"] > 0
    np.testing.assert_array_equal(out["so2"][pos], out["hbo2"][pos] / out["thb"][pos])
    assert np.all(out["so2"][~pos] == 0.0)


# --------------------------------------------------------------------------------------------
# Planted mistakes: each mutation of the oracle source must make at least one pin fail.
# --------------------------------------------------------------------------------------------
MUTATIONS = {
    "haar_sign": ("{0.5, -0.5, -0.5, 0.5},", "{0.5, -0.5, 0.5, -0.5},"),
    "window_order": ("win[1] = in[((long)(2 * r) * w + 2 * c + 1) * C + ch];",
                     "win[1] = in[((long)(2 * r + 1) * w + 2 * c) * C + ch];"),
    "two_sigma_sq": ("double w = exp(-r2 / (2.0 * sigma * sigma) - Lmax);",
                     "double w = exp(-r2 / (sigma * sigma) - 2.0 * Lmax);"),
    "tikhonov_transpose": ("Gi[j][0] * A[c * 2 + 0] + Gi[j][1] * A[c * 2 + 1]",
                           "Gi[j][0] * A[c * 2 + 1] + Gi[j][1] * A[c * 2 + 0]"),
    "lowpass_scale": ("double scale = (double)blk; /* 2^n */", "double scale = (double)blk * 0.5;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    src = open(os.path.join(os.path.dirname(oracle.__file__), "hb_oracle.c")).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, name
    mdir = tmp_path / "mut"
    mdir.mkdir()
    (mdir / "hb_oracle.c").write_text(src.replace(old, new))
    so = str(mdir / "liboracle.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", so, str(mdir / "hb_oracle.c"),
                           "-lm", "-lpthread"])
    monkeypatch.setattr(oracle, "_LIB", so)
    monkeypatch.setattr(oracle, "_SRC", str(mdir / "hb_oracle.c"))
    monkeypatch.setattr(oracle, "_lib", None)
    pins = [test_one_level_reproduces_printed_matrix,
            lambda: test_haar_forward_equals_basis_inner_products(2),
            lambda: test_tikhonov_matches_linear_solve(True),
            test_posterior_truncated_gaussian_at_box_edge,
            lambda: test_identity_bayes_low_pass_plus_per_pixel_details(1)]
    failures = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failures += 1
    monkeypatch.setattr(oracle, "_lib", None)
    assert failures >= 1, f"mutation {name} slipped past every pin"
