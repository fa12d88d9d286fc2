"""The least-squares low pass (the fit of the maximisation step of Section 2, Eq. 9 read as
the ordinary least-squares solution) in the FP64 oracle, pinned by NumPy's least squares,
the exact solve of the illumination system, noiseless patches and relighting invariance."""
import numpy as np
import pytest

import oracle
from paper_1706_07263_gb300 import synth

GRID = dict(n0=32, n1=32, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)


@pytest.mark.parametrize("fmt,levels,intensity", [("u8", 1, False), ("u8", 3, False), ("f32", 2, True),
                                                  ("u8", 3, True), ("f32", 0, False)])
def test_low_pass_is_the_least_squares_fit(fmt, levels, intensity):
    A = synth.make_mixing(6).A
    fr = synth.make_frame(7, 37, 45, A, 5, 2.0, 9.0, 0.02, fmt).rgb
    out = oracle.estimate(fr, A, GRID, levels, 1e-3, lowpass="ls", intensity_lowpass=intensity)
    yb = out["ybar_ll"].reshape(-1, 3)
    ref = np.linalg.lstsq(A, yb.T, rcond=None)[0].T
    got = out["conc_ll"].reshape(-1, 2) / (1 << levels)
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-9)


def test_with_the_illumination_term_the_fit_is_exact():
    A = synth.make_mixing(7).A
    fr = synth.make_frame(8, 24, 40, A, 4, 2.0, 6.0, 0.02, "f32").rgb
    out = oracle.estimate(fr, A, GRID, 2, 1e-3, lowpass="ls", illumination=True, intensity_lowpass=True)
    xi = np.concatenate([A, np.ones((3, 1))], axis=1)
    yb = out["ybar_ll"].reshape(-1, 3)
    ref = np.linalg.solve(xi, yb.T).T[:, :2]
    np.testing.assert_allclose(out["conc_ll"].reshape(-1, 2) / 4, ref, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("levels", [1, 3])
def test_noiseless_patch_is_recovered_exactly(levels):
    A = synth.make_mixing(8).A
    c = np.array([72.5, 31.25])
    I = np.exp(-(A @ c)).astype(np.float64)
    flat = np.broadcast_to(I, (16, 24, 3)).astype(np.float32)
    out = oracle.estimate(flat, A, GRID, levels, 1e-3, lowpass="ls")
    # float input is rounded to FP32 once: the recovered concentrations carry that rounding
    np.testing.assert_allclose(out["hbo2"], c[0], rtol=1e-5)
    np.testing.assert_allclose(out["hb"], c[1], rtol=1e-5)
    np.testing.assert_allclose(out["thb"], c.sum(), rtol=1e-5)


def test_pipeline_identity_with_the_least_squares_low_pass():
    """conc(p) = M y(p) + L ybar(B) - M ybar(B) for every pixel p of superblock B (the Haar
    transform is orthonormal and the detail operator M is linear), here with L the
    least-squares operator on the low pass."""
    A = synth.make_mixing(9).A
    fr = synth.make_frame(9, 32, 32, A, 4, 2.0, 7.0, 0.02, "f32").rgb
    levels, lam = 2, 1e-3
    out = oracle.estimate(fr, A, GRID, levels, lam, lowpass="ls")
    M, _ = oracle.tikhonov_operator(A, lam)
    L = np.linalg.pinv(A)
    y = oracle.log_atten(fr)
    yb = out["ybar_ll"]
    B = 1 << levels
    mb = np.repeat(np.repeat(yb, B, axis=0), B, axis=1)
    conc = y @ M.T + (mb @ L.T - mb @ M.T)
    np.testing.assert_allclose(out["hbo2"], conc[..., 0], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(out["hb"], conc[..., 1], rtol=1e-9, atol=1e-9)


def test_relighting_leaves_the_estimate_unchanged():
    """With the illumination column and the intensity low pass, scaling every intensity by
    one factor shifts -log by a constant in all channels, which the constant column absorbs;
    the directional bands are differences of logarithms and do not change either."""
    A = synth.make_mixing(10).A
    fr = synth.make_frame(10, 24, 32, A, 4, 2.0, 6.0, 0.01, "f32").rgb.astype(np.float64)
    a = oracle.estimate(fr.astype(np.float32), A, GRID, 2, 1e-3, lowpass="ls", illumination=True,
                        intensity_lowpass=True)
    b = oracle.estimate((0.5 * fr).astype(np.float32), A, GRID, 2, 1e-3, lowpass="ls", illumination=True,
                        intensity_lowpass=True)
    np.testing.assert_allclose(b["conc_ll"], a["conc_ll"], rtol=1e-6, atol=1e-6)


def test_the_tikhonov_low_pass_is_still_rejected_with_the_intensity_low_pass():
    A = synth.make_mixing(11).A
    fr = synth.make_frame(11, 16, 16, A, 2, 2.0, 4.0, 0.01, "u8").rgb
    with pytest.raises(ValueError):
        oracle.estimate(fr, A, GRID, 1, 1e-3, lowpass="tikhonov", intensity_lowpass=True)
