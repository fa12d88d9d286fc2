"""The intensity-domain low pass (Eq. 3-8 taken literally: the transform applied to the
intensities and -log taken of the low pass) in the FP64 oracle, pinned by a direct block
mean, Jensen's inequality and the cases where it must equal the log-domain reading."""
import numpy as np
import pytest

import oracle
from paper_1706_07263_gb300 import synth

GRID = dict(n0=32, n1=32, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)


def _block_mean_log(frame, levels):
    eps = 1.0 / 255.0 if frame.dtype == np.uint8 else 1e-6
    I = frame.astype(np.float64) / (255.0 if frame.dtype == np.uint8 else 1.0)
    I = np.maximum(I, eps)
    B = 1 << levels
    H, W, _ = I.shape
    Ip = np.pad(I, ((0, -H % B), (0, -W % B), (0, 0)), mode="edge")
    m = Ip.reshape(Ip.shape[0] // B, B, Ip.shape[1] // B, B, 3).mean(axis=(1, 3))
    return -np.log(m)


@pytest.mark.parametrize("fmt,levels,H,W", [("u8", 1, 20, 30), ("u8", 3, 37, 53), ("f32", 2, 16, 40),
                                             ("f32", 4, 50, 33)])
def test_low_pass_is_minus_log_of_the_block_mean(fmt, levels, H, W):
    A = synth.make_mixing(2).A
    fr = synth.make_frame(4, H, W, A, 4, 2.0, 8.0, 0.02, fmt).rgb
    out = oracle.estimate(fr, A, GRID, levels, 1e-3, intensity_lowpass=True)
    np.testing.assert_allclose(out["ybar_ll"], _block_mean_log(fr, levels), rtol=0, atol=1e-13)


def test_jensen_against_the_log_domain_low_pass():
    A = synth.make_mixing(3).A
    fr = synth.make_frame(3, 32, 48, A, 5, 2.0, 6.0, 0.02, "u8").rgb
    a = oracle.estimate(fr, A, GRID, 2, 1e-3)
    b = oracle.estimate(fr, A, GRID, 2, 1e-3, intensity_lowpass=True)
    assert np.all(b["ybar_ll"] <= a["ybar_ll"] + 1e-14)
    assert np.any(b["ybar_ll"] < a["ybar_ll"] - 1e-6)


def test_constant_blocks_and_no_levels_agree_with_the_log_domain():
    A = synth.make_mixing(4).A
    I = np.exp(-(A @ np.array([60.0, 40.0]))).astype(np.float32)
    flat = np.broadcast_to(I, (16, 24, 3)).copy()
    a = oracle.estimate(flat, A, GRID, 3, 1e-3)
    b = oracle.estimate(flat, A, GRID, 3, 1e-3, intensity_lowpass=True)
    np.testing.assert_allclose(b["thb"], a["thb"], rtol=1e-12)
    fr = synth.make_frame(5, 12, 14, A, 3, 2.0, 5.0, 0.01, "f32").rgb
    a0 = oracle.estimate(fr, A, GRID, 0, 1e-3)
    b0 = oracle.estimate(fr, A, GRID, 0, 1e-3, intensity_lowpass=True)
    np.testing.assert_allclose(b0["thb"], a0["thb"], rtol=1e-12)


def test_zero_codes_are_floored_before_the_mean():
    A = synth.make_mixing(5).A
    fr = np.zeros((8, 8, 3), dtype=np.uint8)
    fr[::2, ::2] = 200
    out = oracle.estimate(fr, A, GRID, 1, 1e-3, intensity_lowpass=True)
    np.testing.assert_allclose(out["ybar_ll"], -np.log((200 + 3 * 1) / (4 * 255.0)), atol=1e-13)
    assert np.all(np.isfinite(out["thb"]))
