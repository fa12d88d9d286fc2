"""Pulse-rate analysis of a THb trace (Section 3.2) and its recovery from a synthetic
pulsing video by the FP64 oracle: the injected frequency is the closed-form answer."""
import os

import numpy as np
import pytest

import oracle
from paper_1706_07263_gb300 import pulse, synth

NTH = os.cpu_count() or 1
GRID = dict(n0=64, n1=64, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)


@pytest.mark.parametrize("f0", [0.9, 1.25, 2.1])
def test_peak_of_a_noisy_sinusoid_with_a_trend(f0):
    fps, n = 30.0, 300
    t = np.arange(n) / fps
    rng = np.random.default_rng(1)
    trace = 80.0 + 0.5 * t + 1.5 * np.sin(2 * np.pi * f0 * t + 0.3) + rng.normal(0, 0.5, n)
    assert abs(pulse.pulse_rate(trace, fps) - f0) < 0.03


def test_smooth_is_a_centred_moving_average():
    x = np.random.default_rng(2).normal(size=50)
    s = pulse.smooth(x, 5)
    np.testing.assert_allclose(s[2:-2], np.convolve(x, np.ones(5) / 5, mode="valid"), rtol=0, atol=1e-12)
    assert s[0] == pytest.approx(x[:3].mean()) and s[-1] == pytest.approx(x[-3:].mean())


def test_parabolic_refinement_hits_an_off_bin_frequency():
    fps, n = 30.0, 300                    # 0.1 Hz bins; 1.25 Hz falls between two
    t = np.arange(n) / fps
    f, p = pulse.change_spectrum(np.sin(2 * np.pi * 1.25 * t), fps, smooth_s=0.0)
    k = int(np.argmax(p))
    assert abs(f[k] - 1.25) == pytest.approx(0.05)
    assert abs(pulse.peak_frequency(f, p) - 1.25) < 0.01


def test_ground_truth_trace_of_the_video_pulses_at_the_injected_rate():
    A = synth.make_mixing(2).A
    v = synth.pulse_video(7, 48, 64, A, f_pulse=1.25)
    patch = (12, 36, 16, 48)
    gt = np.array([pulse.patch_mean(sum(v.fields(k)), patch) for k in range(300)])
    assert abs(pulse.pulse_rate(gt, v.fps) - 1.25) < 0.01


def test_oracle_recovers_the_pulse_rate_from_the_video():
    """64x64 u8 frames at 30 frames/s for 8 s, 2 Haar levels, 64x64 grid; the oracle's THb
    trace over the central patch peaks within the 1.2-1.3 Hz the injected 1.25 Hz allows."""
    A = synth.make_mixing(2).A
    v = synth.pulse_video(7, 64, 64, A, f_pulse=1.25)
    patch = (16, 48, 16, 48)
    trace = np.array([pulse.patch_mean(oracle.estimate(v.frame(k), A, GRID, 2, 1e-3, nthreads=NTH)["thb"], patch)
                      for k in range(240)])
    gt = np.array([pulse.patch_mean(sum(v.fields(k)), patch) for k in range(240)])
    assert 1.2 <= pulse.pulse_rate(trace, v.fps) <= 1.3
    assert np.corrcoef(trace, gt)[0, 1] > 0.8
