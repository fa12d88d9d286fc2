"""Pulse rate from a THb video (the analysis of Section 3.2).

The paper tracks a tissue patch in each view, averages THb over it frame by frame,
low-pass filters the trace, differentiates it, and finds the peak of the power spectrum
of that derivative by fitting a polynomial around it (1.2-1.3 Hz for its subject).  The
synthetic videos here are registered, so the patch is a fixed rectangle; everything else
follows those steps.  Host-side NumPy on a 1-D trace: the per-frame maps come from the
CUDA path (or, in the tests, from the oracle).
"""
from __future__ import annotations

import numpy as np


def patch_mean(thb_map: np.ndarray, patch) -> float:
    """Mean of a THb map over patch = (row0, row1, col0, col1), half-open."""
    r0, r1, c0, c1 = patch
    return float(np.mean(thb_map[r0:r1, c0:c1], dtype=np.float64))


def smooth(trace: np.ndarray, window: int) -> np.ndarray:
    """Centred moving average over an odd number of samples (edges: shrinking window)."""
    trace = np.asarray(trace, dtype=np.float64)
    if window <= 1:
        return trace.copy()
    half = window // 2
    c = np.concatenate([[0.0], np.cumsum(trace)])
    idx = np.arange(trace.size)
    lo = np.maximum(idx - half, 0)
    hi = np.minimum(idx + half + 1, trace.size)
    return (c[hi] - c[lo]) / (hi - lo)


def change_spectrum(trace: np.ndarray, fps: float, smooth_s: float = 0.2):
    """Power spectrum of the derivative of the smoothed trace (Hann window, mean removed).
    Returns (frequencies in Hz, power)."""
    win = max(1, int(round(smooth_s * fps)) | 1)
    d = np.gradient(smooth(trace, win)) * fps
    d = d - d.mean()
    w = np.hanning(d.size)
    p = np.abs(np.fft.rfft(d * w)) ** 2
    f = np.fft.rfftfreq(d.size, 1.0 / fps)
    return f, p


def peak_frequency(f: np.ndarray, p: np.ndarray, band=(0.5, 4.0)) -> float:
    """Frequency of the spectral peak inside band: the largest bin, refined by the vertex of
    the parabola through the log power of it and its two neighbours."""
    inside = np.nonzero((f >= band[0]) & (f <= band[1]))[0]
    k = int(inside[np.argmax(p[inside])])
    if k == 0 or k == f.size - 1:
        return float(f[k])
    y0, y1, y2 = np.log(p[k - 1:k + 2] + 1e-300)
    den = y0 - 2.0 * y1 + y2
    off = 0.5 * (y0 - y2) / den if den < 0 else 0.0
    return float(f[k] + np.clip(off, -0.5, 0.5) * (f[1] - f[0]))


def pulse_rate(trace: np.ndarray, fps: float, smooth_s: float = 0.2, band=(0.5, 4.0)) -> float:
    """Peak frequency (Hz) of the change in a THb trace."""
    f, p = change_spectrum(trace, fps, smooth_s)
    return peak_frequency(f, p, band)
