"""Pulse-rate recovery (Section 3.2) through the CUDA path: the THb trace of a synthetic
pulsing video matches the oracle's frame by frame, and both views of a stereo pair show
the injected rate."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1706_07263_gb300 import Context, build, pulse, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
NTH = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _trace(ctx, video, nframes, patch, every=0, oracle_args=None):
    H, W = video.H, video.W
    thb = torch.empty((H, W), dtype=torch.float32, device=DEV)
    so2 = torch.empty_like(thb)
    out = []
    for k in range(nframes):
        fr = video.frame(k)
        ctx.estimate(torch.from_numpy(fr).to(DEV), thb, so2)
        m = thb.cpu().numpy()
        if every and k % every == 0:
            ref = oracle.estimate(fr, *oracle_args, nthreads=NTH)["thb"]
            rel = np.abs(m - ref) / np.maximum(np.abs(ref), 1.0)
            assert rel.max() <= 1e-4, (k, rel.max())
        out.append(pulse.patch_mean(m, patch))
    return np.array(out)


def test_trace_matches_the_oracle_and_shows_the_pulse():
    A = synth.make_mixing(2).A
    grid = dict(n0=64, n1=64, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)
    v = synth.pulse_video(7, 64, 64, A, f_pulse=1.25)
    patch = (16, 48, 16, 48)
    with Context(A, grid, 2, 1e-3, 64, 64, "u8") as ctx:
        trace = _trace(ctx, v, 240, patch, every=30, oracle_args=(A, grid, 2, 1e-3))
    ref = np.array([pulse.patch_mean(oracle.estimate(v.frame(k), A, grid, 2, 1e-3, nthreads=NTH)["thb"], patch)
                    for k in range(240)])
    np.testing.assert_allclose(trace, ref, rtol=1e-4)
    assert 1.2 <= pulse.pulse_rate(trace, v.fps) <= 1.3


@pytest.mark.parametrize("f0,shifts", [(1.25, (0, 12)), (2.1, (0,))])
def test_stereo_views_show_the_injected_rate(f0, shifts):
    """360x480 frames, 3 levels, 128x128 grid, 10 s at 30 frames/s per view; the right view
    is the left one shifted by a 12 px disparity, its patch shifted with it."""
    A = synth.make_mixing(3).A
    grid = dict(n0=128, n1=128, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)
    with Context(A, grid, 3, 1e-3, 480, 360, "u8") as ctx:
        for sh in shifts:
            v = synth.pulse_video(11, 360, 480, A, f_pulse=f0, shift=sh)
            trace = _trace(ctx, v, 300, (120, 240, 180 + sh, 300 + sh))
            assert abs(pulse.pulse_rate(trace, v.fps) - f0) <= 0.05, (f0, sh)
