"""The intensity-domain low pass (HB_LOWPASS_INTENSITY, Eq. 3-8 literally) on the GPU
against the FP64 oracle with the same reading: block means of -log of the mean intensity
within 3e-7 (one FP32 logarithm of a correctly rounded mean), THb and SO2 within the
usual tolerances; and the serving path with the flag against the single-frame path."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1706_07263_gb300 import Context, HbError, Server, binding, build, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
NTH = os.cpu_count() or 1
FLAG = binding.HB_LOWPASS_INTENSITY


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _grid(n0, n1, sigma=0.02):
    return dict(n0=n0, n1=n1, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=sigma)


@pytest.mark.parametrize("H,W,levels,fmt,g,seed", [
    (20, 30, 1, "u8", (64, 64), 1),
    (37, 53, 3, "u8", (128, 128), 2),
    (64, 200, 4, "u8", (128, 128), 3),
    (50, 70, 2, "f32", (64, 64), 4),
    (33, 65, 4, "f32", (100, 60), 5),
    (9, 11, 0, "u8", (32, 32), 6),
])
def test_pipeline_matches_oracle(H, W, levels, fmt, g, seed):
    mix = synth.make_mixing(seed)
    fr = synth.make_frame(seed, H, W, mix.A, 6, max(2.0, W / 20), max(4.0, W / 5), 0.02, fmt).rgb
    grid = _grid(*g)
    ref = oracle.estimate(fr, mix.A, grid, levels, 1e-3, intensity_lowpass=True, nthreads=NTH)
    frame = torch.from_numpy(fr).to(DEV)
    with Context(mix.A, grid, levels, 1e-3, W, H, fmt, FLAG) as ctx:
        hl, wl = ctx.lowpass_shape()
        thb = torch.empty((H, W), dtype=torch.float32, device=DEV)
        so2 = torch.empty_like(thb)
        yb = torch.empty((hl, wl, 3), dtype=torch.float64, device=DEV)
        cl = torch.empty((hl, wl, 2), dtype=torch.float32, device=DEV)
        ctx.estimate(frame, thb, so2)
        ctx.estimate_debug(frame, yb, cl, torch.empty_like(thb), torch.empty_like(thb))
        torch.cuda.synchronize()
    np.testing.assert_allclose(yb.cpu().numpy(), ref["ybar_ll"], rtol=0, atol=3e-7)
    t = thb.cpu().numpy().astype(np.float64)
    rel = np.abs(t - ref["thb"]) / np.maximum(np.abs(ref["thb"]), 1.0)
    assert rel.max() <= 1e-4, rel.max()
    mask = ref["thb"] >= 1.0
    assert np.abs(so2.cpu().numpy() - ref["so2"])[mask].max(initial=0.0) <= 1e-3


def test_flag_combinations_are_refused():
    A = synth.make_mixing(7).A
    with pytest.raises(HbError):
        Context(A, _grid(16, 16), 2, 1e-3, 32, 32, "u8", FLAG | binding.HB_LOWPASS_TIKHONOV)
    with pytest.raises(HbError):
        Context(A, _grid(16, 16), 5, 1e-3, 64, 64, "u8", FLAG)


def test_serving_with_the_flag_matches_single_frames():
    A = synth.make_mixing(8).A
    grid = _grid(64, 64)
    frames = [synth.make_frame(80 + k, 96, 128, A, 5, 4.0, 20.0, 0.01, "u8").rgb for k in range(4)]
    with Context(A, grid, 2, 1e-3, 128, 96, "u8", FLAG) as ctx:
        alone = []
        for fr in frames:
            thb = torch.empty((96, 128), dtype=torch.float32, device=DEV)
            ctx.estimate(torch.from_numpy(fr).to(DEV), thb, torch.empty_like(thb))
            torch.cuda.synchronize()
            alone.append(thb.cpu().numpy())
    got = {}
    with Server(A, grid, 1e-3, max_batch=4, batch_lowpass_pixels=50_000, flags=FLAG) as srv:
        sid = srv.open_stream(128, 96, 2, slots=4)
        srv.pause(True)
        for k, fr in enumerate(frames):
            assert srv.submit(sid, fr, k)
        srv.pause(False)
        import time
        t0 = time.time()
        while len(got) < 4 and time.time() - t0 < 20:
            for r in srv.poll(8, wait_us=2000):
                got[r["tag"]] = r["thb"].copy()
                srv.release(r["stream"], r["slot"])
    for k in range(4):
        rel = np.abs(got[k] - alone[k]) / np.maximum(np.abs(alone[k]), 1.0)
        assert rel.max() <= 1e-4
