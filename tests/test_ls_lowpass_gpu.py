"""The least-squares low pass (HB_LOWPASS_LS: the fit of Section 2's maximisation step, Eq. 9)
on the GPU against the FP64 oracle, alone and with the illumination term and the
intensity-domain low pass, through the device and the host entry points.

Tolerances are those of the plain path (THb within 1e-4 relative, SO2 within 1e-3); as with
the illumination term, the THb floor below which SO2 is not compared rises from 1 uM with
the gain of the operators (the FP32 error of a concentration is proportional to it)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1706_07263_gb300 import Context, HbError, binding, build, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
NTH = os.cpu_count() or 1
GRID = dict(n0=64, n1=64, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _flags(illum, intensity):
    f = binding.HB_LOWPASS_LS
    if illum:
        f |= binding.HB_ILLUMINATION
    if intensity:
        f |= binding.HB_LOWPASS_INTENSITY
    return f


def _gain(A, lam, illum):
    M, _ = oracle.tikhonov_operator(A, lam)
    Mi, _ = oracle.tikhonov_operator(A, lam, illumination=illum)
    L, _ = oracle.tikhonov_operator(A, 0.0, relative=False, illumination=illum)
    g = lambda X: np.abs(X).sum(1).max()
    return max(1.0, max(g(Mi), g(L)) / g(M))


def _run(rgb, A, levels, lam, flags, debug=False):
    H, W, _ = rgb.shape
    fmt = "u8" if rgb.dtype == np.uint8 else "f32"
    with Context(A, GRID, levels, lam, W, H, fmt, flags) as ctx:
        frame = torch.from_numpy(np.ascontiguousarray(rgb)).to(DEV)
        thb = torch.empty((H, W), dtype=torch.float32, device=DEV)
        so2 = torch.empty_like(thb)
        ctx.estimate(frame, thb, so2)
        out = {"thb": thb, "so2": so2}
        if debug:
            hl, wl = ctx.lowpass_shape()
            out["conc_ll"] = torch.empty((hl, wl, 2), dtype=torch.float32, device=DEV)
            ctx.estimate_debug(frame, None, out["conc_ll"], None, None)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}


def _check(got, ref, A, lam, illum):
    rel = np.abs(got["thb"] - ref["thb"]) / np.maximum(np.abs(ref["thb"]), 1.0)
    assert rel.max() <= 1e-4, rel.max()
    mask = ref["thb"] >= _gain(A, lam, illum)
    assert np.abs(got["so2"] - ref["so2"])[mask].max(initial=0.0) <= 1e-3


@pytest.mark.parametrize("H,W,levels,fmt,illum,intensity,seed", [
    (120, 200, 3, "u8", False, False, 1),
    (37, 53, 2, "f32", True, True, 2),
    (64, 96, 4, "u8", False, True, 3),
    (20, 30, 0, "f32", False, False, 4),
    (96, 160, 5, "u8", True, False, 5),
    (77, 91, 1, "f32", True, False, 6),
])
def test_pipeline_matches_oracle(H, W, levels, fmt, illum, intensity, seed):
    mix = synth.make_mixing(seed)
    fr = synth.make_frame(seed, H, W, mix.A, 6, max(2.0, W / 20), max(4.0, W / 5), 0.01, fmt).rgb
    lam = 1e-3
    got = _run(fr, mix.A, levels, lam, _flags(illum, intensity), debug=True)
    ref = oracle.estimate(fr, mix.A, GRID, levels, lam, lowpass="ls", illumination=illum,
                          intensity_lowpass=intensity, nthreads=NTH)
    _check(got, ref, mix.A, lam, illum)
    d = np.abs(got["conc_ll"] - ref["conc_ll"])
    assert np.all(d <= 1e-3 + 1e-5 * np.abs(ref["conc_ll"])), d.max()


def test_host_entry_points_match_the_device_call():
    mix = synth.make_mixing(7)
    H, W = 240, 320
    frames = [synth.make_frame(70 + k, H, W, mix.A, 6, 10.0, 60.0, 0.01, "u8").rgb for k in range(3)]
    flags = _flags(False, False)
    with Context(mix.A, GRID, 3, 1e-3, W, H, "u8", flags) as ctx:
        ref = []
        for rgb in frames:
            thb = torch.empty((H, W), dtype=torch.float32, device=DEV)
            so2 = torch.empty_like(thb)
            ctx.estimate(torch.from_numpy(rgb).to(DEV), thb, so2)
            ref.append(thb.cpu().numpy())
        hf = [torch.from_numpy(rgb).pin_memory() for rgb in frames]
        th = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in frames]
        sh = [torch.empty_like(t).pin_memory() for t in th]
        stream = torch.cuda.Stream()
        ctx.estimate_host(hf[0], th[0], sh[0], stream=stream)
        np.testing.assert_array_equal(th[0].numpy(), ref[0])
        for k in range(3):
            ctx.estimate_host_async(hf[k], th[k], sh[k], stream=stream)
        stream.synchronize()
        for k in range(3):
            np.testing.assert_array_equal(th[k].numpy(), ref[k])


def test_relighting_leaves_the_estimate_unchanged():
    """With the illumination column and the intensity low pass, halving every intensity
    leaves the estimate unchanged: the GPU result for the relit frame is within the parity
    tolerance of the oracle's result for the original frame (and so is the original's)."""
    mix = synth.make_mixing(8)
    fr = synth.make_frame(8, 64, 96, mix.A, 5, 4.0, 20.0, 0.01, "f32").rgb
    flags, lam = _flags(True, True), 1e-3
    ref = oracle.estimate(fr, mix.A, GRID, 2, lam, lowpass="ls", illumination=True, intensity_lowpass=True,
                          nthreads=NTH)
    _check(_run(fr, mix.A, 2, lam, flags), ref, mix.A, lam, True)
    _check(_run((0.5 * fr).astype(np.float32), mix.A, 2, lam, flags), ref, mix.A, lam, True)


def test_refused_with_the_tikhonov_low_pass_and_the_learned_low_pass():
    A = synth.make_mixing(9).A
    with pytest.raises(HbError):
        Context(A, GRID, 2, 1e-3, 16, 16, "u8", binding.HB_LOWPASS_LS | binding.HB_LOWPASS_TIKHONOV)
    with Context(A, GRID, 2, 1e-3, 16, 16, "u8", binding.HB_LOWPASS_LS) as ctx:
        ctx.mlp_init(1)
        with pytest.raises(HbError):
            ctx.set_lowpass_mode(binding.HB_MODE_MLP, 1e-3, 16)
