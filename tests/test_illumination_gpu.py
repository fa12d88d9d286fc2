"""The constant (illumination) term of Eq. 8 on the GPU (HB_ILLUMINATION) against the
FP64 oracle with the same term, and its invariance to global illumination.

Tolerances are those of the plain path (THb within 1e-4 relative, SO2 within 1e-3) except
for where SO2 is compared: the FP32 error of a concentration is proportional to the gain of
the detail operator, ||M||_inf, which the constant column raises (up to about 8x for these
mixing matrices), so the THb floor below which SO2 = HbO2 / THb is not compared rises from
1 uM by the same factor."""
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
FLAG = binding.HB_ILLUMINATION


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _grid(n0, n1, sigma=0.02):
    return dict(n0=n0, n1=n1, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=sigma)


def _run(rgb, A, grid, levels, lam, flags=FLAG):
    H, W, _ = rgb.shape
    fmt = "u8" if rgb.dtype == np.uint8 else "f32"
    with Context(A, grid, levels, lam, W, H, fmt, flags) as ctx:
        thb = torch.empty((H, W), dtype=torch.float32, device=DEV)
        so2 = torch.empty_like(thb)
        ctx.estimate(torch.from_numpy(np.ascontiguousarray(rgb)).to(DEV), thb, so2)
        torch.cuda.synchronize()
        return thb.cpu().numpy().astype(np.float64), so2.cpu().numpy().astype(np.float64)


def _gain_ratio(A, lam):
    M, _ = oracle.tikhonov_operator(A, lam)
    Mi, _ = oracle.tikhonov_operator(A, lam, illumination=True)
    return max(1.0, np.abs(Mi).sum(1).max() / np.abs(M).sum(1).max())


def _check(got, ref, A, lam=1e-3):
    thb, so2 = got
    rel = np.abs(thb - ref["thb"]) / np.maximum(np.abs(ref["thb"]), 1.0)
    assert rel.max() <= 1e-4, rel.max()
    mask = ref["thb"] >= 1.0 * _gain_ratio(A, lam)
    assert np.abs(so2 - ref["so2"])[mask].max(initial=0.0) <= 1e-3


@pytest.mark.parametrize("H,W,levels,fmt,g,sigma,seed", [
    (40, 56, 2, "u8", (64, 64), 0.02, 1),
    (37, 53, 3, "f32", (128, 128), 0.02, 2),
    (64, 200, 4, "u8", (128, 128), 0.01, 3),
    (20, 30, 0, "f32", (32, 32), 0.03, 4),
    (96, 128, 1, "u8", (100, 60), 0.05, 5),
])
def test_pipeline_matches_oracle(H, W, levels, fmt, g, sigma, seed):
    mix = synth.make_mixing(seed)
    fr = synth.make_frame(seed, H, W, mix.A, 6, max(2.0, W / 20), max(4.0, W / 5), 0.01, fmt).rgb
    grid = _grid(*g, sigma)
    ref = oracle.estimate(fr, mix.A, grid, levels, 1e-3, illumination=True, nthreads=NTH)
    _check(_run(fr, mix.A, grid, levels, 1e-3), ref, mix.A)


def test_posterior_alone_matches_oracle():
    A = synth.make_mixing(8).A
    grid = _grid(128, 128)
    rng = np.random.default_rng(8)
    c = np.stack([rng.uniform(-20, 170, 400), rng.uniform(-20, 120, 400)], axis=1)
    yb = c @ A.T + rng.uniform(-0.8, 0.8, (400, 1)) + rng.normal(0, 0.01, (400, 3))
    ref = oracle.posterior_mean(yb, A, grid, nthreads=NTH, illumination=True)
    with Context(A, grid, 1, 1e-3, 8, 8, "u8", FLAG) as ctx:
        out = torch.empty((400, 2), dtype=torch.float32, device=DEV)
        ctx.posterior_mean(torch.from_numpy(yb).to(DEV), out)
        torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 2e-4 + 2e-6 * np.abs(ref))


def test_tikhonov_low_pass_with_the_term_matches_oracle():
    mix = synth.make_mixing(9)
    fr = synth.make_frame(9, 48, 64, mix.A, 5, 3.0, 12.0, 0.01, "u8").rgb
    grid = _grid(16, 16)
    ref = oracle.estimate(fr, mix.A, grid, 2, 1e-3, lowpass="tikhonov", illumination=True)
    _check(_run(fr, mix.A, grid, 2, 1e-3, FLAG | binding.HB_LOWPASS_TIKHONOV), ref, mix.A)


@pytest.mark.parametrize("s", [0.6, 1.25])
def test_global_illumination_leaves_the_estimate(s):
    mix = synth.make_mixing(10)
    fr = synth.make_frame(10, 120, 160, mix.A, 6, 8.0, 30.0, 0.0, "f32").rgb
    grid = _grid(128, 128)
    base = _run(fr, mix.A, grid, 3, 1e-3)
    lit = _run((fr * s).astype(np.float32), mix.A, grid, 3, 1e-3)
    rel = np.abs(lit[0] - base[0]) / np.maximum(np.abs(base[0]), 1.0)
    assert rel.max() <= 1e-4, rel.max()
    plain = _run(fr, mix.A, grid, 3, 1e-3, 0)
    plain_lit = _run((fr * s).astype(np.float32), mix.A, grid, 3, 1e-3, 0)
    assert np.abs(plain_lit[0] - plain[0]).max() > 1.0


def test_learned_low_pass_is_refused_with_the_term():
    A = synth.make_mixing(11).A
    with Context(A, _grid(32, 32), 2, 1e-3, 32, 32, "u8", FLAG) as ctx:
        ctx.mlp_init(1)
        with pytest.raises(HbError) as e:
            ctx.set_lowpass_mode(binding.HB_MODE_MLP, 1e-3, 16)
        assert e.value.status == 7                    # HB_ERR_STATE
