"""The allocation-free posterior entry point (hb_posterior_mean_static).

Some callers cannot allocate device memory -- a real-time frame loop that must not
block on the allocator, or a plug-in whose host application owns every device
allocation -- so the library also offers the low-pass posterior step with its
working memory in one fixed array inside libhb.so.  This checks, through the C
ABI, that two calls in a row give the same posterior means as the context-based
hb_posterior_mean, within the tolerance of the other posterior parity tests, and
that sizes above the fixed maximum are refused.  The file is named so that pytest
collects it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1706_07263_gb300 import Context, HbError, binding, build, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _inputs(seed, npix, A):
    rng = np.random.default_rng(seed)
    c = np.stack([rng.uniform(-20, 170, npix), rng.uniform(-20, 120, npix)], axis=1)
    return c @ A.T + rng.normal(0, 0.01, (npix, 3))


def test_static_posterior_matches_context_path_twice():
    build.build()
    A = synth.make_mixing(17).A
    grid = dict(n0=128, n1=128, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)
    with Context(A, grid, 3, 1e-3, 64, 64, "u8") as ctx:
        for seed, npix in ((1, 32400), (2, 5000)):   # second call smaller: leftovers must not matter
            yb = torch.from_numpy(_inputs(seed, npix, A)).to(DEV)
            ref = torch.empty((npix, 2), dtype=torch.float32, device=DEV)
            got = torch.full((npix, 2), float("nan"), dtype=torch.float32, device=DEV)
            ctx.posterior_mean(yb, ref)
            binding.posterior_mean_static(A, grid, yb, got)
            torch.cuda.synchronize()
            r = ref.cpu().numpy().astype(np.float64)
            g = got.cpu().numpy().astype(np.float64)
            tol = 2e-4 + 2e-6 * np.abs(r)
            assert np.all(np.abs(g - r) <= tol), f"call npix={npix}: max diff {np.abs(g - r).max():.3e}"


@pytest.mark.parametrize("shape,npix", [((128, 128), 300), ((96, 200), 20000), ((96, 200), 250)])
def test_static_posterior_split_pixels_and_wide_grids_match_twice(shape, npix):
    """The kernels that use the array's partial-sum and arrival-counter regions: a few hundred
    pixels (fewer than the resident warps, so each pixel's rows are split into parts whose
    last arrival adds them up) and a grid wider than the two-pixel kernels take (one pixel
    per warp).  Two calls in a row, each against the context path."""
    build.build()
    A = synth.make_mixing(19).A
    grid = dict(n0=shape[0], n1=shape[1], lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)
    with Context(A, grid, 3, 1e-3, 64, 64, "u8") as ctx:
        for seed in (3, 4):
            yb = torch.from_numpy(_inputs(seed + npix, npix, A)).to(DEV)
            ref = torch.empty((npix, 2), dtype=torch.float32, device=DEV)
            got = torch.full((npix, 2), float("nan"), dtype=torch.float32, device=DEV)
            ctx.posterior_mean(yb, ref)
            binding.posterior_mean_static(A, grid, yb, got)
            torch.cuda.synchronize()
            r = ref.cpu().numpy().astype(np.float64)
            g = got.cpu().numpy().astype(np.float64)
            tol = 2e-4 + 2e-6 * np.abs(r)
            assert np.all(np.abs(g - r) <= tol), f"seed {seed}: max diff {np.abs(g - r).max():.3e}"


def test_static_posterior_refuses_oversize_and_launches_nothing():
    A = synth.make_mixing(18).A
    grid = dict(n0=16, n1=16, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)
    n = binding.STATIC_MAX_PIXELS + 1
    yb = torch.zeros((n, 3), dtype=torch.float64, device=DEV)
    out = torch.full((n, 2), -1.0, dtype=torch.float32, device=DEV)
    with pytest.raises(HbError) as e:
        binding.posterior_mean_static(A, grid, yb, out)
    assert e.value.status == 2
    torch.cuda.synchronize()
    assert bool((out == -1.0).all())
