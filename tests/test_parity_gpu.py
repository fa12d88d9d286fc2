"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded inputs.

Tolerances (the arithmetic behind them is in the design notes):
  * THb: max over pixels of |dTHb| / max(|THb_oracle|, 1 uM) <= 1e-4;
  * SO2: max |dSO2| <= 1e-3 over pixels with THb_oracle >= 1 uM;
  * block means ybar: |d| <= 2e-7 (float32 log table / logf against FP64 -log);
  * posterior means: |d| <= 2e-4 uM + 2e-6 * |c| (FP32 sums of up to 2^14 weights).
"""
import ctypes
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1706_07263_gb300 import Context, build, synth  # noqa: E402
from paper_1706_07263_gb300 import binding  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
NTH = os.cpu_count() or 1

THB_TOL = 1e-4
SO2_TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _grid(n0, n1, sigma=0.02, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0):
    return dict(n0=n0, n1=n1, lo0=lo0, hi0=hi0, lo1=lo1, hi1=hi1, sigma_l=sigma)


def run_gpu(frame_np, A, grid, levels, lam, flags=0, debug=False):
    fmt = "u8" if frame_np.dtype == np.uint8 else "f32"
    H, W, _ = frame_np.shape
    frame = torch.from_numpy(np.ascontiguousarray(frame_np)).to(DEV)
    with Context(A, grid, levels, lam, W, H, fmt, flags) as ctx:
        thb = torch.empty((H, W), dtype=torch.float32, device=DEV)
        so2 = torch.empty_like(thb)
        ctx.estimate(frame, thb, so2)
        out = {"thb": thb, "so2": so2}
        if debug:
            hl, wl = ctx.lowpass_shape()
            out["ybar_ll"] = torch.empty((hl, wl, 3), dtype=torch.float64, device=DEV)
            out["conc_ll"] = torch.empty((hl, wl, 2), dtype=torch.float32, device=DEV)
            out["hbo2"] = torch.empty_like(thb)
            out["hb"] = torch.empty_like(thb)
            ctx.estimate_debug(frame, out["ybar_ll"], out["conc_ll"], out["hbo2"], out["hb"])
        torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}


def compare(got, ref):
    thb_ref = ref["thb"]
    rel = np.abs(got["thb"] - thb_ref) / np.maximum(np.abs(thb_ref), 1.0)
    mask = thb_ref >= 1.0
    so2 = np.abs(got["so2"] - ref["so2"])[mask]
    return float(rel.max()), float(so2.max()) if so2.size else 0.0


def check(got, ref, what=""):
    thb_err, so2_err = compare(got, ref)
    assert thb_err <= THB_TOL, f"{what} THb rel err {thb_err:.3e}"
    assert so2_err <= SO2_TOL, f"{what} SO2 abs err {so2_err:.3e}"
    assert np.all(np.isfinite(got["thb"])) and np.all(np.isfinite(got["so2"]))
    return thb_err, so2_err


def small_frame(seed, H, W, fmt="f32", noise=0.005, nblobs=4, smin=3.0, smax=10.0):
    mix = synth.make_mixing(seed)
    fr = synth.make_frame(seed, H, W, mix.A, nblobs, smin, smax, noise, fmt)
    return mix.A, fr.rgb


# ------------------------------------------------------------------------------------------
# posterior step alone
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n0,n1,sigma", [(5, 7, 0.05), (64, 64, 0.02), (128, 128, 0.02), (128, 128, 0.005),
                                         (128, 128, 0.1), (33, 100, 0.02), (1, 17, 0.02), (1, 1, 0.02),
                                         (200, 300, 0.03), (16, 256, 0.01)])
def test_posterior_mean_matches_oracle(n0, n1, sigma):
    rng = np.random.default_rng(n0 * 1000 + n1)
    A = synth.make_mixing(n0 + n1).A
    grid = _grid(n0, n1, sigma)
    c = np.stack([rng.uniform(-20, 170, 300), rng.uniform(-20, 120, 300)], axis=1)
    yb = c @ A.T + rng.normal(0, 0.01, (300, 3))
    yb[:5] = [[0, 0, 0], [3, 3, 3], [-0.5, 0.2, 1.0], [2.5, 0.1, 0.1], [1e-3, 1e-3, 1e-3]]
    ref = oracle.posterior_mean(yb, A, grid, nthreads=NTH)
    with Context(A, grid, 1, 1e-3, 8, 8, "u8") as ctx:
        ybt = torch.from_numpy(yb).to(DEV)
        out = torch.empty((yb.shape[0], 2), dtype=torch.float32, device=DEV)
        ctx.posterior_mean(ybt, out)
        torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref)
    tol = 2e-4 + 2e-6 * np.abs(ref)
    assert np.all(err <= tol), f"max err {err.max():.3e} at {np.unravel_index(err.argmax(), err.shape)}"


def test_posterior_brute_force_tiny_image_4x4():
    """A 4x4 frame at one level: 4 low-pass pixels, a 5x7 grid, against the oracle."""
    A, rgb = small_frame(21, 4, 4, noise=0.02)
    grid = _grid(5, 7, 0.05)
    got = run_gpu(rgb, A, grid, 1, 1e-3, debug=True)
    ref = oracle.estimate(rgb, A, grid, 1, 1e-3)
    np.testing.assert_allclose(got["ybar_ll"], ref["ybar_ll"], atol=2e-7)
    np.testing.assert_allclose(got["conc_ll"], ref["conc_ll"], atol=2 * (2e-4 + 2e-6 * 300))
    check(got, ref, "4x4")


# ------------------------------------------------------------------------------------------
# whole pipeline
# ------------------------------------------------------------------------------------------
CASES = [
    # (H, W, levels, fmt, grid (n0, n1), sigma, seed)
    (8, 8, 1, "f32", (8, 8), 0.05, 1),
    (8, 8, 3, "u8", (16, 16), 0.02, 2),
    (13, 22, 2, "f32", (32, 24), 0.02, 3),
    (37, 53, 3, "u8", (64, 64), 0.02, 4),
    (64, 200, 4, "u8", (128, 128), 0.02, 5),
    (70, 130, 5, "f32", (40, 40), 0.03, 6),
    (128, 96, 6, "u8", (64, 32), 0.02, 7),
    (1, 1, 2, "u8", (16, 16), 0.02, 8),
    (1, 300, 3, "f32", (64, 64), 0.02, 9),
    (300, 1, 1, "u8", (64, 64), 0.02, 10),
    (20, 30, 0, "f32", (32, 32), 0.02, 11),
    (96, 2100, 2, "u8", (128, 128), 0.005, 12),
    (64, 64, 3, "u8", (128, 128), 0.1, 13),
    # enough low-pass pixels for the single-pass frame kernel, ragged in both directions, at
    # every level it takes (1 and 2 levels with a strip's rounds split over warps); its THb is
    # compared bit for bit with the three-kernel debug path below
    (130, 1030, 1, "u8", (64, 64), 0.02, 14),
    (250, 1500, 2, "f32", (96, 80), 0.02, 15),
    (1001, 777, 3, "u8", (128, 128), 0.02, 16),
]


@pytest.mark.parametrize("H,W,levels,fmt,g,sigma,seed", CASES)
def test_pipeline_matches_oracle(H, W, levels, fmt, g, sigma, seed):
    A, rgb = small_frame(seed, H, W, fmt, noise=0.01, nblobs=6, smin=max(2.0, W / 20), smax=max(4.0, W / 5))
    grid = _grid(*g, sigma)
    got = run_gpu(rgb, A, grid, levels, 1e-3, debug=True)
    ref = oracle.estimate(rgb, A, grid, levels, 1e-3, nthreads=NTH)
    np.testing.assert_allclose(got["ybar_ll"], ref["ybar_ll"], atol=2e-7)
    tol_c = 2 * (1 << levels) * (2e-4 + 2e-6 * np.abs(ref["conc_ll"] / (1 << levels)))
    assert np.all(np.abs(got["conc_ll"] - ref["conc_ll"]) <= tol_c)
    check(got, ref, f"{H}x{W} L{levels}")
    np.testing.assert_array_equal(got["thb"], got["hbo2"].astype(np.float32) + got["hb"].astype(np.float32))


def test_small_256_float_frame():
    """256x256 float frame, 1 level, 64x64 grid (the small configuration)."""
    wl = synth.SMALL_256
    mix, fr = synth.workload_inputs(wl)
    grid = synth.grid_spec(wl)
    got = run_gpu(fr.rgb, mix.A, grid, wl.levels, wl.lam)
    ref = oracle.estimate(fr.rgb, mix.A, grid, wl.levels, wl.lam, nthreads=NTH)
    thb_err, so2_err = check(got, ref, wl.name)
    print(f"{wl.name}: THb max rel err {thb_err:.3e}, SO2 max abs err {so2_err:.3e}")


def test_hd_1080_u8_frame():
    """1920x1080 8-bit frame, 3 levels, 128x128 grid, elementwise against the oracle."""
    wl = synth.HD_1080
    mix, fr = synth.workload_inputs(wl)
    grid = synth.grid_spec(wl)
    got = run_gpu(fr.rgb, mix.A, grid, wl.levels, wl.lam, debug=True)
    ref = oracle.estimate(fr.rgb, mix.A, grid, wl.levels, wl.lam, nthreads=NTH)
    np.testing.assert_allclose(got["ybar_ll"], ref["ybar_ll"], atol=2e-7)
    thb_err, so2_err = check(got, ref, wl.name)
    print(f"{wl.name}: THb max rel err {thb_err:.3e}, SO2 max abs err {so2_err:.3e}")


def _close_to_every_node(got_thb, got_so2, full_thb, full_so2):
    """Nodes carrying all but 2^-30 of the posterior mass, sums added in another order, and
    along each row the weights advanced by the FP32 ratio recurrence (the first ratio carries
    the rounding of its exponent, a few 1e-6 in log2, and each step one more rounding: a
    drift of at most about 1e-4 relative over the 23 steps of the longest row, which tilts a
    low-pass mean by a few 1e-5 uM): outputs agree to 2e-5 relative in THb and 5e-5 in SO2
    where THb >= 1 uM."""
    d = np.abs(got_thb - full_thb) / np.maximum(np.abs(full_thb), 1.0)
    assert d.max() <= 2e-5, d.max()
    mask = np.abs(full_thb) >= 1.0
    assert np.abs(got_so2 - full_so2)[mask].max(initial=0.0) <= 5e-5


def test_support_bounds_leave_the_result_unchanged():
    """The posterior enumerates, per pixel, only the grid rows and in each row only the
    column interval whose weights carry all but 2^-30 of the posterior mass, and sums each
    such row in closed form (or node by node with HB_NODE_SUMS); every output agrees with
    enumerating the whole grid (HB_FULL_GRID) to a few FP32 roundings, and the node and row
    counters show the work saved."""
    wl = synth.HD_1080
    mix, fr = synth.workload_inputs(wl)
    grid = synth.grid_spec(wl)
    frame = torch.from_numpy(fr.rgb).to(DEV)
    outs, nodes, rows = {}, {}, {}
    for flags in (0, binding.HB_NODE_SUMS, binding.HB_FULL_GRID):
        with Context(mix.A, grid, wl.levels, wl.lam, wl.W, wl.H, wl.fmt, flags) as ctx:
            thb = torch.empty((wl.H, wl.W), dtype=torch.float32, device=DEV)
            so2 = torch.empty_like(thb)
            ctx.timing_start(4)
            ctx.estimate(frame, thb, so2)
            nodes[flags], rows[flags] = ctx.timing_nodes(), ctx.timing_rows()
            ctx.timing_read()
            outs[flags] = (thb.cpu().numpy(), so2.cpu().numpy())
    hl, wl_ = (wl.H + 7) // 8, (wl.W + 7) // 8
    full = binding.HB_FULL_GRID
    assert nodes[full] == hl * wl_ * grid["n0"] * grid["n1"] and rows[full] == 0
    assert 0 < nodes[binding.HB_NODE_SUMS] < 0.1 * nodes[full] and rows[binding.HB_NODE_SUMS] == 0
    # closed form: every live row of every pixel (a few dozen per pixel), no node summed one by one
    assert nodes[0] == 0 and 10 * hl * wl_ < rows[0] < hl * wl_ * grid["n0"]
    for flags in (0, binding.HB_NODE_SUMS):
        _close_to_every_node(*outs[flags], *outs[full])


@pytest.mark.parametrize("n0,n1,sigma", [(128, 128, 0.02), (96, 100, 0.005), (64, 16, 0.1), (150, 64, 0.05)])
def test_column_intervals_keep_every_weighted_node(n0, n1, sigma):
    """40,000 pixels (two per warp): concentrations inside and around the grid's box, a few far
    outside the model, noise; the posterior over the rows' column intervals against every
    node (HB_FULL_GRID) and, on a sample, against the oracle."""
    rng = np.random.default_rng(11 * n0 + n1)
    A = synth.make_mixing(9).A
    grid = _grid(n0, n1, sigma)
    n = 40_000
    c = np.stack([rng.uniform(-40, 190, n), rng.uniform(-40, 140, n)], axis=1)
    c[:50] *= 40.0                                   # far outside the model
    yb = c @ A.T + rng.normal(0, 0.01, (n, 3))
    got = []
    for flags in (0, binding.HB_NODE_SUMS, binding.HB_FULL_GRID):
        with Context(A, grid, 1, 1e-3, 8, 8, "u8", flags) as ctx:
            out = torch.empty((n, 2), dtype=torch.float32, device=DEV)
            ctx.posterior_mean(torch.from_numpy(yb).to(DEV), out)
            torch.cuda.synchronize()
            got.append(out.cpu().numpy().astype(np.float64))
    for g in got[:2]:
        assert np.all(np.isfinite(g))
        d = np.abs(g - got[2])
        assert np.all(d <= 2e-5 + 1e-6 * np.abs(got[2])), d.max()
    pick = rng.choice(n, 1500, replace=False)
    pick[:20] = np.arange(20)
    ref = oracle.posterior_mean(yb[pick], A, grid, nthreads=NTH)
    assert np.all(np.abs(got[0][pick] - ref) <= 2e-4 + 2e-6 * np.abs(ref))


@pytest.mark.parametrize("mix_seed,hb_box,n0,n1", [(9, (0.0, 100.0), 128, 128), (9, (0.0, 12.0), 128, 24),
                                                    (9, (-30.0, 130.0), 128, 200), (4, (0.0, 100.0), 64, 64),
                                                    (17, (0.0, 100.0), 64, 64), (2, (0.0, 100.0), 128, 128)])
def test_closed_form_rows_against_node_sums(mix_seed, hb_box, n0, n1):
    """Rows summed in closed form (inside the grid: the full-line sum; cut off by the box on
    one side: the tabulated one-sided sum) beside rows summed node by node in the same warps
    (cut off on both sides: a posterior wider than the Hb box; a peak beyond the table: far
    outside the model): 40,000 pixels in and around the box against HB_NODE_SUMS, every node
    (HB_FULL_GRID) and, on a sample, the oracle.  Both counters must show work, so both kinds
    of row occur.  The 64x64 grids of mixings 4 and 17 have row Gaussians 0.73 and 0.61
    columns wide, where the first Poisson term moves a row's mean column by up to 2e-4 and
    3e-3 columns (mixing 2's 128x128 grid: 0.98 columns, 1e-7)."""
    rng = np.random.default_rng(n1 + 7 * mix_seed)
    A = synth.make_mixing(mix_seed).A
    grid = _grid(n0, n1, 0.02, lo1=hb_box[0], hi1=hb_box[1])
    n = 40_000
    span = hb_box[1] - hb_box[0]
    c = np.stack([rng.uniform(-40, 190, n), rng.uniform(hb_box[0] - 0.4 * span, hb_box[1] + 0.4 * span, n)], axis=1)
    c[:64] *= 40.0                                   # far outside the model
    yb = c @ A.T + rng.normal(0, 0.01, (n, 3))
    got, nodes, rows = [], [], []
    for flags in (0, binding.HB_NODE_SUMS, binding.HB_FULL_GRID):
        with Context(A, grid, 1, 1e-3, 8, 8, "u8", flags) as ctx:
            out = torch.empty((n, 2), dtype=torch.float32, device=DEV)
            ctx.timing_start(2)
            ctx.posterior_mean(torch.from_numpy(yb).to(DEV), out)
            nodes.append(ctx.timing_nodes())
            rows.append(ctx.timing_rows())
            ctx.timing_read()
            got.append(out.cpu().numpy().astype(np.float64))
    assert rows[0] > 0 and nodes[0] > 0, (rows[0], nodes[0])
    assert rows[1] == 0 and rows[2] == 0
    for g in got[:2]:
        assert np.all(np.isfinite(g))
        d = np.abs(g - got[2])
        assert np.all(d <= 2e-5 + 1e-6 * np.abs(got[2])), d.max()
    pick = rng.choice(n, 1500, replace=False)
    pick[:20] = np.arange(20)
    ref = oracle.posterior_mean(yb[pick], A, grid, nthreads=NTH)
    assert np.all(np.abs(got[0][pick] - ref) <= 2e-4 + 2e-6 * np.abs(ref))


@pytest.mark.parametrize("n1", [16, 60, 128])
def test_two_pixel_posterior_with_an_odd_pixel_count(n1):
    """404x604 at 2 levels: 101 x 151 = 15,251 low-pass pixels (odd, enough for two pixels per
    warp), so the last round has one empty half-warp; against the oracle, and against
    enumerating every node."""
    A, rgb = small_frame(45, 404, 604, "u8", noise=0.01, nblobs=8, smin=20.0, smax=120.0)
    grid = _grid(64, n1)
    ref = oracle.estimate(rgb, A, grid, 2, 1e-3, nthreads=NTH)
    got = run_gpu(rgb, A, grid, 2, 1e-3)
    check(got, ref, f"odd pixels n1={n1}")
    full = run_gpu(rgb, A, grid, 2, 1e-3, flags=binding.HB_FULL_GRID)
    _close_to_every_node(got["thb"], got["so2"], full["thb"], full["so2"])


@pytest.mark.parametrize("n0,n1,sigma", [(128, 128, 0.02), (200, 300, 0.005), (64, 16, 0.1), (128, 1, 0.02)])
def test_support_rows_posterior_alone_matches_full_grid(n0, n1, sigma):
    """Few pixels (a pixel split over several warps): the row bound changes only how rows
    are shared out, so both variants agree with the oracle and with each other."""
    rng = np.random.default_rng(7 * n0 + n1)
    A = synth.make_mixing(5).A
    grid = _grid(n0, n1, sigma)
    c = np.stack([rng.uniform(-20, 170, 200), rng.uniform(-20, 120, 200)], axis=1)
    yb = c @ A.T + rng.normal(0, 0.01, (200, 3))
    ref = oracle.posterior_mean(yb, A, grid, nthreads=NTH)
    got = []
    for flags in (0, binding.HB_FULL_GRID):
        with Context(A, grid, 1, 1e-3, 8, 8, "u8", flags) as ctx:
            out = torch.empty((yb.shape[0], 2), dtype=torch.float32, device=DEV)
            ctx.posterior_mean(torch.from_numpy(yb).to(DEV), out)
            torch.cuda.synchronize()
            got.append(out.cpu().numpy().astype(np.float64))
    tol = 2e-4 + 2e-6 * np.abs(ref)
    for g in got:
        assert np.all(np.abs(g - ref) <= tol)
    assert np.all(np.abs(got[0] - got[1]) <= tol)


@pytest.mark.parametrize("levels", [1, 3])
def test_all_tikhonov_mode_matches_oracle(levels):
    A, rgb = small_frame(31, 48, 64, "u8", noise=0.01)
    grid = _grid(16, 16)
    got = run_gpu(rgb, A, grid, levels, 1e-3, flags=binding.HB_LOWPASS_TIKHONOV)
    ref = oracle.estimate(rgb, A, grid, levels, 1e-3, lowpass="tikhonov")
    check(got, ref, "tikhonov")


def test_absolute_lambda_flag():
    A, rgb = small_frame(32, 32, 32, "f32")
    grid = _grid(32, 32)
    got = run_gpu(rgb, A, grid, 2, 2e-5, flags=binding.HB_LAMBDA_ABSOLUTE)
    ref = oracle.estimate(rgb, A, grid, 2, 2e-5, relative=False)
    check(got, ref, "absolute lambda")


def test_noiseless_constant_patch_recovers_node():
    A = synth.make_mixing(1).A
    n0, n1 = 31, 21
    c_star = np.array([np.linspace(0, 150, n0)[12], np.linspace(0, 100, n1)[7]])
    I = np.exp(-(A @ c_star)).astype(np.float32)
    frame = np.broadcast_to(I, (32, 48, 3)).copy()
    spacing = np.linalg.norm(A @ np.array([150 / 30, 0.0]))
    grid = _grid(n0, n1, 0.25 * spacing)
    got = run_gpu(frame, A, grid, 3, 1e-3, debug=True)
    np.testing.assert_allclose(got["hbo2"], c_star[0], atol=1e-3)
    np.testing.assert_allclose(got["hb"], c_star[1], atol=1e-3)


# ------------------------------------------------------------------------------------------
# boundary behaviour
# ------------------------------------------------------------------------------------------
def test_strided_frame_and_host_entry_match_plain_call():
    A, rgb = small_frame(41, 40, 72, "u8")
    grid = _grid(32, 32)
    base = run_gpu(rgb, A, grid, 2, 1e-3)
    padded = np.zeros((40, 72 * 3 + 37), dtype=np.uint8)
    padded[:, :72 * 3] = rgb.reshape(40, -1)
    frame = torch.from_numpy(padded).to(DEV)
    with Context(A, grid, 2, 1e-3, 72, 40, "u8") as ctx:
        thb = torch.empty((40, 72), dtype=torch.float32, device=DEV)
        so2 = torch.empty_like(thb)
        ctx.estimate(frame, thb, so2, row_stride_bytes=padded.strides[0])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(thb.cpu().numpy(), base["thb"].astype(np.float32))
        np.testing.assert_array_equal(so2.cpu().numpy(), base["so2"].astype(np.float32))
        th = np.empty((40, 72), np.float32)
        sh = np.empty((40, 72), np.float32)
        ctx.estimate_host(padded, th, sh)
        np.testing.assert_array_equal(th, base["thb"].astype(np.float32))
        np.testing.assert_array_equal(sh, base["so2"].astype(np.float32))


@pytest.mark.parametrize("case", ["hd_bayes", "tikhonov"])
def test_host_entry_in_bands_matches_the_device_call(case):
    """hb_estimate_host pipelines the frame in bands of superblock rows (copies overlapping the
    kernels); every pixel comes out bit-identical to hb_estimate on the same frame."""
    if case == "hd_bayes":
        wl = synth.HD_1080
        mix, fr = synth.workload_inputs(wl)
        A, rgb, grid, levels, flags = mix.A, fr.rgb, synth.grid_spec(wl), wl.levels, 0
    else:
        A, rgb = small_frame(44, 300, 500, "u8", noise=0.01, nblobs=6, smin=10.0, smax=60.0)
        grid, levels, flags = _grid(16, 16), 2, binding.HB_LOWPASS_TIKHONOV
    H, W, _ = rgb.shape
    with Context(A, grid, levels, 1e-3, W, H, "u8", flags) as ctx:
        thb = torch.empty((H, W), dtype=torch.float32, device=DEV)
        so2 = torch.empty_like(thb)
        ctx.estimate(torch.from_numpy(rgb).to(DEV), thb, so2)
        torch.cuda.synchronize()
        hf = torch.from_numpy(rgb).pin_memory()
        th = torch.empty((H, W), dtype=torch.float32).pin_memory()
        sh = torch.empty_like(th).pin_memory()
        for _ in range(2):                      # the default stream: direct calls
            ctx.estimate_host(hf, th, sh)
            np.testing.assert_array_equal(th.numpy(), thb.cpu().numpy())
            np.testing.assert_array_equal(sh.numpy(), so2.cpu().numpy())
        stream = torch.cuda.Stream()
        for k in range(4):                      # a stream: direct, captured, then replayed
            th.zero_()
            sh.zero_()
            n0 = ctx.launch_count()
            ctx.estimate_host(hf, th, sh, stream=stream)
            assert ctx.launch_count() > n0
            np.testing.assert_array_equal(th.numpy(), thb.cpu().numpy())
            np.testing.assert_array_equal(sh.numpy(), so2.cpu().numpy())
        th2 = torch.empty_like(th).pin_memory()  # other buffers: the graph is not reused for them
        ctx.estimate_host(hf, th2, sh, stream=stream)
        np.testing.assert_array_equal(th2.numpy(), thb.cpu().numpy())
        # the streamed (graph-replayed) frame against the FP64 oracle
        ctx.estimate_host(hf, th, sh, stream=stream)
        ref = oracle.estimate(rgb, A, grid, levels, 1e-3, nthreads=NTH,
                              lowpass="tikhonov" if flags & binding.HB_LOWPASS_TIKHONOV else "bayes")
        check({"thb": th.numpy().astype(np.float64), "so2": sh.numpy().astype(np.float64)}, ref, f"host {case}")


@pytest.mark.parametrize("case", ["hd_bayes", "small_tikhonov", "small_bayes", "f32_bayes"])
def test_asynchronous_host_calls_overlap_and_match(case):
    """hb_estimate_host_async: six different frames queued back to back on one stream (two
    staging sets in turn, so frames overlap), each into its own pinned outputs; after one
    synchronisation every frame equals hb_estimate on it bit for bit, as does a device call made
    while they are in flight and a synchronous call after them."""
    if case == "hd_bayes":
        wl = synth.HD_1080
        mix = synth.make_mixing(wl.seed)
        A, grid, levels, flags, H, W = mix.A, synth.grid_spec(wl), wl.levels, 0, wl.H, wl.W
        frames = [synth.make_frame(700 + k, H, W, A, wl.nblobs, wl.smin, wl.smax, wl.noise, "u8").rgb
                  for k in range(6)]
    elif case == "small_tikhonov":
        A = synth.make_mixing(44).A
        grid, levels, flags, H, W = _grid(16, 16), 2, binding.HB_LOWPASS_TIKHONOV, 300, 500
        frames = [synth.make_frame(800 + k, H, W, A, 6, 10.0, 60.0, 0.01, "u8").rgb for k in range(6)]
    elif case == "small_bayes":                   # 300 low-pass pixels: the one-pixel-per-unit kernel
        A = synth.make_mixing(45).A
        grid, levels, flags, H, W = _grid(64, 64), 3, 0, 120, 160
        frames = [synth.make_frame(850 + k, H, W, A, 4, 5.0, 30.0, 0.01, "u8").rgb for k in range(6)]
    else:                                         # float frames, 2 levels, a ragged size
        A = synth.make_mixing(46).A
        grid, levels, flags, H, W = _grid(128, 96), 2, 0, 602, 998
        frames = [synth.make_frame(870 + k, H, W, A, 8, 10.0, 80.0, 0.005, "f32").rgb for k in range(6)]
    fmt = "u8" if frames[0].dtype == np.uint8 else "f32"
    with Context(A, grid, levels, 1e-3, W, H, fmt, flags) as ctx:
        ref = []
        for rgb in frames:
            thb = torch.empty((H, W), dtype=torch.float32, device=DEV)
            so2 = torch.empty_like(thb)
            ctx.estimate(torch.from_numpy(rgb).to(DEV), thb, so2)
            ref.append((thb.cpu().numpy(), so2.cpu().numpy()))
        hf = [torch.from_numpy(rgb).pin_memory() for rgb in frames]
        th = [torch.full((H, W), -1.0, dtype=torch.float32).pin_memory() for _ in frames]
        sh = [torch.full((H, W), -1.0, dtype=torch.float32).pin_memory() for _ in frames]
        stream = torch.cuda.Stream()
        for k in range(len(frames)):
            ctx.estimate_host_async(hf[k], th[k], sh[k], stream=stream)
        # a device call while they are in flight: it waits for them (they share the context's
        # low-pass arrays), and neither disturbs the other
        thb = torch.empty((H, W), dtype=torch.float32, device=DEV)
        so2 = torch.empty_like(thb)
        ctx.estimate(torch.from_numpy(frames[2]).to(DEV), thb, so2)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(thb.cpu().numpy(), ref[2][0])
        stream.synchronize()
        for k in range(len(frames)):
            np.testing.assert_array_equal(th[k].numpy(), ref[k][0])
            np.testing.assert_array_equal(sh[k].numpy(), ref[k][1])
        # two of the streamed frames against the FP64 oracle
        for k in (1, 4):
            want = oracle.estimate(frames[k], A, grid, levels, 1e-3, nthreads=NTH,
                                   lowpass="tikhonov" if flags & binding.HB_LOWPASS_TIKHONOV else "bayes")
            check({"thb": th[k].numpy().astype(np.float64), "so2": sh[k].numpy().astype(np.float64)}, want,
                  f"async {case} frame {k}")
        th[0].zero_()
        ctx.estimate_host(hf[3], th[0], sh[0], stream=stream)
        np.testing.assert_array_equal(th[0].numpy(), ref[3][0])


def test_repeated_calls_are_deterministic_and_counted():
    A, rgb = small_frame(42, 64, 64, "u8")
    grid = _grid(64, 64)
    frame = torch.from_numpy(rgb).to(DEV)
    with Context(A, grid, 3, 1e-3, 64, 64, "u8") as ctx:
        outs = []
        ctx.timing_start(16)
        for _ in range(3):
            thb = torch.empty((64, 64), dtype=torch.float32, device=DEV)
            so2 = torch.empty_like(thb)
            ctx.estimate(frame, thb, so2)
            outs.append((thb, so2))
        t = ctx.timing_read()
        assert ctx.launch_count() == 9   # analysis, posterior, synthesis per frame
        assert t["analysis"][1] == 3 and t["lowpass"][1] == 3 and t["synthesis"][1] == 3
        assert all(t[k][0] > 0 for k in ("analysis", "lowpass", "synthesis"))
        for thb, so2 in outs[1:]:
            assert torch.equal(thb, outs[0][0]) and torch.equal(so2, outs[0][1])


def test_bad_stride_and_cpu_tensor_are_rejected():
    A, rgb = small_frame(43, 16, 16, "f32")
    with Context(A, _grid(8, 8), 1, 1e-3, 16, 16, "f32") as ctx:
        frame = torch.from_numpy(rgb).to(DEV)
        thb = torch.empty((16, 16), dtype=torch.float32, device=DEV)
        with pytest.raises(ValueError):   # the binding refuses it before the call
            ctx.estimate(frame, thb, thb.clone(), row_stride_bytes=16 * 3 * 4 - 4)
        # and the library itself, called directly through the C ABI
        so2 = thb.clone()
        rc = binding.load().hb_estimate(ctx.handle, ctypes.c_void_p(frame.data_ptr()), 16 * 3 * 4 - 4,
                                        ctypes.c_void_p(thb.data_ptr()), ctypes.c_void_p(so2.data_ptr()), None)
        assert rc == 1
        with pytest.raises(ValueError):
            ctx.estimate(torch.from_numpy(rgb), thb, thb.clone())


@pytest.mark.parametrize("mode", ["bayes", "ls", "mlp", "tikhonov"])
def test_frames_back_to_back_match_single_calls(mode):
    """Frames enqueued back to back on one stream -- each written into the same input buffer
    by a torch kernel just before the call, each frame's analysis launched as a programmatic
    dependent of the kernel before it -- give the THb/SO2 of one synchronised call per frame,
    bit for bit, in every low-pass mode."""
    mix = synth.make_mixing(3)
    H, W = 270, 480
    frames = [torch.from_numpy(synth.make_frame(300 + k, H, W, mix.A, 8, 5.0, 40.0, 0.01, "u8").rgb).to(DEV)
              for k in range(4)]
    flags = {"bayes": 0, "ls": binding.HB_LOWPASS_LS, "mlp": 0, "tikhonov": binding.HB_LOWPASS_TIKHONOV}[mode]
    with Context(mix.A, _grid(128, 128), 3, 1e-3, W, H, "u8", flags) as ctx:
        if mode == "mlp":
            ctx.mlp_init(1)
            ctx.set_lowpass_mode(binding.HB_MODE_MLP, float("inf"), 64)
        ref = []
        for f in frames:
            thb = torch.empty((H, W), dtype=torch.float32, device=DEV)
            so2 = torch.empty_like(thb)
            ctx.estimate(f, thb, so2)
            torch.cuda.synchronize()
            ref.append((thb, so2))
        buf = torch.empty_like(frames[0])
        outs = [(torch.empty((H, W), dtype=torch.float32, device=DEV),
                 torch.empty((H, W), dtype=torch.float32, device=DEV)) for _ in range(8)]
        for r in range(8):
            torch.add(frames[r % 4], 0, out=buf)   # a kernel writes the next frame in place
            ctx.estimate(buf, *outs[r])
        torch.cuda.synchronize()
        for r in range(8):
            assert torch.equal(outs[r][0], ref[r % 4][0]) and torch.equal(outs[r][1], ref[r % 4][1]), r


def test_streamed_drifting_stereo_frames_match_oracle():
    """The stereo stream of the bench (drifting 1080p scene, two views, 8-bit): frames copied
    host->device on a copy stream while the previous frame is estimated on a compute stream;
    the first left and the last right frame of the stream against the FP64 oracle."""
    wl = synth.HD_1080
    mix = synth.make_mixing(2)
    grid = synth.grid_spec(wl)
    n = 6
    video = synth.drift_video(2, wl.H, wl.W, mix.A, wl.nblobs, wl.smin, wl.smax, 3.0, wl.noise, "u8")
    ring = [torch.from_numpy(video.frame(i // 2, i & 1)).pin_memory() for i in range(2 * n)]
    copy_s, comp_s = torch.cuda.Stream(), torch.cuda.Stream()
    dbuf = [torch.empty((wl.H, wl.W, 3), dtype=torch.uint8, device=DEV) for _ in range(2)]
    outs = [(torch.empty((wl.H, wl.W), dtype=torch.float32, device=DEV),
             torch.empty((wl.H, wl.W), dtype=torch.float32, device=DEV)) for _ in range(2 * n)]
    copied = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]
    with Context(mix.A, grid, wl.levels, wl.lam, wl.W, wl.H, "u8") as ctx:
        for e in freed:
            e.record(comp_s)
        for i in range(2 * n):
            b = i & 1
            with torch.cuda.stream(copy_s):
                copy_s.wait_event(freed[b])
                dbuf[b].copy_(ring[i], non_blocking=True)
                copied[b].record(copy_s)
            with torch.cuda.stream(comp_s):
                comp_s.wait_event(copied[b])
                ctx.estimate(dbuf[b], *outs[i], stream=comp_s)
                freed[b].record(comp_s)
        torch.cuda.synchronize()
    for i in (0, 2 * n - 1):
        ref = oracle.estimate(ring[i].numpy(), mix.A, grid, wl.levels, wl.lam, nthreads=NTH)
        got = {"thb": outs[i][0].cpu().numpy().astype(np.float64), "so2": outs[i][1].cpu().numpy().astype(np.float64)}
        thb_err, so2_err = check(got, ref, f"streamed frame {i}")
        print(f"streamed frame {i}: THb max rel err {thb_err:.3e}, SO2 max abs err {so2_err:.3e}")
