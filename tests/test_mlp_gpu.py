"""The learned low-pass stand-in on the GPU: forward and gradient parity with the FP64
reference (oracle/mlp.py), training, and the per-frame fallback to the exact posterior."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import mlp  # noqa: E402
from paper_1706_07263_gb300 import Context, HbError, binding, build, surrogate, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
GRID = dict(n0=128, n1=128, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)


@pytest.fixture(scope="module")
def trained():
    """A network trained on pairs from seeded 512x512 frames (3 levels, 128x128 grid)."""
    build.build()
    wl = synth.Workload("train512", 512, 512, 3, (128, 128), 12, 10.0, 60.0, 0.01, "u8", 41)
    mix = synth.make_mixing(1)
    ctx = Context(mix.A, GRID, wl.levels, wl.lam, wl.W, wl.H, wl.fmt)
    frames = surrogate.workload_frames(wl, mix, 12, 500)
    ys, cs = surrogate.training_pairs(ctx, frames, DEV)
    phases = ((3e-3, 3000), (1e-3, 3000), (3e-4, 3000), (1e-4, 3000))
    losses = surrogate.train_phases(ctx, ys[:-4096], cs[:-4096], phases=phases, seed=3)
    yield dict(ctx=ctx, A=mix.A, ys=ys, cs=cs, losses=losses, wl=wl, mix=mix)
    ctx.close()


def _pairs(n=4096, seed=0):
    rng = np.random.default_rng(seed)
    A = synth.make_mixing(1).A
    c = np.stack([rng.uniform(-10, 160, n), rng.uniform(-10, 110, n)], 1)
    ybar = (c @ A.T + rng.normal(0, 0.01, (n, 3))).astype(np.float32)
    target = np.clip(c + rng.normal(0, 2, c.shape), [0, 0], [150, 100]).astype(np.float32)
    return A, ybar, target


# A BF16 rounding whose FP64 value lies within FLIP_REL (relative) of the midpoint between two
# BF16 numbers may go either way on the GPU, whose pre-rounding values are FP32; the FP64
# reference rounds each such value the other way on its own and adds up what that changes
# (oracle.mlp.forward_envelope / gradient_envelope).  The FP32 evaluation of z1, z2 and dz2
# (sums of at most 64 products) is good to a few 1e-7 of the terms' scale, far inside 2^-15.
FLIP_REL = 2.0 ** -15


def test_forward_matches_reference_element_by_element():
    """Every output of the network against the FP64 reference: within the reference's own
    rounding envelope, plus 1e-6 of the box (FP32 products, GELU to 1.5e-7, the baseline's
    erfcx) and 2^-21 of the sum of |A+| |ybar| (the FP32 least-squares point, whose terms
    cancel), sample by sample and axis by axis."""
    A, ybar, _ = _pairs(n=2048)
    with Context(A, GRID, 3, 1e-3, 64, 64, "u8") as ctx:
        ctx.mlp_init(11)
        params = ctx.mlp_get_params()
        out = torch.empty((ybar.shape[0], 2), dtype=torch.float32, device=DEV)
        ctx.mlp_forward(torch.from_numpy(ybar).to(DEV), out)
        torch.cuda.synchronize()
    nm = mlp.norm_for(A, GRID)
    ref, env = mlp.forward_envelope(params, nm, ybar.astype(np.float64), rel=FLIP_REL)
    d = np.abs(out.cpu().numpy() - ref)
    bound = env + 1e-6 * nm["ext"] + 2.0 ** -21 * (np.abs(ybar.astype(np.float64)) @ np.abs(nm["Ap"]).T)
    bad = d > bound
    assert not bad.any(), (f"{int(bad.sum())} of {d.size} outputs outside; worst excess "
                           f"{(d - bound).max():.3e} uM; samples needing the flip envelope: "
                           f"{int((env > 0).any(axis=1).sum())}")


def test_gradient_matches_reference_element_by_element():
    """Every entry of the loss gradient (4,546 parameters, 512 pairs) against the FP64
    reference: |g - ref| <= envelope + 2^-16 l1, where the envelope adds up what each
    ambiguous BF16 rounding of h1, h2 or dz2 changes when rounded the other way alone, and
    l1 (the entry's sum of absolute per-sample terms) scales the FP32 accumulation error (at
    most 128 terms per partial sum, 64 partials).  The norm comparison is kept as a summary."""
    A, ybar, target = _pairs(n=512, seed=1)
    with Context(A, GRID, 3, 1e-3, 64, 64, "u8") as ctx:
        ctx.mlp_init(12)
        params = ctx.mlp_get_params()
        g = torch.empty(binding.MLP_NPARAMS, dtype=torch.float32, device=DEV)
        loss = torch.empty(1, dtype=torch.float32, device=DEV)
        ctx.mlp_gradient(torch.from_numpy(ybar).to(DEV), torch.from_numpy(target).to(DEV), g, loss)
        torch.cuda.synchronize()
    nm = mlp.norm_for(A, GRID)
    ref_loss, ref_g, env, l1 = mlp.gradient_envelope(params, nm, ybar.astype(np.float64),
                                                     target.astype(np.float64), rel=FLIP_REL)
    got = g.cpu().numpy().astype(np.float64)
    assert float(loss.item()) == pytest.approx(ref_loss, rel=1e-4)
    d = np.abs(got - ref_g)
    bound = env + 2.0 ** -16 * l1
    bad = d > bound
    names = np.array(["W1"] * (mlp.OFF_B1 - mlp.OFF_W1) + ["b1"] * (mlp.OFF_W2 - mlp.OFF_B1) +
                     ["W2"] * (mlp.OFF_B2 - mlp.OFF_W2) + ["b2"] * (mlp.OFF_W3 - mlp.OFF_B2) +
                     ["W3"] * (mlp.OFF_B3 - mlp.OFF_W3) + ["b3"] * (mlp.NPARAMS - mlp.OFF_B3))
    assert not bad.any(), (f"{int(bad.sum())} entries outside ({sorted(set(names[bad]))}); worst excess "
                           f"{(d - bound).max():.3e} at {int(np.argmax(d - bound))}")
    # summary: the whole vector
    assert np.linalg.norm(got - ref_g) <= 1e-3 * np.linalg.norm(ref_g)


def test_training_reduces_loss_and_fits_held_out_pairs(trained):
    losses = trained["losses"]
    assert np.all(np.isfinite(losses))
    assert losses[-50:].mean() < 0.05 * losses[:10].mean()
    ctx, ys, cs = trained["ctx"], trained["ys"], trained["cs"]
    out = torch.empty((4096, 2), dtype=torch.float32, device=DEV)
    ctx.mlp_forward(ys[-4096:], out)
    torch.cuda.synchronize()
    err = ((out - cs[-4096:]).abs().cpu().numpy() / np.array([150.0, 100.0])).max(axis=1)
    assert err.mean() < 2e-3, err.mean()


def _frame(trained, seed):
    wl, mix = trained["wl"], trained["mix"]
    fr = synth.make_frame(seed, wl.H, wl.W, mix.A, wl.nblobs, wl.smin, wl.smax, wl.noise, wl.fmt)
    return torch.from_numpy(fr.rgb).to(DEV)


def _run(ctx, frame):
    thb = torch.empty(frame.shape[:2], dtype=torch.float32, device=DEV)
    so2 = torch.empty_like(thb)
    ctx.estimate(frame, thb, so2)
    torch.cuda.synchronize()
    return thb, so2


def test_forced_fallback_reproduces_the_exact_path(trained):
    ctx = trained["ctx"]
    frame = _frame(trained, 900)
    ctx.set_lowpass_mode(binding.HB_MODE_BAYES)
    thb0, so20 = _run(ctx, frame)
    good = ctx.mlp_get_params()
    bad = good.copy()
    bad[mlp.OFF_B3:] = 0.5                       # every estimate off by half the box
    ctx.mlp_set_params(bad)
    ctx.set_lowpass_mode(binding.HB_MODE_MLP, 1e-3, 256)
    f0, b0, _ = ctx.lowpass_stats()
    thb1, so21 = _run(ctx, frame)
    f1, b1, _ = ctx.lowpass_stats()
    assert (f1 - f0, b1 - b0) == (1, 1)
    assert torch.equal(thb0, thb1) and torch.equal(so20, so21)
    ctx.mlp_set_params(good)
    ctx.set_lowpass_mode(binding.HB_MODE_MLP, float("inf"), 256)   # never falls back
    thb2, _ = _run(ctx, frame)
    assert ctx.lowpass_stats()[1] == b1
    # the network's THb differs from the exact path by its low-pass error: a few 1e-3 relative
    # typically, more in the few blocks at the box edges where the network is least accurate
    rel = ((thb2 - thb0).abs() / thb0.abs().clamp(min=1.0)).flatten()
    assert rel.median().item() < 5e-3, rel.median().item()
    absq = torch.quantile((thb2 - thb0).abs().flatten(), 0.99).item()
    assert absq < 0.01 * 250.0, absq      # 99% of pixels within 1% of the THb range
    ctx.set_lowpass_mode(binding.HB_MODE_BAYES)


def _debug(ctx, frame):
    hl, wl = ctx.lowpass_shape()
    ybar = torch.empty((hl, wl, 3), dtype=torch.float64, device=DEV)
    conc = torch.empty((hl, wl, 2), dtype=torch.float32, device=DEV)
    ctx.estimate_debug(frame, ybar, conc, None, None)
    torch.cuda.synchronize()
    return ybar, conc


@pytest.mark.parametrize("nsample", [1, 5, 256, 3001])
def test_check_size_leaves_the_estimate_unchanged(trained, nsample):
    """The sampled check runs in extra CTAs of the inference launch (a few drawn pixels per
    CTA): however many pixels it draws, the network's estimate is the same bit for bit, and a
    corrupted network still falls back to the exact path."""
    ctx = trained["ctx"]
    frame = _frame(trained, 920)
    good = ctx.mlp_get_params()
    try:
        ctx.set_lowpass_mode(binding.HB_MODE_BAYES)
        exact = _run(ctx, frame)
        ctx.set_lowpass_mode(binding.HB_MODE_MLP, float("inf"), 256)
        ref = _run(ctx, frame)
        ctx.set_lowpass_mode(binding.HB_MODE_MLP, float("inf"), nsample)
        b0 = ctx.lowpass_stats()[1]
        got = _run(ctx, frame)
        assert ctx.lowpass_stats()[1] == b0
        assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])
        bad = good.copy()
        bad[mlp.OFF_B3:] = 0.5
        ctx.mlp_set_params(bad)
        ctx.set_lowpass_mode(binding.HB_MODE_MLP, 1e-3, nsample)
        got = _run(ctx, frame)
        assert ctx.lowpass_stats()[1] == b0 + 1
        assert torch.equal(got[0], exact[0]) and torch.equal(got[1], exact[1])
    finally:
        ctx.mlp_set_params(good)
        ctx.set_lowpass_mode(binding.HB_MODE_BAYES)


@pytest.mark.parametrize("shape", [None, (100, 150), (41, 67)])
def test_learned_low_pass_in_the_debug_output(trained, shape):
    """hb_estimate_debug in learned mode: the low-pass coefficients are 2^levels times the
    network's estimate for the frame's block means (hb_mlp_forward on the same inputs, bit for
    bit), or, after a failed check, those of the exact path.  Besides the training frame size
    (4,096 low-pass samples), two frames whose 247 and 54 samples end in a partial 8-sample
    tile."""
    wl = trained["wl"]
    if shape is None:
        ctx, frame = trained["ctx"], _frame(trained, 921)
    else:
        H, W = shape
        fr = synth.make_frame(922, H, W, trained["mix"].A, 4, 3.0, 20.0, 0.01, "u8")
        frame = torch.from_numpy(fr.rgb).to(DEV)
        ctx = Context(trained["mix"].A, GRID, wl.levels, wl.lam, W, H, "u8")
        ctx.mlp_set_params(trained["ctx"].mlp_get_params())
    good = ctx.mlp_get_params()
    try:
        ctx.set_lowpass_mode(binding.HB_MODE_BAYES)
        _, exact = _debug(ctx, frame)
        ctx.set_lowpass_mode(binding.HB_MODE_MLP, float("inf"), 256)
        ybar, conc = _debug(ctx, frame)
        out = torch.empty((ybar.shape[0] * ybar.shape[1], 2), dtype=torch.float32, device=DEV)
        ctx.mlp_forward(ybar.reshape(-1, 3).float().contiguous(), out)
        torch.cuda.synchronize()
        assert torch.equal(conc.reshape(-1, 2), out * float(1 << wl.levels))
        bad = good.copy()
        bad[mlp.OFF_B3:] = 0.5
        ctx.mlp_set_params(bad)
        ctx.set_lowpass_mode(binding.HB_MODE_MLP, 1e-3, 256)
        _, conc = _debug(ctx, frame)
        assert torch.equal(conc, exact)
    finally:
        ctx.mlp_set_params(good)
        ctx.set_lowpass_mode(binding.HB_MODE_BAYES)
        if shape is not None:
            ctx.close()


def test_certified_learned_mode_stays_within_tolerance(trained):
    """The learned mode as it is meant to run: the network certified at half the tolerance
    (hb_mlp_certify), the fallback gated on the largest of 256 sampled errors.  On held-out
    frames, every low-pass pixel of every frame that did not fall back is within tol of the
    exact path (error relative to the box extents), so THb is within tol (ext0 + ext1) uM of
    it at every pixel; the pixels the route sent to the exact posterior are the exact path's,
    bit for bit; and a change of the parameters ends the certification."""
    ctx, wl = trained["ctx"], trained["wl"]
    tol = 1e-3
    ext = np.array([GRID["hi0"] - GRID["lo0"], GRID["hi1"] - GRID["lo1"]])
    good = ctx.mlp_get_params()
    trusted = ctx.mlp_certify(0.5 * tol)
    assert 0.0 < trusted <= 1.0
    kept = 0
    try:
        for seed in range(940, 946):
            frame = _frame(trained, seed)
            ctx.set_lowpass_mode(binding.HB_MODE_BAYES)
            t_exact, _ = _run(ctx, frame)
            _, c_exact = _debug(ctx, frame)
            ctx.set_lowpass_mode(binding.HB_MODE_MLP, tol, 256)
            f0, b0, r0 = ctx.lowpass_stats()
            t_mlp, _ = _run(ctx, frame)
            f1, b1, r1 = ctx.lowpass_stats()
            _, c_mlp = _debug(ctx, frame)
            assert f1 - f0 == 1
            if b1 > b0:                                   # fell back: the exact path itself
                assert torch.equal(t_mlp, t_exact)
                continue
            kept += 1
            err = ((c_mlp - c_exact).abs().cpu().numpy() / (ext * (1 << wl.levels))).max()
            assert err <= tol, (seed, err)
            dthb = (t_mlp - t_exact).abs().max().item()
            assert dthb <= tol * ext.sum() + 1e-3, (seed, dthb)
            same = bool((c_mlp == c_exact).all(dim=-1).sum().item() >= r1 - r0)
            assert same, (seed, r1 - r0)
        assert kept >= 1, "every frame fell back"
        # a parameter change ends the certification: no pixel is routed any more
        ctx.mlp_set_params(good)
        _, _, r2 = ctx.lowpass_stats()
        _run(ctx, _frame(trained, 950))
        assert ctx.lowpass_stats()[2] == r2
    finally:
        ctx.mlp_set_params(good)
        ctx.set_lowpass_mode(binding.HB_MODE_BAYES)


def test_mean_gate_mode_still_falls_back_on_a_broken_network(trained):
    """HB_MODE_MLP_MEAN_GATE (the mean of the sampled errors against tol, kept for
    comparison) falls back on a corrupted network like the default gate."""
    ctx = trained["ctx"]
    frame = _frame(trained, 960)
    good = ctx.mlp_get_params()
    try:
        ctx.set_lowpass_mode(binding.HB_MODE_BAYES)
        exact = _run(ctx, frame)
        bad = good.copy()
        bad[mlp.OFF_B3:] = 0.5
        ctx.mlp_set_params(bad)
        ctx.set_lowpass_mode(binding.HB_MODE_MLP_MEAN_GATE, 1e-3, 256)
        b0 = ctx.lowpass_stats()[1]
        got = _run(ctx, frame)
        assert ctx.lowpass_stats()[1] == b0 + 1
        assert torch.equal(got[0], exact[0]) and torch.equal(got[1], exact[1])
    finally:
        ctx.mlp_set_params(good)
        ctx.set_lowpass_mode(binding.HB_MODE_BAYES)


def _fnv1a(data: bytes) -> int:
    h = 2166136261
    for b in data:
        h = ((h ^ b) * 16777619) & 0xFFFFFFFF
    return h


def test_network_file_round_trip(trained, tmp_path):
    """hb_mlp_save / hb_mlp_load: the file has the documented layout (header, the model, the
    parameters, an FNV-1a hash); loaded into a new context of the same model it gives the same
    parameters and the same learned-mode frame, bit for bit.  A file cut short, one byte too
    long, with one byte altered or with another header is refused with HB_ERR_IO and leaves
    the network as it was; a network of another model (sigma_l) is refused with HB_ERR_STATE."""
    ctx, wl, mix = trained["ctx"], trained["wl"], trained["mix"]
    path = tmp_path / "net.hbmlp"
    ctx.mlp_save(path)
    raw = path.read_bytes()
    n = binding.MLP_NPARAMS
    assert len(raw) == 16 + 88 + 4 * n + 4 and raw[:8] == b"HBMLPv1\n"
    assert int.from_bytes(raw[8:12], "little") == n and int.from_bytes(raw[12:16], "little") == 0
    model = np.frombuffer(raw[16:104], dtype="<f8")
    expect = list(np.asarray(mix.A, dtype=np.float64).reshape(-1)) + [GRID["lo0"], GRID["hi0"], GRID["lo1"],
                                                                      GRID["hi1"], GRID["sigma_l"]]
    np.testing.assert_array_equal(model, np.array(expect))
    np.testing.assert_array_equal(np.frombuffer(raw[104:104 + 4 * n], dtype="<f4"), ctx.mlp_get_params())
    assert int.from_bytes(raw[-4:], "little") == _fnv1a(raw[:-4])
    frame = _frame(trained, 930)
    with Context(mix.A, GRID, wl.levels, wl.lam, wl.W, wl.H, wl.fmt) as other:
        with pytest.raises(HbError) as e:
            other.mlp_save(tmp_path / "none.hbmlp")      # no network yet
        assert e.value.status == 7
        other.mlp_load(path)
        np.testing.assert_array_equal(other.mlp_get_params(), ctx.mlp_get_params())
        try:
            for c in (ctx, other):
                c.set_lowpass_mode(binding.HB_MODE_MLP, float("inf"), 256)
            a, b = _run(ctx, frame), _run(other, frame)
        finally:
            ctx.set_lowpass_mode(binding.HB_MODE_BAYES)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
        before = other.mlp_get_params()
        flipped = bytearray(raw)
        flipped[200] ^= 0x10
        bad = {"short": raw[:-1], "long": raw + b"\0", "flipped": bytes(flipped), "header": b"X" + raw[1:]}
        for name, data in bad.items():
            q = tmp_path / f"{name}.hbmlp"
            q.write_bytes(data)
            with pytest.raises(HbError) as e:
                other.mlp_load(q)
            assert e.value.status == 8, name
        with pytest.raises(HbError) as e:
            other.mlp_load(tmp_path / "missing.hbmlp")
        assert e.value.status == 8
        np.testing.assert_array_equal(other.mlp_get_params(), before)
    with Context(mix.A, dict(GRID, sigma_l=0.03), wl.levels, wl.lam, wl.W, wl.H, wl.fmt) as third:
        with pytest.raises(HbError) as e:
            third.mlp_load(path)
        assert e.value.status == 7


def test_asynchronous_host_calls_in_learned_mode(trained):
    """hb_estimate_host_async with the learned low pass (one whole-frame band per call, frames
    overlapping): with a working network each frame equals the device call bit for bit; with a
    corrupted one every frame falls back and equals the exact path."""
    ctx, wl = trained["ctx"], trained["wl"]
    frames = [_frame(trained, 910 + k) for k in range(3)]
    ctx.set_lowpass_mode(binding.HB_MODE_BAYES)
    exact = [_run(ctx, f) for f in frames]
    good = ctx.mlp_get_params()
    hf = [f.cpu().pin_memory() for f in frames]
    th = [torch.empty((wl.H, wl.W), dtype=torch.float32).pin_memory() for _ in frames]
    sh = [torch.empty_like(t).pin_memory() for t in th]
    stream = torch.cuda.Stream()
    try:
        ctx.set_lowpass_mode(binding.HB_MODE_MLP, float("inf"), 256)
        device = [_run(ctx, f) for f in frames]
        for k in range(3):
            ctx.estimate_host_async(hf[k], th[k], sh[k], stream=stream)
        stream.synchronize()
        for k in range(3):
            assert torch.equal(th[k], device[k][0].cpu()) and torch.equal(sh[k], device[k][1].cpu())
        bad = good.copy()
        bad[mlp.OFF_B3:] = 0.5
        ctx.mlp_set_params(bad)
        ctx.set_lowpass_mode(binding.HB_MODE_MLP, 1e-3, 256)
        b0 = ctx.lowpass_stats()[1]
        for k in range(3):
            ctx.estimate_host_async(hf[k], th[k], sh[k], stream=stream)
        stream.synchronize()
        assert ctx.lowpass_stats()[1] - b0 == 3
        for k in range(3):
            assert torch.equal(th[k], exact[k][0].cpu()) and torch.equal(sh[k], exact[k][1].cpu())
    finally:
        ctx.mlp_set_params(good)
        ctx.set_lowpass_mode(binding.HB_MODE_BAYES)


def test_mlp_mode_is_faster_than_the_grid_search(trained):
    """What the network replaces: the grid search of every node (HB_FULL_GRID, the method as
    the paper describes it).  A 1920x1080 frame (3 levels, 128x128 grid) with the network, its
    sampled check and the gated fallback takes well under half that time.  (Against the exact
    path with its support bounds, which skips the nodes whose weights do not matter, the
    network gains far less; the bench reports that ratio.)"""
    wl, mix = synth.HD_1080, trained["mix"]
    fr = synth.make_frame(902, wl.H, wl.W, mix.A, wl.nblobs, wl.smin, wl.smax, wl.noise, wl.fmt)
    frame = torch.from_numpy(fr.rgb).to(DEV)
    thb = torch.empty((wl.H, wl.W), dtype=torch.float32, device=DEV)
    so2 = torch.empty_like(thb)

    def frame_ms(ctx):
        for _ in range(3):
            ctx.estimate(frame, thb, so2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(20):
            ctx.estimate(frame, thb, so2)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 20

    with Context(mix.A, GRID, wl.levels, wl.lam, wl.W, wl.H, wl.fmt, binding.HB_FULL_GRID) as ctx:
        grid_ms = frame_ms(ctx)
    with Context(mix.A, GRID, wl.levels, wl.lam, wl.W, wl.H, wl.fmt) as ctx:
        ctx.mlp_set_params(trained["ctx"].mlp_get_params())
        ctx.set_lowpass_mode(binding.HB_MODE_MLP, float("inf"), 256)
        mlp_ms = frame_ms(ctx)
    assert mlp_ms < 0.5 * grid_ms, (mlp_ms, grid_ms)


def test_mode_requires_a_network():
    A = synth.make_mixing(2).A
    with Context(A, GRID, 3, 1e-3, 64, 64, "u8") as ctx:
        with pytest.raises(HbError):
            ctx.set_lowpass_mode(binding.HB_MODE_MLP, 1e-3, 16)
        ctx.mlp_init(1)
        for tol, nsample in ((1e-3, 0), (1e-3, (1 << 24) + 1), (-1.0, 16), (float("nan"), 16)):
            with pytest.raises(HbError) as e:
                ctx.set_lowpass_mode(binding.HB_MODE_MLP, tol, nsample)
            assert e.value.status == 1, (tol, nsample)
        ctx.set_lowpass_mode(binding.HB_MODE_MLP, 1e-3, 1 << 24)
