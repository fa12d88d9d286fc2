"""Out-of-bounds evidence for the output buffers (compute-sanitizer is closed on this machine):
every output the library writes -- THb, SO2, and the debug outputs (block means, low-pass
concentrations, HbO2, Hb) -- is a view into a larger buffer whose elements before and after
the view hold a sentinel bit pattern; after calls on ragged sizes (1x1 up to 602x998, 0..6
levels, 8-bit and float input, device and host entry points) every sentinel is intact."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1706_07263_gb300 import Context, build, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
PAD = 4096                      # sentinel elements on each side of a view
GRID = dict(n0=64, n1=48, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)


def _guarded(n, dtype):
    """(buffer, view of n elements in its middle); the rest holds a sentinel pattern."""
    nbytes = torch.tensor([], dtype=dtype).element_size()
    buf = torch.empty(n + 2 * PAD, dtype=dtype, device=DEV)
    buf.view(torch.uint8).fill_(0xA5)
    return buf, buf[PAD:PAD + n], nbytes


def _intact(buf, n):
    raw = buf.view(torch.uint8)
    es = raw.numel() // buf.numel()
    head, tail = raw[:PAD * es], raw[(PAD + n) * es:]
    return bool((head == 0xA5).all()) and bool((tail == 0xA5).all())


@pytest.mark.parametrize("H,W,levels,fmt", [(1, 1, 0, "u8"), (1, 1, 3, "f32"), (13, 22, 1, "u8"), (13, 22, 2, "f32"),
                                            (13, 22, 4, "u8"), (37, 41, 5, "u8"), (602, 998, 3, "u8"),
                                            (602, 998, 6, "f32"), (300, 500, 2, "u8"), (1080, 1920, 3, "u8")])
def test_outputs_are_written_inside_their_views(H, W, levels, fmt):
    build.build()
    mix = synth.make_mixing(5)
    fr = synth.make_frame(61 + H + W, H, W, mix.A, 6, 2.0, 30.0, 0.01, fmt)
    frame = torch.from_numpy(fr.rgb).to(DEV)
    with Context(mix.A, GRID, levels, 1e-3, W, H, fmt) as ctx:
        hl, wl = ctx.lowpass_shape()
        bufs = {}
        for name, n, dt in (("thb", H * W, torch.float32), ("so2", H * W, torch.float32),
                            ("ybar", hl * wl * 3, torch.float64), ("conc", hl * wl * 2, torch.float32),
                            ("hbo2", H * W, torch.float32), ("hb", H * W, torch.float32)):
            bufs[name] = (*_guarded(n, dt)[:2], n)
        v = {k: b[1] for k, b in bufs.items()}
        for _ in range(2):
            ctx.estimate(frame, v["thb"], v["so2"])
            ctx.estimate_debug(frame, v["ybar"], v["conc"], v["hbo2"], v["hb"])
        torch.cuda.synchronize()
        for name, (buf, view, n) in bufs.items():
            assert _intact(buf, n), f"{name} written outside its {n} elements"
            assert bool(torch.isfinite(view).all()), name
        # the host entry points, into NumPy arrays with sentinel margins
        host = {k: np.full(H * W + 2 * PAD, np.float32(np.nan), np.float32) for k in ("thb", "so2")}
        for k in host:
            host[k].view(np.uint32)[:] = 0xA5A5A5A5
        th = host["thb"][PAD:PAD + H * W].reshape(H, W)
        sh = host["so2"][PAD:PAD + H * W].reshape(H, W)
        ctx.estimate_host(fr.rgb, th, sh)
        for k, a in host.items():
            u = a.view(np.uint32)
            assert (u[:PAD] == 0xA5A5A5A5).all() and (u[PAD + H * W:] == 0xA5A5A5A5).all(), k
        np.testing.assert_array_equal(th, v["thb"].cpu().numpy().reshape(H, W))
