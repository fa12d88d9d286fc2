"""The binding refuses buffers whose type, size or device differ from what the C entry
points assume, before any call reaches the library: a float32 block-mean array read as
float64, an output shorter than the pixels it receives, or a tensor on another device
than the call runs on would otherwise make a kernel read or write out of bounds.  These
run without a GPU: CPU tensors, NumPy arrays and a stand-in object for a CUDA tensor."""
import types

import numpy as np
import pytest

from paper_1706_07263_gb300 import binding

torch = pytest.importorskip("torch")

GRID = dict(n0=16, n1=16, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)
A = np.array([[0.01, 0.004], [0.012, 0.006], [0.011, 0.003]])


class FakeCuda:
    """What _dev_ptr reads of a CUDA tensor: dtype, element count, device, layout."""

    is_cuda = True

    def __init__(self, dtype, n, index=0, contiguous=True):
        self.dtype = dtype
        self._n = n
        self.device = types.SimpleNamespace(index=index)
        self._c = contiguous

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        return 4096


def test_dev_ptr_checks_dtype_count_device_and_layout():
    ok = FakeCuda(torch.float64, 30)
    assert binding._dev_ptr(ok, "ybar", "float64", 30, multiple=3, device=0).value == 4096
    with pytest.raises(ValueError, match="dtype float64"):
        binding._dev_ptr(FakeCuda(torch.float32, 30), "ybar", "float64", multiple=3, device=0)
    with pytest.raises(ValueError, match="multiple of 3"):
        binding._dev_ptr(FakeCuda(torch.float64, 31), "ybar", "float64", multiple=3, device=0)
    with pytest.raises(ValueError, match="at least 20"):
        binding._dev_ptr(FakeCuda(torch.float32, 19), "conc", "float32", 20, device=0)
    with pytest.raises(ValueError, match="cuda:1"):
        binding._dev_ptr(FakeCuda(torch.float32, 20, index=1), "conc", "float32", 20, device=0)
    with pytest.raises(ValueError, match="contiguous"):
        binding._dev_ptr(FakeCuda(torch.float32, 20, contiguous=False), "conc", "float32", 20, device=0)
    with pytest.raises(ValueError, match="CUDA tensor"):
        binding._dev_ptr(torch.zeros(20), "conc", "float32", 20)


def test_static_posterior_refuses_wrong_types_and_sizes():
    with pytest.raises(ValueError, match="dtype float64"):
        binding.posterior_mean_static(A, GRID, torch.zeros((10, 3), dtype=torch.float32),
                                      torch.zeros((10, 2)))
    with pytest.raises(ValueError, match="multiple of 3"):
        binding.posterior_mean_static(A, GRID, torch.zeros(10, dtype=torch.float64), torch.zeros((10, 2)))
    with pytest.raises(ValueError, match="CUDA tensor"):
        binding.posterior_mean_static(A, GRID, torch.zeros((10, 3), dtype=torch.float64),
                                      torch.zeros((10, 2), dtype=torch.float64))


def _context(fmt="u8", width=64, height=48, levels=3):
    """A Context as hb_create would leave it, without a device (nothing reaches the library:
    every call below is refused while its arguments are checked)."""
    c = object.__new__(binding.Context)
    c._h = None
    c.fmt, c.width, c.height, c.levels, c.device = fmt, width, height, levels, 0
    b = 1 << levels
    c.npix_ll = ((height + b - 1) // b) * ((width + b - 1) // b)
    return c


def test_context_calls_refuse_mismatched_buffers():
    c = _context()
    frame = FakeCuda(torch.uint8, 48 * 64 * 3)
    good = FakeCuda(torch.float32, 48 * 64)
    with pytest.raises(ValueError, match="dtype uint8"):
        c.estimate(FakeCuda(torch.float32, 48 * 64 * 3), good, good, row_stride_bytes=64 * 3)
    with pytest.raises(ValueError, match="at least"):
        c.estimate(FakeCuda(torch.uint8, 48 * 64 * 3 - 1), good, good, row_stride_bytes=64 * 3)
    with pytest.raises(ValueError, match="row stride"):
        c.estimate(frame, good, good, row_stride_bytes=64 * 3 - 1)
    with pytest.raises(ValueError, match="thb"):
        c.estimate(frame, FakeCuda(torch.float32, 48 * 64 - 1), good, row_stride_bytes=64 * 3)
    with pytest.raises(ValueError, match="cuda:1"):
        c.estimate(frame, good, FakeCuda(torch.float32, 48 * 64, index=1), row_stride_bytes=64 * 3)
    n = c.npix_ll
    with pytest.raises(ValueError, match="dtype float64"):
        c.posterior_mean(FakeCuda(torch.float32, 3 * n), FakeCuda(torch.float32, 2 * n))
    with pytest.raises(ValueError, match="at least"):
        c.posterior_mean(FakeCuda(torch.float64, 3 * n), FakeCuda(torch.float32, 2 * n - 1))
    with pytest.raises(ValueError, match="float32"):
        c.mlp_forward(FakeCuda(torch.float64, 3 * n), FakeCuda(torch.float32, 2 * n))
    with pytest.raises(ValueError, match="target"):
        c.mlp_train(FakeCuda(torch.float32, 3 * n), FakeCuda(torch.float32, 2 * n - 2), 1)
    with pytest.raises(ValueError, match="grad"):
        c.mlp_gradient(FakeCuda(torch.float32, 3 * n), FakeCuda(torch.float32, 2 * n),
                       FakeCuda(torch.float32, binding.MLP_NPARAMS - 1), FakeCuda(torch.float32, 1))


def test_host_calls_refuse_mismatched_buffers():
    c = _context(fmt="f32", width=20, height=16, levels=2)
    thb = np.zeros((16, 20), np.float32)
    with pytest.raises(ValueError, match="dtype float32"):
        c.estimate_host(np.zeros((16, 20, 3), np.uint8), thb, thb.copy())
    with pytest.raises(ValueError, match="16 rows"):
        c.estimate_host(np.zeros((15, 20, 3), np.float32), thb, thb.copy())
    with pytest.raises(ValueError, match="so2"):
        c.estimate_host_async(np.zeros((16, 20, 3), np.float32), thb, np.zeros((16, 19), np.float32))
    with pytest.raises(ValueError, match="16 rows"):
        c.estimate_host(np.zeros((16, 19, 3), np.float32), thb, thb.copy())
    with pytest.raises(ValueError, match="16 rows"):                       # pixels of a row not contiguous
        c.estimate_host(np.zeros((16, 40, 3), np.float32)[:, ::2], thb, thb.copy())
    with pytest.raises(ValueError, match="thb"):
        c.estimate_host(np.zeros((16, 20, 3), np.float32), np.zeros((16, 20), np.float64), thb)
