"""CPU-side checks of the C ABI: the library builds, loads without a GPU, exports every
symbol include/hb.h declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1706_07263_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hb.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hb_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_header_declares_the_binding_symbols():
    assert declared_functions() == sorted(binding.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_strerror_names_every_status(lib):
    for code in range(9):
        msg = lib.hb_strerror(code).decode()
        assert msg and msg != "unknown status"
    assert lib.hb_strerror(99).decode() == "unknown status"


def _create(lib, **kw):
    A = np.array([[0.01, 0.004], [0.012, 0.006], [0.011, 0.003]])
    mix = binding._Mixing()
    for c in range(3):
        for j in range(2):
            mix.A[c][j] = A[c, j]
    g = dict(n0=64, n1=64, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)
    g.update(kw.pop("grid", {}))
    grid = binding._Grid(g["n0"], g["n1"], g["lo0"], g["hi0"], g["lo1"], g["hi1"], g["sigma_l"])
    args = dict(levels=1, lam=1e-3, width=64, height=64, fmt=binding.HB_IN_U8_HWC, flags=0)
    args.update(kw)
    h = ctypes.c_void_p()
    rc = lib.hb_create(ctypes.byref(mix), ctypes.byref(grid), args["levels"], args["lam"], args["width"],
                       args["height"], args["fmt"], args["flags"], ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("kw,status", [
    (dict(levels=7), 2), (dict(levels=-1), 2), (dict(width=0), 2), (dict(height=-5), 2),
    (dict(grid=dict(n0=0)), 2), (dict(grid=dict(sigma_l=0.0)), 2), (dict(grid=dict(hi0=-1.0)), 2),
    (dict(fmt=5), 1), (dict(flags=1 << 9), 1), (dict(lam=-1.0), 1), (dict(lam=float("nan")), 1),
    (dict(levels=0, flags=binding.HB_LOWPASS_TIKHONOV), 1),
    (dict(flags=binding.HB_LOWPASS_LS | binding.HB_LOWPASS_TIKHONOV), 1),
    (dict(levels=5, flags=binding.HB_LOWPASS_LS | binding.HB_LOWPASS_INTENSITY), 1),
])
def test_create_rejects_bad_arguments_without_a_device(lib, kw, status):
    rc, h = _create(lib, **kw)
    assert rc == status
    assert not h.value


def test_null_arguments_are_rejected(lib):
    assert lib.hb_create(None, None, 1, 1e-3, 8, 8, 1, 0, None) == 1
    assert lib.hb_estimate(None, None, 0, None, None, None) == 1
    assert lib.hb_estimate_host(None, None, 0, None, None, None) == 1
    assert lib.hb_estimate_host_async(None, None, 0, None, None, None) == 1
    assert lib.hb_posterior_mean(None, None, 0, None, None) == 1
    assert lib.hb_lowpass_shape(None, None, None) == 1
    assert lib.hb_launch_count(None) == 0
    assert lib.hb_server_drain(None, 0) == 1
    assert lib.hb_server_pause(None, 1) == 1
    assert lib.hb_mlp_save(None, b"net.bin") == 1
    assert lib.hb_mlp_load(None, b"net.bin") == 1
    lib.hb_destroy(None)


def test_host_buffer_helpers():
    """Addresses and row strides of host frames as the host entry points pass them: NumPy
    arrays and CPU tensors, contiguous or a row slice of a wider frame."""
    torch = pytest.importorskip("torch")
    a = np.zeros((6, 10, 3), dtype=np.uint8)
    assert binding._host_ptr(a).value == a.ctypes.data
    assert binding._host_row_stride(a) == 30
    sub = a[:, 2:7]
    assert binding._host_row_stride(sub) == 30 and binding._host_ptr(sub).value == a.ctypes.data + 6
    t = torch.zeros((4, 5, 3), dtype=torch.float32)
    assert binding._host_ptr(t).value == t.data_ptr()
    assert binding._host_row_stride(t) == 5 * 3 * 4
    assert binding._host_row_stride(t[:, 1:4]) == 60
