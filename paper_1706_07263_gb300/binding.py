"""ctypes binding of libhb.so (include/hb.h).

Argument marshalling only: tensors are passed as raw device pointers, streams as
``cudaStream_t`` handles, and every step of the estimator runs in the library's
CUDA kernels.  There is no CPU path: loading fails loudly when the library has
not been built, and calls on tensors that are not on a CUDA device are refused.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhb.so")

HB_IN_F32_HWC = 0
HB_IN_U8_HWC = 1
HB_LAMBDA_ABSOLUTE = 1 << 0
HB_LOWPASS_TIKHONOV = 1 << 1
STAGES = ("analysis", "lowpass", "synthesis", "frame")

STATUS = {0: "HB_OK", 1: "HB_ERR_ARG", 2: "HB_ERR_SHAPE", 3: "HB_ERR_CUDA", 4: "HB_ERR_OOM", 5: "HB_ERR_BUDGET",
          6: "HB_ERR_TIMEOUT", 7: "HB_ERR_STATE", 8: "HB_ERR_IO"}

# Every symbol include/hb.h declares (checked by the CPU tests against the built library).
EXPORTED = ("hb_create", "hb_destroy", "hb_estimate", "hb_estimate_host", "hb_estimate_host_async", "hb_estimate_debug",
            "hb_posterior_mean",
            "hb_lowpass_shape", "hb_launch_count", "hb_timing_start", "hb_timing_read", "hb_timing_nodes", "hb_timing_rows",
            "hb_strerror",
            "hb_mlp_init", "hb_mlp_set_params", "hb_mlp_get_params", "hb_mlp_save", "hb_mlp_load", "hb_lowpass_pairs", "hb_mlp_train",
            "hb_mlp_gradient", "hb_mlp_forward", "hb_set_lowpass_mode", "hb_lowpass_stats", "hb_mlp_certify",
            "hb_server_create", "hb_server_destroy", "hb_stream_open", "hb_stream_close", "hb_submit", "hb_poll",
            "hb_release", "hb_server_pause", "hb_server_drain", "hb_server_stats", "hb_posterior_mean_static",
            "hb_measure_ex2_rate")
HB_FULL_GRID = 1 << 2
HB_ILLUMINATION = 1 << 5
HB_LOWPASS_INTENSITY = 1 << 6
HB_LOWPASS_LS = 1 << 7
HB_NODE_SUMS = 1 << 8
HB_SERVE_SEQUENTIAL = 1 << 4
MLP_NPARAMS = 4546
HB_MODE_BAYES = 0
HB_MODE_MLP = 1
HB_MODE_MLP_MEAN_GATE = 2
STATIC_MAX_PIXELS = 65536


class _Result(ctypes.Structure):
    _fields_ = [("stream_id", ctypes.c_int), ("slot", ctypes.c_int), ("tag", ctypes.c_uint64),
                ("latency_ms", ctypes.c_double), ("thb_host", ctypes.c_void_p), ("so2_host", ctypes.c_void_p)]


class _ServerInfo(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_long), ("frames", ctypes.c_long), ("max_batch_frames", ctypes.c_long),
                ("queued", ctypes.c_long), ("mean_batch_frames", ctypes.c_double), ("bytes_in_use", ctypes.c_size_t),
                ("budget_bytes", ctypes.c_size_t)]


class HbError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


class _Mixing(ctypes.Structure):
    _fields_ = [("A", (ctypes.c_double * 2) * 3)]


class _Grid(ctypes.Structure):
    _fields_ = [("n0", ctypes.c_int), ("n1", ctypes.c_int), ("lo0", ctypes.c_double), ("hi0", ctypes.c_double),
                ("lo1", ctypes.c_double), ("hi1", ctypes.c_double), ("sigma_l", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libhb.so and declare its signatures.  Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run paper_1706_07263_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    P, I, L, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_size_t
    lib.hb_create.argtypes = [ctypes.POINTER(_Mixing), ctypes.POINTER(_Grid), I, D, I, I, I, ctypes.c_uint,
                              ctypes.POINTER(P)]
    lib.hb_destroy.argtypes = [P]
    lib.hb_destroy.restype = None
    lib.hb_estimate.argtypes = [P, P, S, P, P, P]
    lib.hb_estimate_host.argtypes = [P, P, S, P, P, P]
    lib.hb_estimate_host_async.argtypes = [P, P, S, P, P, P]
    lib.hb_estimate_debug.argtypes = [P, P, S, P, P, P, P, P]
    lib.hb_posterior_mean.argtypes = [P, P, L, P, P]
    lib.hb_lowpass_shape.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.hb_launch_count.argtypes = [P]
    lib.hb_launch_count.restype = L
    lib.hb_timing_start.argtypes = [P, I]
    lib.hb_timing_read.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(L)]
    lib.hb_timing_nodes.argtypes = [P, ctypes.POINTER(ctypes.c_ulonglong)]
    lib.hb_timing_rows.argtypes = [P, ctypes.POINTER(ctypes.c_ulonglong * 2)]
    lib.hb_strerror.argtypes = [I]
    lib.hb_strerror.restype = ctypes.c_char_p
    lib.hb_posterior_mean_static.argtypes = [ctypes.POINTER(_Mixing), ctypes.POINTER(_Grid), P, L, P, P]
    F = ctypes.POINTER(ctypes.c_float)
    lib.hb_mlp_init.argtypes = [P, ctypes.c_uint]
    lib.hb_mlp_set_params.argtypes = [P, F]
    lib.hb_mlp_get_params.argtypes = [P, F]
    lib.hb_mlp_save.argtypes = [P, ctypes.c_char_p]
    lib.hb_mlp_load.argtypes = [P, ctypes.c_char_p]
    lib.hb_lowpass_pairs.argtypes = [P, P, S, P, P, P]
    lib.hb_mlp_train.argtypes = [P, P, P, L, I, I, D, ctypes.c_uint, F, P]
    lib.hb_mlp_gradient.argtypes = [P, P, P, L, P, P, P]
    lib.hb_mlp_forward.argtypes = [P, P, L, P, P]
    lib.hb_set_lowpass_mode.argtypes = [P, I, D, I]
    lib.hb_lowpass_stats.argtypes = [P, ctypes.POINTER(L), ctypes.POINTER(L), ctypes.POINTER(L)]
    lib.hb_mlp_certify.argtypes = [P, D, ctypes.POINTER(D), P]
    lib.hb_server_create.argtypes = [ctypes.POINTER(_Mixing), ctypes.POINTER(_Grid), D, ctypes.c_uint, I, S, I, L,
                                     ctypes.POINTER(P)]
    lib.hb_server_destroy.argtypes = [P]
    lib.hb_server_destroy.restype = None
    lib.hb_stream_open.argtypes = [P, I, I, I, I, ctypes.POINTER(I)]
    lib.hb_stream_close.argtypes = [P, I]
    lib.hb_submit.argtypes = [P, I, P, S, ctypes.c_uint64]
    lib.hb_poll.argtypes = [P, ctypes.POINTER(_Result), I, ctypes.POINTER(I), I]
    lib.hb_release.argtypes = [P, I, I]
    lib.hb_server_stats.argtypes = [P, ctypes.POINTER(_ServerInfo)]
    lib.hb_server_pause.argtypes = [P, I]
    lib.hb_server_drain.argtypes = [P, I]
    lib.hb_measure_ex2_rate.argtypes = [ctypes.POINTER(D), ctypes.POINTER(I)]
    for name in EXPORTED:
        getattr(lib, name)
    _lib = lib
    return lib


def _check(rc: int, what: str):
    if rc != 0:
        raise HbError(rc, what)


def _dev_ptr(t, what, dtype=None, min_numel=None, multiple=None, device=None):
    """Device pointer of a tensor, after checking what the C side assumes of it.

    dtype: the element type the entry point reads or writes ("float32", "float64", "uint8");
    min_numel: the fewest elements it touches; multiple: the element count must divide by it;
    device: the CUDA device index the call runs on ("current": the current device).  Violations raise ValueError before
    anything is launched, so no kernel is ever given a buffer shorter than it assumes."""
    if t is None:
        return None
    if dtype is not None and str(getattr(t, "dtype", "")).replace("torch.", "") != dtype:
        raise ValueError(f"{what} must have dtype {dtype}, not {getattr(t, 'dtype', type(t).__name__)}")
    n = int(t.numel())
    if multiple is not None and n % multiple:
        raise ValueError(f"{what} must hold a multiple of {multiple} elements, not {n}")
    if min_numel is not None and n < min_numel:
        raise ValueError(f"{what} must hold at least {min_numel} elements, not {n}")
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{what} must be a CUDA tensor")
    if device == "current":
        device = _current_device()
    if device is not None and t.device.index != device:
        raise ValueError(f"{what} is on cuda:{t.device.index}, but the call runs on cuda:{device}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _current_device():
    import torch
    return torch.cuda.current_device()


def _frame_dtype(fmt):
    return "uint8" if fmt == "u8" else "float32"


def _host_ptr(a, what="buffer", dtype=None, min_numel=None):
    """Address of a host buffer: a CPU tensor (pinned for speed) or a NumPy array, after
    checking its element type and that it holds at least min_numel elements."""
    if getattr(a, "is_cuda", False):
        raise ValueError(f"{what} must be in host memory")
    if dtype is not None and str(getattr(a, "dtype", "")).replace("torch.", "") != dtype:
        raise ValueError(f"{what} must have dtype {dtype}, not {getattr(a, 'dtype', type(a).__name__)}")
    if min_numel is not None:
        n = int(a.numel() if hasattr(a, "numel") and callable(a.numel) else np.asarray(a).size)
        if n < min_numel:
            raise ValueError(f"{what} must hold at least {min_numel} elements, not {n}")
    return ctypes.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)


def _host_row_stride(frame) -> int:
    """Bytes between rows of an HWC host frame (NumPy array or CPU tensor)."""
    return frame.strides[0] if isinstance(frame, np.ndarray) else frame.stride(0) * frame.element_size()


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """One estimator configuration (hb_create); see include/hb.h for the semantics."""

    def __init__(self, A, grid: dict, levels: int, lam: float, width: int, height: int, fmt: str = "u8",
                 flags: int = 0):
        lib = load()
        mix = _Mixing()
        A = np.asarray(A, dtype=np.float64).reshape(3, 2)
        for c in range(3):
            for j in range(2):
                mix.A[c][j] = float(A[c, j])
        g = _Grid(int(grid["n0"]), int(grid["n1"]), float(grid["lo0"]), float(grid["hi0"]), float(grid["lo1"]),
                  float(grid["hi1"]), float(grid["sigma_l"]))
        self.fmt = fmt
        self.width, self.height, self.levels = width, height, levels
        self._h = ctypes.c_void_p()
        _check(lib.hb_create(ctypes.byref(mix), ctypes.byref(g), levels, float(lam), width, height,
                             HB_IN_U8_HWC if fmt == "u8" else HB_IN_F32_HWC, flags, ctypes.byref(self._h)),
               "hb_create")
        # hb_create binds the context to the current device; its calls run there
        self.device = _current_device()
        b = 1 << levels
        self.npix_ll = ((height + b - 1) // b) * ((width + b - 1) // b)

    def _frame(self, frame, stride, what="frame"):
        """Pointer of a device frame after checking its type, device and extent for `stride`."""
        es = 1 if self.fmt == "u8" else 4
        if stride < self.width * 3 * es:
            raise ValueError(f"row stride {stride} B is shorter than a row of {self.width} RGB pixels")
        need = ((self.height - 1) * stride + self.width * 3 * es + es - 1) // es
        return _dev_ptr(frame, what, _frame_dtype(self.fmt), need, device=self.device)

    def _map(self, t, what):
        """Pointer of an H x W float32 output map on the context's device."""
        return _dev_ptr(t, what, "float32", self.width * self.height, device=self.device)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().hb_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def lowpass_shape(self):
        hl, wl = ctypes.c_int(), ctypes.c_int()
        _check(load().hb_lowpass_shape(self._h, ctypes.byref(hl), ctypes.byref(wl)), "hb_lowpass_shape")
        return hl.value, wl.value

    def estimate(self, frame, thb, so2, stream=None, row_stride_bytes=None):
        stride = row_stride_bytes if row_stride_bytes is not None else frame.stride(0) * frame.element_size()
        _check(load().hb_estimate(self._h, self._frame(frame, stride), stride, self._map(thb, "thb"),
                                  self._map(so2, "so2"), _stream(stream)), "hb_estimate")

    def estimate_host(self, frame: np.ndarray, thb: np.ndarray, so2: np.ndarray, stream=None):
        """Host buffers in and out (NumPy or pinned CPU tensors)."""
        _check(load().hb_estimate_host(self._h, self._host_frame(frame), _host_row_stride(frame),
                                       self._host_map(thb, "thb"), self._host_map(so2, "so2"), _stream(stream)),
               "hb_estimate_host")

    def estimate_host_async(self, frame, thb, so2, stream=None):
        """As estimate_host, returning before the results arrive: they are in thb/so2 once
        `stream` has been synchronised; the buffers must stay alive and untouched until then."""
        _check(load().hb_estimate_host_async(self._h, self._host_frame(frame), _host_row_stride(frame),
                                             self._host_map(thb, "thb"), self._host_map(so2, "so2"),
                                             _stream(stream)), "hb_estimate_host_async")

    def _host_frame(self, frame):
        """Address of a host HWC frame after checking its type and the pixels within a row."""
        p = _host_ptr(frame, "frame", _frame_dtype(self.fmt))
        row = frame[0] if len(frame.shape) > 1 else frame
        contiguous = row.flags["C_CONTIGUOUS"] if isinstance(row, np.ndarray) else row.is_contiguous()
        if frame.shape[0] != self.height or not contiguous or int(np.prod(frame.shape[1:])) < 3 * self.width:
            raise ValueError(f"frame must have {self.height} rows of at least {self.width} contiguous RGB pixels "
                             f"(e.g. shape ({self.height}, {self.width}, 3)), not shape {tuple(frame.shape)}")
        return p

    def _host_map(self, a, what):
        if isinstance(a, np.ndarray) and not a.flags["C_CONTIGUOUS"] or hasattr(a, "is_contiguous") and \
                not a.is_contiguous():
            raise ValueError(f"{what} must be contiguous")
        return _host_ptr(a, what, "float32", self.width * self.height)

    def estimate_debug(self, frame, ybar=None, conc=None, hbo2=None, hb=None, stream=None):
        stride = frame.stride(0) * frame.element_size()
        n = self.npix_ll
        _check(load().hb_estimate_debug(self._h, self._frame(frame, stride), stride,
                                        _dev_ptr(ybar, "ybar", "float64", 3 * n, device=self.device),
                                        _dev_ptr(conc, "conc", "float32", 2 * n, device=self.device),
                                        self._map(hbo2, "hbo2"), self._map(hb, "hb"),
                                        _stream(stream)), "hb_estimate_debug")

    def posterior_mean(self, ybar, conc, stream=None):
        """ybar: float64 (npix, 3) block means; conc: float32, at least npix x 2 values."""
        p_y = _dev_ptr(ybar, "ybar", "float64", multiple=3, device=self.device)
        npix = ybar.numel() // 3
        p_c = _dev_ptr(conc, "conc", "float32", 2 * npix, device=self.device)
        _check(load().hb_posterior_mean(self._h, p_y, npix, p_c, _stream(stream)), "hb_posterior_mean")

    # -------------------------------------------------------------- learned stand-in
    def mlp_init(self, seed: int = 0):
        _check(load().hb_mlp_init(self._h, seed), "hb_mlp_init")

    def mlp_set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        if p.size != MLP_NPARAMS:
            raise ValueError(f"expected {MLP_NPARAMS} parameters")
        _check(load().hb_mlp_set_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "hb_mlp_set_params")

    def mlp_get_params(self) -> np.ndarray:
        p = np.empty(MLP_NPARAMS, dtype=np.float32)
        _check(load().hb_mlp_get_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "hb_mlp_get_params")
        return p

    def mlp_save(self, path):
        """Write the network and the model it was trained for to a file (hb_mlp_save)."""
        _check(load().hb_mlp_save(self._h, os.fsencode(path)), "hb_mlp_save")

    def mlp_load(self, path):
        """Read a network written by mlp_save (hb_mlp_load); raises HbError with HB_ERR_IO for
        a file that is not one, HB_ERR_STATE for a network of another model."""
        _check(load().hb_mlp_load(self._h, os.fsencode(path)), "hb_mlp_load")

    def lowpass_pairs(self, frame, ybar, conc, stream=None):
        stride = frame.stride(0) * frame.element_size()
        n = self.npix_ll
        _check(load().hb_lowpass_pairs(self._h, self._frame(frame, stride), stride,
                                       _dev_ptr(ybar, "ybar", "float32", 3 * n, device=self.device),
                                       _dev_ptr(conc, "conc", "float32", 2 * n, device=self.device),
                                       _stream(stream)), "hb_lowpass_pairs")

    def mlp_train(self, ybar, target, steps: int, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
                  stream=None) -> np.ndarray:
        losses = np.empty(max(steps, 1), dtype=np.float32)
        p_y = _dev_ptr(ybar, "ybar", "float32", multiple=3, device=self.device)
        n = ybar.numel() // 3
        p_t = _dev_ptr(target, "target", "float32", 2 * n, device=self.device)
        _check(load().hb_mlp_train(self._h, p_y, p_t, n, steps, batch, float(lr), seed,
                                   losses.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _stream(stream)),
               "hb_mlp_train")
        return losses[:steps]

    def mlp_gradient(self, ybar, target, grad, loss, stream=None):
        p_y = _dev_ptr(ybar, "ybar", "float32", multiple=3, device=self.device)
        n = ybar.numel() // 3
        _check(load().hb_mlp_gradient(self._h, p_y, _dev_ptr(target, "target", "float32", 2 * n, device=self.device),
                                      n, _dev_ptr(grad, "grad", "float32", MLP_NPARAMS, device=self.device),
                                      _dev_ptr(loss, "loss", "float32", 1, device=self.device),
                                      _stream(stream)), "hb_mlp_gradient")

    def mlp_forward(self, ybar, conc, stream=None):
        p_y = _dev_ptr(ybar, "ybar", "float32", multiple=3, device=self.device)
        n = ybar.numel() // 3
        _check(load().hb_mlp_forward(self._h, p_y, n, _dev_ptr(conc, "conc", "float32", 2 * n, device=self.device),
                                     _stream(stream)), "hb_mlp_forward")

    def set_lowpass_mode(self, mode: int, tol: float = 1e-3, nsample: int = 256):
        _check(load().hb_set_lowpass_mode(self._h, mode, float(tol), nsample), "hb_set_lowpass_mode")

    def lowpass_stats(self):
        """(frames in a learned mode, frames that fell back, low-pass pixels the route sent to
        the exact posterior in the others)."""
        f, b, r = ctypes.c_long(), ctypes.c_long(), ctypes.c_long()
        _check(load().hb_lowpass_stats(self._h, ctypes.byref(f), ctypes.byref(b), ctypes.byref(r)),
               "hb_lowpass_stats")
        return f.value, b.value, r.value

    def mlp_certify(self, tol: float, stream=None) -> float:
        """hb_mlp_certify: trust map of the current network at tolerance tol; returns the share
        of trusted cells."""
        frac = ctypes.c_double()
        _check(load().hb_mlp_certify(self._h, float(tol), ctypes.byref(frac), _stream(stream)), "hb_mlp_certify")
        return frac.value

    def launch_count(self) -> int:
        return int(load().hb_launch_count(self._h))

    def timing_start(self, max_launches: int):
        _check(load().hb_timing_start(self._h, max_launches), "hb_timing_start")

    def timing_nodes(self) -> int:
        """Grid nodes the posterior enumerated since timing_start (synchronises the device)."""
        v = ctypes.c_ulonglong(0)
        _check(load().hb_timing_nodes(self._h, ctypes.byref(v)), "hb_timing_nodes")
        return int(v.value)

    def timing_rows(self, edge: bool = False) -> int:
        """Grid rows the posterior summed in closed form since timing_start (edge: only those
        the box edge cuts off); synchronises the device.  Their nodes are not in timing_nodes."""
        v = (ctypes.c_ulonglong * 2)()
        _check(load().hb_timing_rows(self._h, v), "hb_timing_rows")
        return int(v[1] if edge else v[0])

    def timing_read(self) -> dict:
        ms = (ctypes.c_double * len(STAGES))()
        n = (ctypes.c_long * len(STAGES))()
        _check(load().hb_timing_read(self._h, ms, n), "hb_timing_read")
        return {STAGES[k]: (ms[k], n[k]) for k in range(len(STAGES))}


def _structs(A, grid):
    mix = _Mixing()
    A = np.asarray(A, dtype=np.float64).reshape(3, 2)
    for c in range(3):
        for j in range(2):
            mix.A[c][j] = float(A[c, j])
    g = _Grid(int(grid["n0"]), int(grid["n1"]), float(grid["lo0"]), float(grid["hi0"]), float(grid["lo1"]),
              float(grid["hi1"]), float(grid["sigma_l"]))
    return mix, g


class Server:
    """Continuous-batching server of include/hb.h (hb_server_*).  Results come back as
    NumPy views of the server's pinned host buffers, valid until release()."""

    def __init__(self, A, grid: dict, lam: float, fmt: str = "u8", budget_bytes: int = 20 << 30, max_batch: int = 16,
                 batch_lowpass_pixels: int = 2_000_000, sequential: bool = False, flags: int = 0):
        lib = load()
        mix, g = _structs(A, grid)
        self._h = ctypes.c_void_p()
        self.fmt = fmt
        self.shapes = {}
        fl = flags | (HB_SERVE_SEQUENTIAL if sequential else 0)
        _check(lib.hb_server_create(ctypes.byref(mix), ctypes.byref(g), float(lam), fl,
                                    HB_IN_U8_HWC if fmt == "u8" else HB_IN_F32_HWC, int(budget_bytes), max_batch,
                                    int(batch_lowpass_pixels), ctypes.byref(self._h)), "hb_server_create")

    def open_stream(self, width: int, height: int, levels: int, slots: int = 4) -> int:
        sid = ctypes.c_int(-1)
        _check(load().hb_stream_open(self._h, width, height, levels, slots, ctypes.byref(sid)), "hb_stream_open")
        self.shapes[sid.value] = (height, width)
        return sid.value

    def close_stream(self, sid: int):
        _check(load().hb_stream_close(self._h, sid), "hb_stream_close")
        self.shapes.pop(sid, None)

    def submit(self, sid: int, frame: np.ndarray, tag: int = 0) -> bool:
        """Queue a frame; False when every slot of the stream is busy."""
        fr = np.ascontiguousarray(frame)
        h, w = self.shapes.get(sid, fr.shape[:2])  # an unknown stream is the library's to refuse
        if fr.shape != (h, w, 3) or fr.dtype != (np.uint8 if self.fmt == "u8" else np.float32):
            raise ValueError(f"stream {sid} takes ({h}, {w}, 3) {self.fmt} frames, not {fr.shape} {fr.dtype}")
        rc = load().hb_submit(self._h, sid, ctypes.c_void_p(fr.ctypes.data), fr.strides[0], tag)
        if rc == 7:
            return False
        _check(rc, "hb_submit")
        return True

    def poll(self, max_results: int = 64, wait_us: int = 0):
        res = (_Result * max(max_results, 1))()
        n = ctypes.c_int(0)
        _check(load().hb_poll(self._h, res, max_results, ctypes.byref(n), wait_us), "hb_poll")
        out = []
        for k in range(n.value):
            r = res[k]
            h, w = self.shapes[r.stream_id]
            fp = ctypes.POINTER(ctypes.c_float)
            out.append(dict(stream=r.stream_id, slot=r.slot, tag=r.tag, latency_ms=r.latency_ms,
                            thb=np.ctypeslib.as_array(ctypes.cast(r.thb_host, fp), shape=(h, w)),
                            so2=np.ctypeslib.as_array(ctypes.cast(r.so2_host, fp), shape=(h, w))))
        return out

    def release(self, sid: int, slot: int):
        _check(load().hb_release(self._h, sid, slot), "hb_release")

    def pause(self, paused: bool = True):
        _check(load().hb_server_pause(self._h, int(paused)), "hb_server_pause")

    def drain(self, timeout_ms: int = 10000):
        """Wait until every submitted frame has completed; HbError (status 6) on timeout."""
        _check(load().hb_server_drain(self._h, int(timeout_ms)), "hb_server_drain")

    def stats(self) -> dict:
        i = _ServerInfo()
        _check(load().hb_server_stats(self._h, ctypes.byref(i)), "hb_server_stats")
        return {k: getattr(i, k) for k, _ in _ServerInfo._fields_}

    def close(self):
        if self._h:
            load().hb_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def measure_ex2_rate():
    """(ex2 results per SM clock per SM, SM count) of the current device (hb_measure_ex2_rate)."""
    r, n = ctypes.c_double(), ctypes.c_int()
    _check(load().hb_measure_ex2_rate(ctypes.byref(r), ctypes.byref(n)), "hb_measure_ex2_rate")
    return r.value, n.value


def strerror(status: int) -> str:
    return load().hb_strerror(status).decode()


def posterior_mean_static(A, grid: dict, ybar, conc, stream=None):
    """hb_posterior_mean_static: the posterior step with no allocation (see include/hb.h).

    For callers that may not allocate device memory: real-time loops that must not
    block on the allocator, plug-ins whose host owns all device memory, deployments
    with a fixed device footprint.  ybar: CUDA float64 tensor (npix, 3); conc: CUDA
    float32 tensor (npix, 2), npix <= STATIC_MAX_PIXELS.  The first call on a device
    looks up the library's fixed working array and should precede any stream
    capture; calls share that array, so they must not overlap on the GPU."""
    lib = load()
    mix = _Mixing()
    A = np.asarray(A, dtype=np.float64).reshape(3, 2)
    for c in range(3):
        for j in range(2):
            mix.A[c][j] = float(A[c, j])
    g = _Grid(int(grid["n0"]), int(grid["n1"]), float(grid["lo0"]), float(grid["hi0"]), float(grid["lo1"]),
              float(grid["hi1"]), float(grid["sigma_l"]))
    p_y = _dev_ptr(ybar, "ybar", "float64", multiple=3, device="current")
    npix = ybar.numel() // 3
    p_c = _dev_ptr(conc, "conc", "float32", 2 * npix, device="current")
    _check(lib.hb_posterior_mean_static(ctypes.byref(mix), ctypes.byref(g), p_y, npix, p_c, _stream(stream)),
           "hb_posterior_mean_static")
