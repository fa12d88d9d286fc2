"""FP64 CPU oracle of the haemoglobin estimator (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package.  It wraps ``hb_oracle.c`` (plain C, FP64, libm) with
ctypes and shares nothing with the CUDA library: no code, header, table or
constant.  ``build()`` compiles the C file with gcc; it is called on first
use when the shared object is missing or older than the source.

Functions (all NumPy in, NumPy out, float64):
  log_atten(frame)                      y = -ln(max(I, eps))                (Eq. 8's -log)
  haar_level(x) / haar_level_inv(...)   one 2x2-window transform level     (Eq. 1-2, Eq. 4)
  tikhonov_operator(A, lam, relative)   M = (A^T A + gamma I)^-1 A^T       (Eq. 5)
  posterior_mean(ybar, A, grid)         grid posterior mean, flat prior    (Section 2, Eq. 8-11)
  estimate(frame, A, grid, levels, lam) whole per-frame estimator
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hb_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

FMT = {"f32": 0, "u8": 1}


def build(force: bool = False) -> str:
    """Compile hb_oracle.c into liboracle.so (gcc, -O2, IEEE semantics kept)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        D = ctypes.POINTER(ctypes.c_double)
        V = ctypes.c_void_p
        i, l, d = ctypes.c_int, ctypes.c_long, ctypes.c_double
        lib.hbo_log_atten.argtypes = [V, i, i, i, l, d, D]
        lib.hbo_pad_edge.argtypes = [D, i, i, i, i, i, D]
        lib.hbo_haar_level.argtypes = [D, i, i, i, D, D, D, D]
        lib.hbo_haar_level_inv.argtypes = [D, D, D, D, i, i, i, D]
        lib.hbo_tikhonov_operator.argtypes = [D, d, i, D]
        lib.hbo_tikhonov_operator.restype = d
        lib.hbo_tikhonov_operator_illum.argtypes = [D, d, i, D]
        lib.hbo_tikhonov_operator_illum.restype = d
        lib.hbo_posterior_mean.argtypes = [D, D, i, i, d, d, d, d, d, i, D]
        lib.hbo_posterior_mean_many.argtypes = [D, l, D, i, i, d, d, d, d, d, i, i, D]
        lib.hbo_estimate.argtypes = [V, i, i, i, l, D, d, i, i, i, d, d, d, d, d, i, i, i, i, i,
                                     D, D, D, D, D, D]
        lib.hbo_estimate.restype = i
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def eps_for(fmt: str) -> float:
    """Intensity floor before the logarithm: one 8-bit code step, or 1e-6 for float input."""
    return 1.0 / 255.0 if fmt == "u8" else 1e-6


def log_atten(frame: np.ndarray) -> np.ndarray:
    fmt = "u8" if frame.dtype == np.uint8 else "f32"
    fr = np.ascontiguousarray(frame if fmt == "u8" else frame.astype(np.float32))
    H, W, _ = fr.shape
    y = np.empty((H, W, 3))
    _load().hbo_log_atten(fr.ctypes.data, FMT[fmt], H, W, fr.strides[0], eps_for(fmt), _p(y))
    return y


def pad_edge(x: np.ndarray, Hp: int, Wp: int) -> np.ndarray:
    x = _f64(x)
    H, W, C = x.shape
    out = np.empty((Hp, Wp, C))
    _load().hbo_pad_edge(_p(x), H, W, C, Hp, Wp, _p(out))
    return out


def haar_level(x: np.ndarray):
    """One analysis level; returns (LL, D1, D2, D3), each (h/2, w/2, C)."""
    x = _f64(x)
    h, w, C = x.shape
    bands = [np.empty((h // 2, w // 2, C)) for _ in range(4)]
    _load().hbo_haar_level(_p(x), h, w, C, *[_p(b) for b in bands])
    return tuple(bands)


def haar_level_inv(ll, d1, d2, d3) -> np.ndarray:
    ll, d1, d2, d3 = (_f64(b) for b in (ll, d1, d2, d3))
    h2, w2, C = ll.shape
    out = np.empty((2 * h2, 2 * w2, C))
    _load().hbo_haar_level_inv(_p(ll), _p(d1), _p(d2), _p(d3), h2, w2, C, _p(out))
    return out


def haar_forward(x: np.ndarray, levels: int):
    """Multi-level analysis: returns (LL_n, [(D1, D2, D3) for level 1..n])."""
    details = []
    cur = _f64(x)
    for _ in range(levels):
        ll, d1, d2, d3 = haar_level(cur)
        details.append((d1, d2, d3))
        cur = ll
    return cur, details


def haar_inverse(ll: np.ndarray, details) -> np.ndarray:
    cur = _f64(ll)
    for d1, d2, d3 in reversed(details):
        cur = haar_level_inv(cur, d1, d2, d3)
    return cur


def tikhonov_operator(A: np.ndarray, lam: float, relative: bool = True, illumination: bool = False):
    """Returns (M 2x3, gamma); illumination: with the constant column of Eq. 8."""
    A = _f64(A).reshape(3, 2)
    M = np.empty((2, 3))
    fn = _load().hbo_tikhonov_operator_illum if illumination else _load().hbo_tikhonov_operator
    g = fn(_p(A), float(lam), int(relative), _p(M))
    return M, g


def posterior_mean(ybar: np.ndarray, A: np.ndarray, grid: dict, nthreads: int = 1,
                   illumination: bool = False) -> np.ndarray:
    """Posterior mean (HbO2, Hb) for each row of ybar (..., 3); illumination: with the
    constant term of Eq. 8 integrated out."""
    yb = _f64(ybar)
    shape = yb.shape[:-1]
    yb = yb.reshape(-1, 3)
    A = _f64(A).reshape(3, 2)
    out = np.empty((yb.shape[0], 2))
    _load().hbo_posterior_mean_many(_p(yb), yb.shape[0], _p(A), grid["n0"], grid["n1"], grid["lo0"], grid["hi0"],
                                    grid["lo1"], grid["hi1"], grid["sigma_l"], int(illumination), nthreads, _p(out))
    return out.reshape(shape + (2,))


def estimate(frame: np.ndarray, A: np.ndarray, grid: dict, levels: int, lam: float, relative: bool = True,
             lowpass: str = "bayes", nthreads: int = 1, illumination: bool = False,
             intensity_lowpass: bool = False) -> dict:
    """Whole estimator on one HWC frame (uint8 codes or float32 intensities); illumination:
    with the constant (illumination) term of Eq. 8; intensity_lowpass: the low pass is -log
    of the block mean of the intensities (Eq. 3-8 literally); lowpass: "bayes" (the grid
    posterior mean, Eq. 8-11), "tikhonov" (M on every band, Eq. 5) or "ls" (least squares on
    the low pass, Eq. 9).

    Returns a dict of float64 arrays: hbo2, hb, thb, so2 (H, W); ybar_ll
    (hl, wl, 3); conc_ll (hl, wl, 2)."""
    fmt = "u8" if frame.dtype == np.uint8 else "f32"
    fr = np.ascontiguousarray(frame if fmt == "u8" else frame.astype(np.float32))
    H, W, _ = fr.shape
    blk = 1 << levels
    Hp, Wp = -(-H // blk) * blk, -(-W // blk) * blk
    hl, wl = Hp >> levels, Wp >> levels
    out = {k: np.empty((H, W)) for k in ("hbo2", "hb", "thb", "so2")}
    out["ybar_ll"] = np.empty((hl, wl, 3))
    out["conc_ll"] = np.empty((hl, wl, 2))
    A = _f64(A).reshape(3, 2)
    rc = _load().hbo_estimate(fr.ctypes.data, FMT[fmt], H, W, fr.strides[0], _p(A), float(lam), int(relative),
                              grid["n0"], grid["n1"], grid["lo0"], grid["hi0"], grid["lo1"], grid["hi1"],
                              grid["sigma_l"], levels, {"bayes": 0, "tikhonov": 1, "ls": 2}[lowpass], int(illumination),
                              int(intensity_lowpass), nthreads,
                              _p(out["hbo2"]), _p(out["hb"]), _p(out["thb"]), _p(out["so2"]),
                              _p(out["ybar_ll"]), _p(out["conc_ll"]))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return out
