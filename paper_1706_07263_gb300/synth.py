"""Seeded synthetic workloads for the haemoglobin-estimation path.

This module only *makes inputs*: a 3x2 mixing matrix built from smooth
spectra, smooth concentration fields, and RGB frames rendered from them with
the Beer-Lambert forward model (Section 2: the fit "satisfies the
Beer-Lambert relation").  It contains none of the estimator's arithmetic
(no Haar transform, no Tikhonov inverse, no posterior), so both the FP64
oracle and the CUDA path can take their inputs from here without sharing
any of the method.

The paper's workloads (RGB views synthesised from in-vivo multispectral data
through calibrated da Vinci camera curves, Section 3.1, and stereo
laparoscope video, Section 3.2) are not available; these generators stand
in for their shape and size only ("mega-pixel sized input images",
Section 3.1).

Recipe (all host-side NumPy, FP64, seeded with ``numpy.random.default_rng``):

* mixing matrix A (3x2): RGB sensitivities are Gaussians at 600/540/460 nm
  with FWHM 80 nm on 400..700 nm at 1 nm steps; the two extinction curves
  (HbO2, Hb) are each a sum of three Gaussians (centre U(400,700) nm, width
  U(10,60) nm, amplitude U(0.2,1)).  A[c, j] is the sensitivity-weighted
  mean of curve j in channel c.  A is rescaled so that the darkest channel
  at the box corner (150, 100) uM has attenuation 2.5, and redrawn until
  cond(A) < 50.
* fields: HbO2 and Hb are each a sum of K Gaussian blobs (centres uniform in
  the frame, sigma U(smin, smax) px, amplitude U(0, 1)), affinely rescaled
  to [0, 150] and [0, 100] uM.
* render: I_c = exp(-sum_j A[c, j] conc_j) + N(0, noise^2); optionally
  quantised to 8 bits as round(255 * clip(I, 0, 1)).
"""
from __future__ import annotations

import dataclasses
import numpy as np

BOX_HBO2 = (0.0, 150.0)   # uM
BOX_HB = (0.0, 100.0)     # uM
WAVELENGTHS = np.arange(400.0, 701.0, 1.0)
RGB_CENTRES = (600.0, 540.0, 460.0)
RGB_FWHM = 80.0


@dataclasses.dataclass
class Mixing:
    A: np.ndarray          # (3, 2) float64, attenuation per uM
    cond: float
    seed: int
    draws: int             # how many spectra draws were needed


@dataclasses.dataclass
class Frame:
    """One rendered RGB frame and the fields it was rendered from."""
    rgb: np.ndarray        # (H, W, 3) float32 intensities or uint8 codes
    fmt: str               # "f32" or "u8"
    hbo2: np.ndarray       # (H, W) float64 ground truth, uM
    hb: np.ndarray         # (H, W) float64 ground truth, uM


def _gauss(x, mu, sigma):
    return np.exp(-0.5 * ((x - mu) / sigma) ** 2)


def make_mixing(seed: int, max_cond: float = 50.0, corner_atten: float = 2.5) -> Mixing:
    """Draw a 3x2 mixing matrix from seeded smooth spectra (see module doc)."""
    rng = np.random.default_rng(seed)
    sig = RGB_FWHM / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    S = np.stack([_gauss(WAVELENGTHS, c, sig) for c in RGB_CENTRES])        # (3, L)
    for draw in range(1, 10001):
        curves = []
        for _ in range(2):
            mu = rng.uniform(400.0, 700.0, 3)
            wd = rng.uniform(10.0, 60.0, 3)
            amp = rng.uniform(0.2, 1.0, 3)
            curves.append(sum(a * _gauss(WAVELENGTHS, m, w) for a, m, w in zip(amp, mu, wd)))
        E = np.stack(curves, axis=1)                                           # (L, 2)
        A = (S @ E) / S.sum(axis=1, keepdims=True)                             # (3, 2)
        corner = A @ np.array([BOX_HBO2[1], BOX_HB[1]])
        A = A * (corner_atten / corner.max())
        cond = float(np.linalg.cond(A))
        if cond < max_cond:
            return Mixing(A=A, cond=cond, seed=seed, draws=draw)
    raise RuntimeError("no well-conditioned mixing matrix found")


def make_fields(rng: np.random.Generator, H: int, W: int, nblobs: int, smin: float, smax: float,
                centres=None, sigmas=None, amps=None):
    """Two smooth fields (HbO2, Hb) in uM, each a sum of Gaussian blobs.

    Blob parameters may be passed in (video generators move the centres);
    otherwise they are drawn from ``rng``.  Returns (hbo2, hb, params)."""
    ys = np.arange(H, dtype=np.float64)
    xs = np.arange(W, dtype=np.float64)
    out = []
    params = []
    for f, box in enumerate((BOX_HBO2, BOX_HB)):
        if centres is None:
            cy = rng.uniform(0, H, nblobs)
            cx = rng.uniform(0, W, nblobs)
            sg = rng.uniform(smin, smax, nblobs)
            am = rng.uniform(0.0, 1.0, nblobs)
        else:
            cy, cx = centres[f]
            sg, am = sigmas[f], amps[f]
        field = np.zeros((H, W))
        for b in range(nblobs):
            field += am[b] * np.outer(_gauss(ys, cy[b], sg[b]), _gauss(xs, cx[b], sg[b]))
        lo, hi = field.min(), field.max()
        field = (field - lo) / (hi - lo if hi > lo else 1.0)
        out.append(box[0] + field * (box[1] - box[0]))
        params.append(((cy, cx), sg, am))
    return out[0], out[1], params


def render(A: np.ndarray, hbo2: np.ndarray, hb: np.ndarray, rng: np.random.Generator,
           noise: float, fmt: str) -> np.ndarray:
    """Beer-Lambert RGB intensities plus Gaussian noise, as float32 or uint8 codes."""
    att = hbo2[..., None] * A[:, 0] + hb[..., None] * A[:, 1]          # (H, W, 3)
    I = np.exp(-att)
    if noise > 0:
        I = I + rng.normal(0.0, noise, I.shape)
    if fmt == "u8":
        return np.rint(255.0 * np.clip(I, 0.0, 1.0)).astype(np.uint8)
    if fmt == "f32":
        return I.astype(np.float32)
    raise ValueError(fmt)


def make_frame(seed: int, H: int, W: int, A: np.ndarray, nblobs: int, smin: float, smax: float,
               noise: float, fmt: str) -> Frame:
    rng = np.random.default_rng(seed)
    hbo2, hb, _ = make_fields(rng, H, W, nblobs, smin, smax)
    return Frame(render(A, hbo2, hb, rng, noise, fmt), fmt, hbo2, hb)


# ---------------------------------------------------------------------------------------------
# Named workloads.  Sizes, blob counts, noise and grids follow the configurations the method is
# measured on: a small 256x256 float frame, a 1920x1080 8-bit frame, stereo video, a serving mix.
# ---------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    H: int
    W: int
    levels: int
    grid: tuple            # (n0, n1)
    nblobs: int
    smin: float
    smax: float
    noise: float
    fmt: str
    seed: int
    lam: float = 1e-3
    sigma_l: float = 0.02


SMALL_256 = Workload("frame256_f32_l1_g64", 256, 256, 1, (64, 64), 8, 10.0, 40.0, 0.005, "f32", 0)
HD_1080 = Workload("frame1080p_u8_l3_g128", 1080, 1920, 3, (128, 128), 32, 20.0, 120.0, 0.01, "u8", 1)


def workload_inputs(wl: Workload):
    """(mixing, frame) for a named single-frame workload; mixing drawn from the same seed."""
    mix = make_mixing(wl.seed)
    fr = make_frame(wl.seed, wl.H, wl.W, mix.A, wl.nblobs, wl.smin, wl.smax, wl.noise, wl.fmt)
    return mix, fr


def grid_spec(wl: Workload):
    """Grid dictionary: inclusive linspace nodes over the concentration box."""
    return dict(n0=wl.grid[0], n1=wl.grid[1], lo0=BOX_HBO2[0], hi0=BOX_HBO2[1],
                lo1=BOX_HB[0], hi1=BOX_HB[1], sigma_l=wl.sigma_l)


# ---------------------------------------------------------------------------------------------
# Pulsing video (the stand-in for the tongue video of Section 3.2, whose total haemoglobin
# shows the heart rate): static smooth fields whose concentrations, inside a soft tissue patch,
# are scaled by 1 + depth * sin(2 pi f t + phase); every frame adds sensor noise and a small
# global illumination jitter (a per-frame intensity factor), which makes the per-frame THb
# trace noisy the way the paper's trace is.
# ---------------------------------------------------------------------------------------------
@dataclasses.dataclass
class PulseVideo:
    A: np.ndarray
    H: int
    W: int
    fps: float
    f_pulse: float         # Hz
    depth: float           # relative modulation of both concentrations at the patch centre
    phase: float
    hbo2: np.ndarray       # (H, W) static fields, uM
    hb: np.ndarray
    window: np.ndarray     # (H, W) modulation weight in [0, 1]
    noise: float
    jitter: float          # standard deviation of the per-frame intensity factor
    fmt: str
    seed: int
    shift: int = 0         # horizontal disparity of this view, px (stereo pairs)

    def fields(self, k: int):
        """Ground-truth (HbO2, Hb) of frame k."""
        s = 1.0 + self.depth * np.sin(2.0 * np.pi * self.f_pulse * k / self.fps + self.phase) * self.window
        return self.hbo2 * s, self.hb * s

    def frame(self, k: int) -> np.ndarray:
        rng = np.random.default_rng((self.seed, self.shift, k))
        hbo2, hb = self.fields(k)
        att = hbo2[..., None] * self.A[:, 0] + hb[..., None] * self.A[:, 1]
        I = np.exp(-att) * (1.0 + self.jitter * rng.standard_normal())
        if self.noise > 0:
            I = I + rng.normal(0.0, self.noise, I.shape)
        if self.shift:
            I = np.roll(I, self.shift, axis=1)
        if self.fmt == "u8":
            return np.rint(255.0 * np.clip(I, 0.0, 1.0)).astype(np.uint8)
        return I.astype(np.float32)


def pulse_video(seed: int, H: int, W: int, A: np.ndarray, fps: float = 30.0, f_pulse: float = 1.25,
                depth: float = 0.03, nblobs: int = 8, noise: float = 0.01, jitter: float = 0.004,
                fmt: str = "u8", shift: int = 0) -> PulseVideo:
    """A pulsing video (see above).  The blobs are sized to the frame (sigma W/12..W/4) and
    the tissue patch is a Gaussian window at the frame centre with sigma min(H, W) / 4."""
    rng = np.random.default_rng(seed)
    hbo2, hb, _ = make_fields(rng, H, W, nblobs, W / 12.0, W / 4.0)
    # keep clear of the box edges so that the modulation stays inside the prior's support
    hbo2 = 20.0 + 0.7 * hbo2
    hb = 10.0 + 0.7 * hb
    ys = np.arange(H) - (H - 1) / 2.0
    xs = np.arange(W) - (W - 1) / 2.0
    sg = min(H, W) / 4.0
    window = np.outer(np.exp(-0.5 * (ys / sg) ** 2), np.exp(-0.5 * (xs / sg) ** 2))
    phase = float(rng.uniform(0.0, 2.0 * np.pi))
    return PulseVideo(A, H, W, fps, f_pulse, depth, phase, hbo2, hb, window, noise, jitter, fmt, seed, shift)


# ---------------------------------------------------------------------------------------------
# Drifting stereo video (the stand-in for the stereo laparoscope sequences): the 1080p
# generator's blob fields, whose centres move by a seeded velocity per blob (|v| uniform in
# [0, vmax] px per frame, uniform direction); the right view is the same scene shifted by a
# seeded horizontal disparity, with its own sensor noise.  Fields are evaluated as a matrix
# product of the blobs' separable Gaussian factors, in float32, so that a 1920x1080 frame takes
# tens of milliseconds and host threads can render frames ahead of a GPU consumer.
# ---------------------------------------------------------------------------------------------
@dataclasses.dataclass
class DriftVideo:
    A: np.ndarray
    H: int
    W: int
    params: list           # per field: ((cy, cx), sigma, amplitude) of its blobs at frame 0
    vel: np.ndarray        # (2 fields, nblobs, 2): (vy, vx) px per frame
    disparity: float       # px, right view
    noise: float
    fmt: str
    seed: int

    def fields(self, k: int, eye: int = 0):
        ys = np.arange(self.H, dtype=np.float32)[:, None]
        xs = np.arange(self.W, dtype=np.float32)[:, None]
        out = []
        for f, box in enumerate((BOX_HBO2, BOX_HB)):
            (cy, cx), sg, am = self.params[f]
            cyk = (cy + k * self.vel[f, :, 0]).astype(np.float32)
            cxk = (cx + k * self.vel[f, :, 1] + (self.disparity if eye else 0.0)).astype(np.float32)
            s = sg.astype(np.float32)
            gy = np.exp(-0.5 * ((ys - cyk) / s) ** 2) * am.astype(np.float32)   # (H, nblobs)
            gx = np.exp(-0.5 * ((xs - cxk) / s) ** 2)                           # (W, nblobs)
            field = gy @ gx.T
            lo, hi = float(field.min()), float(field.max())
            field = (field - lo) * np.float32(1.0 / (hi - lo if hi > lo else 1.0))
            out.append(np.float32(box[0]) + field * np.float32(box[1] - box[0]))
        return out[0], out[1]

    def frame(self, k: int, eye: int = 0) -> np.ndarray:
        hbo2, hb = self.fields(k, eye)
        A = self.A.astype(np.float32)
        att = hbo2[..., None] * A[:, 0] + hb[..., None] * A[:, 1]
        I = np.exp(-att)
        rng = np.random.default_rng((self.seed, eye, k))
        if self.noise > 0:
            I += rng.standard_normal(I.shape, dtype=np.float32) * np.float32(self.noise)
        if self.fmt == "u8":
            return np.rint(np.float32(255.0) * np.clip(I, 0.0, 1.0)).astype(np.uint8)
        return I


def drift_video(seed: int, H: int, W: int, A: np.ndarray, nblobs: int = 32, smin: float = 20.0,
                smax: float = 120.0, vmax: float = 3.0, noise: float = 0.01, fmt: str = "u8") -> DriftVideo:
    """A drifting stereo video (see above), seeded."""
    rng = np.random.default_rng(seed)
    _, _, params = make_fields(rng, 8, 8, nblobs, smin, smax)   # blob draws only (tiny fields)
    # centres over the full frame (make_fields drew them for an 8x8 frame)
    params = [((rng.uniform(0, H, nblobs), rng.uniform(0, W, nblobs)), sg, am) for (_, sg, am) in params]
    speed = rng.uniform(0.0, vmax, (2, nblobs))
    ang = rng.uniform(0.0, 2.0 * np.pi, (2, nblobs))
    vel = np.stack([speed * np.sin(ang), speed * np.cos(ang)], axis=-1)
    disparity = float(rng.uniform(5.0, 20.0))
    return DriftVideo(A, H, W, params, vel, disparity, noise, fmt, seed)
