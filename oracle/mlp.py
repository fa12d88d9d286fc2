"""FP64 reference of the learned low-pass stand-in (test infrastructure only).

Only the tests may import this module.  It restates the network the CUDA library
trains -- 3 -> 64 -> 64 -> 2, exact (erf) GELU, BF16 weights, BF16 rounding of the
hidden activations h1, h2 and of the back-propagated dz2, everything else exact --
and derives its gradient by hand.  With ``exact=True`` all BF16 rounding is skipped,
which is what the finite-difference pins check.

Model (per sample, ybar = block-mean log-attenuation, 3 values):
    x = T ybar + t0
    z1 = W1 x + b1,  h1 = r(gelu(z1))
    z2 = W2 h1 + b2, h2 = r(gelu(z2))
    o  = W3 h2 + b3
    c  = clip(A+ ybar, box) + osc * o
with r() = BF16 rounding.  T maps ybar to its least-squares concentrations, scaled to
[-4, 4] over the box (rows 0, 1), and to its component outside the range of A in
sigma_l units (row 2); osc is the posterior standard deviation per axis,
sigma_l sqrt(((A^T A)^-1)_jj).  Loss: mean over samples and both outputs of
(o - t)^2, t = (c_target - clip(A+ ybar)) / osc.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

N_IN, N_HID, N_OUT = 3, 64, 2
OFF_W1 = 0
OFF_B1 = OFF_W1 + N_HID * N_IN
OFF_W2 = OFF_B1 + N_HID
OFF_B2 = OFF_W2 + N_HID * N_HID
OFF_W3 = OFF_B2 + N_HID
OFF_B3 = OFF_W3 + N_OUT * N_HID
NPARAMS = OFF_B3 + N_OUT


def bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even) through the FP32 value; float64 out."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    bad = ~np.isfinite(f)
    out[bad] = f[bad]
    return out


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def norm_for(A, grid: dict) -> dict:
    """Input transform, least-squares baseline and output scale for a mixing matrix and grid."""
    A = np.asarray(A, dtype=np.float64).reshape(3, 2)
    lo = np.array([grid["lo0"], grid["lo1"]], dtype=np.float64)
    hi = np.array([grid["hi0"] if grid["n0"] > 1 else grid["lo0"], grid["hi1"] if grid["n1"] > 1 else grid["lo1"]])
    P = np.linalg.pinv(A)
    half = np.where(hi > lo, 0.5 * (hi - lo), 1.0)
    centre = 0.5 * (lo + hi)
    n = np.cross(A[:, 0], A[:, 1])
    T = np.vstack([4.0 * P / half[:, None], n / np.linalg.norm(n) / grid["sigma_l"]])
    t0 = np.array([-4.0 * centre[0] / half[0], -4.0 * centre[1] / half[1], 0.0])
    osc = grid["sigma_l"] * np.sqrt(np.diag(np.linalg.inv(A.T @ A)))
    return dict(T=T, t0=t0, Ap=P, lo=lo, hi=hi, osc=osc, ext=np.where(hi > lo, hi - lo, 1.0))


def unpack(params, exact=False):
    p = np.asarray(params, dtype=np.float64)
    if not exact:
        p = bf16(p)
    return dict(W1=p[OFF_W1:OFF_B1].reshape(N_HID, N_IN), b1=p[OFF_B1:OFF_W2], W2=p[OFF_W2:OFF_B2].reshape(N_HID, N_HID),
                b2=p[OFF_B2:OFF_W3], W3=p[OFF_W3:OFF_B3].reshape(N_OUT, N_HID), b3=p[OFF_B3:])


def baseline(nm, ybar):
    return np.clip(np.asarray(ybar, np.float64) @ nm["Ap"].T, nm["lo"], nm["hi"])


def forward(params, nm, ybar, exact=False) -> dict:
    r = (lambda v: v) if exact else bf16
    w = unpack(params, exact)
    x = np.asarray(ybar, np.float64) @ nm["T"].T + nm["t0"]
    z1 = x @ w["W1"].T + w["b1"]
    h1 = r(gelu(z1))
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = r(gelu(z2))
    o = h2 @ w["W3"].T + w["b3"]
    return dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2, o=o, c=baseline(nm, ybar) + nm["osc"] * o)


def loss_and_grad(params, nm, ybar, target, exact=False):
    """Mean loss and its gradient with respect to the (master) parameters."""
    r = (lambda v: v) if exact else bf16
    w = unpack(params, exact)
    f = forward(params, nm, ybar, exact)
    n = f["o"].shape[0]
    t = (np.asarray(target, np.float64) - baseline(nm, ybar)) / nm["osc"]
    e = f["o"] - t
    loss = np.mean(e * e)
    do = 2.0 * e / e.size
    g = np.zeros(NPARAMS)
    g[OFF_W3:OFF_B3] = (do.T @ f["h2"]).reshape(-1)
    g[OFF_B3:] = do.sum(axis=0)
    dz2 = r((do @ w["W3"]) * gelu_grad(f["z2"]))
    g[OFF_W2:OFF_B2] = (dz2.T @ f["h1"]).reshape(-1)
    g[OFF_B2:OFF_W3] = dz2.sum(axis=0)
    dz1 = (dz2 @ w["W2"]) * gelu_grad(f["z1"])
    g[OFF_W1:OFF_B1] = (dz1.T @ f["x"]).reshape(-1)
    g[OFF_B1:OFF_W2] = dz1.sum(axis=0)
    assert n > 0
    return loss, g
