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
    c  = b(ybar) + osc * o
with r() = BF16 rounding.  T maps ybar to its least-squares concentrations, scaled to
[-4, 4] over the box (rows 0, 1), and to its component outside the range of A in
sigma_l units (row 2); osc is the posterior standard deviation per axis,
sigma_l sqrt(((A^T A)^-1)_jj).  Loss: mean over samples and both outputs of
(o - t)^2, t = (c_target - b(ybar)) / osc.

Baseline b (the network learns what it leaves over).  Without the box the posterior of
a flat prior is the Gaussian N(c_ls, S), c_ls = A+ ybar, S = sigma_l^2 (A^T A)^-1.  Cut
by one edge e of the box -- the half plane n_e . c >= p_e, n_e a signed unit axis -- its
mean moves to c_ls + S n_e lambda(d_e) / s_e with s_e = sqrt(n_e^T S n_e), the distance
d_e = (n_e . c_ls - p_e) / s_e (positive inside) and lambda(d) = phi(d) / Phi(d) (the
inverse Mills ratio of the normal distribution, written sqrt(2 / pi) / erfcx(-d / sqrt 2)
so that it stays finite on both sides).  b adds these shifts of the four edges to c_ls:
exact for a pixel near one edge of a continuous box, it leaves the network the corners,
where two edges act together, and the grid's discreteness.  It is smooth, where the
clipped least-squares point has a kink at every edge.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf, erfcx

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
    S = grid["sigma_l"] ** 2 * np.linalg.inv(A.T @ A)
    osc = np.sqrt(np.diag(S))
    # the four edges: (axis, sign of n_e, position p_e in n_e units)
    edges = [(0, 1.0, lo[0]), (0, -1.0, -hi[0]), (1, 1.0, lo[1]), (1, -1.0, -hi[1])]
    return dict(T=T, t0=t0, Ap=P, lo=lo, hi=hi, osc=osc, ext=np.where(hi > lo, hi - lo, 1.0), S=S, edges=edges)


def mills(d):
    """phi(d) / Phi(d) for the standard normal distribution, finite for every real d."""
    return np.sqrt(2.0 / np.pi) / erfcx(-np.asarray(d, np.float64) / np.sqrt(2.0))


def unpack(params, exact=False):
    p = np.asarray(params, dtype=np.float64)
    if not exact:
        p = bf16(p)
    return dict(W1=p[OFF_W1:OFF_B1].reshape(N_HID, N_IN), b1=p[OFF_B1:OFF_W2], W2=p[OFF_W2:OFF_B2].reshape(N_HID, N_HID),
                b2=p[OFF_B2:OFF_W3], W3=p[OFF_W3:OFF_B3].reshape(N_OUT, N_HID), b3=p[OFF_B3:])


def baseline(nm, ybar):
    """c_ls plus the mean shift of each edge's one-sided truncation (see the module notes)."""
    c = np.asarray(ybar, np.float64) @ nm["Ap"].T
    b = c.copy()
    for axis, sign, pos in nm["edges"]:
        s = nm["osc"][axis]
        d = (sign * c[..., axis] - pos) / s
        b += mills(d)[..., None] * (sign * nm["S"][:, axis] / s)
    return b


def forward(params, nm, ybar, exact=False, override=None) -> dict:
    """The network's pass over the rows of ybar.  override = (site, unit, value): the rounded
    activation of one site ("h1" or "h2") of unit `unit` takes `value` in every row (used
    with a single row, by the rounding envelopes below)."""
    r = (lambda v: v) if exact else bf16
    w = unpack(params, exact)
    x = np.asarray(ybar, np.float64) @ nm["T"].T + nm["t0"]
    z1 = x @ w["W1"].T + w["b1"]
    h1 = r(gelu(z1))
    if override and override[0] == "h1":
        h1[:, override[1]] = override[2]
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = r(gelu(z2))
    if override and override[0] == "h2":
        h2[:, override[1]] = override[2]
    o = h2 @ w["W3"].T + w["b3"]
    return dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2, o=o, c=baseline(nm, ybar) + nm["osc"] * o)


def _loss_grad(params, nm, ybar, target, exact=False, override=None, n_total=None):
    """Loss sum and gradient of the given rows, normalised as a mean over n_total samples;
    override as in forward, or ("dz2", unit, value) for the rounded back-propagated dz2."""
    r = (lambda v: v) if exact else bf16
    w = unpack(params, exact)
    f = forward(params, nm, ybar, exact, override if override and override[0] != "dz2" else None)
    n = n_total or f["o"].shape[0]
    t = (np.asarray(target, np.float64) - baseline(nm, ybar)) / nm["osc"]
    e = f["o"] - t
    do = 2.0 * e / (n * N_OUT)
    g = np.zeros(NPARAMS)
    g[OFF_W3:OFF_B3] = (do.T @ f["h2"]).reshape(-1)
    g[OFF_B3:] = do.sum(axis=0)
    dz2 = r((do @ w["W3"]) * gelu_grad(f["z2"]))
    if override and override[0] == "dz2":
        dz2[:, override[1]] = override[2]
    g[OFF_W2:OFF_B2] = (dz2.T @ f["h1"]).reshape(-1)
    g[OFF_B2:OFF_W3] = dz2.sum(axis=0)
    dz1 = (dz2 @ w["W2"]) * gelu_grad(f["z1"])
    g[OFF_W1:OFF_B1] = (dz1.T @ f["x"]).reshape(-1)
    g[OFF_B1:OFF_W2] = dz1.sum(axis=0)
    return float(np.sum(e * e)), g, dict(f=f, do=do, dz2=dz2, dz1=dz1)


def loss_and_grad(params, nm, ybar, target, exact=False):
    """Mean loss and its gradient with respect to the (master) parameters."""
    n = np.asarray(ybar).shape[0]
    assert n > 0
    lsum, g, _ = _loss_grad(params, nm, ybar, target, exact)
    return lsum / (n * N_OUT), g


# ---- rounding envelopes -----------------------------------------------------------------
# The CUDA kernels compute every pre-rounding value in FP32, this reference in FP64; where a
# value lies within a hair of the midpoint between two BF16 numbers the two may round it to
# different neighbours ("flips").  The envelopes bound what such flips can do: every
# rounding whose FP64 value is within `rel` (relative) of a midpoint is rounded the other
# way on its own, in its own sample, and the absolute changes of the result are added up.

def bf16_other(v):
    """The BF16 neighbour of v that bf16(v) did not round to, and the midpoint between them."""
    f = np.asarray(v, dtype=np.float32)
    u = f.view(np.uint32)
    lo = (u & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)        # towards zero
    hi = ((u & np.uint32(0xFFFF0000)) + np.uint32(0x10000)).view(np.float32).astype(np.float64)
    r = bf16(v)
    return np.where(r == lo, hi, lo), 0.5 * (lo + hi)


def _ambiguous(v, rel):
    other, mid = bf16_other(v)
    return np.abs(np.asarray(v, np.float64) - mid) <= rel * np.abs(v), other


def forward_envelope(params, nm, ybar, rel=2.0 ** -14):
    """(c, envelope): the network's output and, per sample and axis, the sum of |change of c|
    over the ambiguous roundings of h1 and h2 of that sample."""
    f = forward(params, nm, ybar)
    env = np.zeros_like(f["c"])
    for site, z in (("h1", f["z1"]), ("h2", f["z2"])):
        amb, other = _ambiguous(gelu(z), rel)
        for s, u in zip(*np.nonzero(amb)):
            alt = forward(params, nm, ybar[s:s + 1], override=(site, u, other[s, u]))["c"][0]
            env[s] += np.abs(alt - f["c"][s])
    return f["c"], env


def gradient_envelope(params, nm, ybar, target, rel=2.0 ** -14):
    """(loss, g, envelope, l1): the mean loss and gradient, the per-parameter sum of |change
    of g| over the ambiguous roundings of h1, h2 and dz2 (each flipped alone in its sample),
    and the per-parameter sum of the absolute per-sample terms (the scale of FP32
    accumulation errors)."""
    ybar = np.asarray(ybar, np.float64)
    target = np.asarray(target, np.float64)
    n = ybar.shape[0]
    loss, g = loss_and_grad(params, nm, ybar, target)
    env = np.zeros(NPARAMS)
    l1 = np.zeros(NPARAMS)
    w = unpack(params)
    for s in range(n):
        ys, ts = ybar[s:s + 1], target[s:s + 1]
        _, gs, aux = _loss_grad(params, nm, ys, ts, n_total=n)
        f = aux["f"]
        # absolute per-sample terms of every entry
        l1[OFF_W3:OFF_B3] += (np.abs(aux["do"]).T @ np.abs(f["h2"])).reshape(-1)
        l1[OFF_B3:] += np.abs(aux["do"][0])
        l1[OFF_W2:OFF_B2] += (np.abs(aux["dz2"]).T @ np.abs(f["h1"])).reshape(-1)
        l1[OFF_B2:OFF_W3] += np.abs(aux["dz2"][0])
        l1[OFF_W1:OFF_B1] += (np.abs(aux["dz1"]).T @ np.abs(f["x"])).reshape(-1)
        l1[OFF_B1:OFF_W2] += np.abs(aux["dz1"][0])
        dz2_pre = (aux["do"] @ w["W3"]) * gelu_grad(f["z2"])
        for site, v in (("h1", gelu(f["z1"])), ("h2", gelu(f["z2"])), ("dz2", dz2_pre)):
            amb, other = _ambiguous(v, rel)
            for u in np.nonzero(amb[0])[0]:
                _, ga, _ = _loss_grad(params, nm, ys, ts, override=(site, u, other[0, u]), n_total=n)
                env += np.abs(ga - gs)
    return loss, g, env, l1
