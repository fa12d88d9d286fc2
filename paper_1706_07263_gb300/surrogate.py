"""Training workflow of the learned low-pass stand-in (the kernels live in libhb.so).

The network replaces the grid posterior on the low-pass band; it is trained on pairs
(block-mean log-attenuation -> posterior mean) that the exact posterior kernel
produces on seeded synthetic frames, then certified against the exact posterior over
the whole range of inputs (``Context.mlp_certify``): the pixels where it was not found
within tolerance go to the exact posterior, and at run time the exact posterior stays
its per-frame fallback (see ``Context.set_lowpass_mode``).  Everything here is
orchestration: frames are rendered by ``synth``, every numeric step runs on the GPU
through the C ABI, and parameters are saved as ``.npz`` files.
"""
from __future__ import annotations

import numpy as np

from . import binding, synth


def training_pairs(ctx: binding.Context, frames, device):
    """(ybar [N, 3] float32, conc [N, 2] float32) CUDA tensors from a list of HWC frames."""
    import torch
    hl, wl = ctx.lowpass_shape()
    n = hl * wl
    ys = torch.empty((len(frames) * n, 3), dtype=torch.float32, device=device)
    cs = torch.empty((len(frames) * n, 2), dtype=torch.float32, device=device)
    for k, f in enumerate(frames):
        ft = torch.from_numpy(np.ascontiguousarray(f)).to(device)
        ctx.lowpass_pairs(ft, ys[k * n:(k + 1) * n], cs[k * n:(k + 1) * n])
    torch.cuda.synchronize(device)
    return ys, cs


def workload_frames(wl: synth.Workload, mix: synth.Mixing, count: int, first_seed: int):
    """`count` frames of a workload's generator (same mixing matrix, fields drawn from
    seeds first_seed, first_seed + 1, ...)."""
    return [synth.make_frame(first_seed + k, wl.H, wl.W, mix.A, wl.nblobs, wl.smin, wl.smax, wl.noise, wl.fmt).rgb
            for k in range(count)]


def train(ctx: binding.Context, ybar, conc, steps: int, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
          init_seed: int = 0, init: bool = True):
    """Initialise (optionally) and train; returns the per-step minibatch losses."""
    if init:
        ctx.mlp_init(init_seed)
    return ctx.mlp_train(ybar, conc, steps, batch=batch, lr=lr, seed=seed)


# Learning-rate phases of the default recipe: Adam, batch 4096, 56k steps, the rate halved
# six times from 3e-3.
DEFAULT_PHASES = ((3e-3, 8000), (1.5e-3, 8000), (7.5e-4, 8000), (3.75e-4, 8000), (1.9e-4, 8000), (1e-4, 8000),
                  (5e-5, 8000))


def train_phases(ctx: binding.Context, ybar, conc, phases=DEFAULT_PHASES, batch: int = 4096, seed: int = 0,
                 init_seed: int = 0):
    """Initialise and train through successive (learning rate, steps) phases; Adam's state
    carries over between phases.  Returns the concatenated per-step losses."""
    ctx.mlp_init(init_seed)
    out = [ctx.mlp_train(ybar, conc, steps, batch=batch, lr=lr, seed=seed + 7919 * k)
           for k, (lr, steps) in enumerate(phases)]
    return np.concatenate(out)


def density_resampled(ybar, conc, A, grid: dict, alpha: float = 0.25, cells: int = 48, seed: int = 0):
    """The pairs drawn again (with replacement, as many as there are) with probability
    proportional to count^-alpha of their least-squares point's cell in a cells x cells map
    over the box widened by a tenth: the frames are smooth fields, so the rare regions (the
    corners of the box, where two edges cut the likelihood together) get more of the
    minibatches than their share of the pixels.  alpha = 0 keeps the frames' distribution."""
    import torch
    A = np.asarray(A, dtype=np.float64)
    P = torch.tensor(np.linalg.pinv(A), dtype=torch.float32, device=ybar.device)
    c = ybar @ P.T
    lo = torch.tensor([grid["lo0"], grid["lo1"]], dtype=torch.float32, device=ybar.device)
    hi = torch.tensor([grid["hi0"], grid["hi1"]], dtype=torch.float32, device=ybar.device)
    pad = 0.1 * (hi - lo)
    u = ((c - (lo - pad)) / (hi - lo + 2 * pad) * cells).floor().clamp(0, cells - 1).long()
    cell = u[:, 0] * cells + u[:, 1]
    cnt = torch.bincount(cell, minlength=cells * cells).double()
    w = cnt[cell].pow(-alpha)
    g = torch.Generator(device=ybar.device).manual_seed(seed)
    idx = torch.multinomial(w / w.sum(), ybar.shape[0], replacement=True, generator=g)
    return ybar[idx].contiguous(), conc[idx].contiguous()


def train_certified(ctx: binding.Context, ybar, conc, A, grid: dict, cert_tol: float, alpha: float = 0.25,
                    phases=DEFAULT_PHASES, batch: int = 4096, seed: int = 0, init_seed: int = 0):
    """The default recipe: density-resampled pairs, phased training, then the certification
    of the trained network at cert_tol (hb_mlp_certify).  Returns (losses, trusted share of
    the certification map)."""
    ys, cs = density_resampled(ybar, conc, A, grid, alpha, seed=seed)
    losses = train_phases(ctx, ys, cs, phases=phases, batch=batch, seed=seed, init_seed=init_seed)
    del ys, cs
    return losses, ctx.mlp_certify(cert_tol)


def edge_weighted(ybar, conc, A, grid: dict, sigmas: float = 4.0, repeat: int = 8):
    """Training set with the pairs whose least-squares estimate lies within `sigmas`
    posterior standard deviations of a box edge (or outside the box) repeated `repeat`
    times: frames are smooth, so the edges, where the prior truncates the likelihood
    and the posterior mean departs from the least-squares point, are rare otherwise."""
    import torch
    A = np.asarray(A, dtype=np.float64)
    P = torch.tensor(np.linalg.pinv(A), dtype=torch.float32, device=ybar.device)
    sd = grid["sigma_l"] * np.sqrt(np.diag(np.linalg.inv(A.T @ A)))
    lo = torch.tensor([grid["lo0"], grid["lo1"]], dtype=torch.float32, device=ybar.device)
    hi = torch.tensor([grid["hi0"], grid["hi1"]], dtype=torch.float32, device=ybar.device)
    band = torch.tensor(sigmas * sd, dtype=torch.float32, device=ybar.device)
    ls = ybar @ P.T
    near = ((ls < lo + band) | (ls > hi - band)).any(dim=1)
    idx = torch.nonzero(near).squeeze(1)
    if idx.numel() == 0 or repeat <= 1:
        return ybar, conc
    rep = idx.repeat(repeat - 1)
    return torch.cat([ybar, ybar[rep]]), torch.cat([conc, conc[rep]])


def save(ctx: binding.Context, path: str, **meta):
    np.savez(path, params=ctx.mlp_get_params(), **{k: np.asarray(v) for k, v in meta.items()})


def load(ctx: binding.Context, path: str):
    with np.load(path) as z:
        ctx.mlp_set_params(z["params"])
