"""The constant (illumination) term of Eq. 8 in the FP64 oracle: the Tikhonov operator over
xi = [A | 1], the posterior with the per-pixel offset integrated out, and what the term is
for -- estimates that do not move when the whole frame is lit more or less brightly."""
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1706_07263_gb300 import synth

NTH = os.cpu_count() or 1


def _xi(A):
    return np.hstack([A, np.ones((3, 1))])


@pytest.mark.parametrize("lam,relative", [(1e-3, True), (2e-5, False), (0.1, True)])
def test_operator_is_the_regularised_solve_over_xi(lam, relative):
    A = synth.make_mixing(4).A
    M, g = oracle.tikhonov_operator(A, lam, relative, illumination=True)
    assert g == pytest.approx(lam * np.trace(A.T @ A) / 2 if relative else lam)
    xi = _xi(A)
    ref = np.linalg.solve(xi.T @ xi + g * np.eye(3), xi.T)[:2]
    np.testing.assert_allclose(M, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_unregularised_operator_inverts_xi():
    """With gamma = 0, M xi = the first two rows of I: a constant offset maps to zero
    concentration and A c maps back to c."""
    A = synth.make_mixing(5).A
    M, _ = oracle.tikhonov_operator(A, 0.0, False, illumination=True)
    np.testing.assert_allclose(M @ np.ones(3), 0.0, atol=1e-9 * np.abs(M).max())
    np.testing.assert_allclose(M @ A, np.eye(2), atol=1e-9)


def test_posterior_integrates_the_offset_out():
    """Posterior mean with the offset kappa integrated numerically over the real line under a
    flat prior, node by node, on a 5 x 7 grid."""
    A = synth.make_mixing(6).A
    grid = dict(n0=5, n1=7, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.05)
    g0 = np.linspace(0, 150, 5)
    g1 = np.linspace(0, 100, 7)
    rng = np.random.default_rng(3)
    for _ in range(3):
        c = np.array([rng.uniform(20, 130), rng.uniform(10, 90)])
        yb = A @ c + rng.uniform(-0.5, 0.5) + rng.normal(0, 0.02, 3)
        like = np.empty((5, 7))
        for i, a in enumerate(g0):
            for j, b in enumerate(g1):
                r = yb - A @ np.array([a, b])
                like[i, j] = integrate.quad(lambda k: np.exp(-np.sum((r - k) ** 2) / (2 * 0.05 ** 2)),
                                            r.mean() - 1, r.mean() + 1, epsabs=0, epsrel=1e-12)[0]
        ref = np.array([(like * g0[:, None]).sum(), (like * g1[None, :]).sum()]) / like.sum()
        got = oracle.posterior_mean(yb, A, grid, illumination=True)
        np.testing.assert_allclose(got, ref, rtol=1e-8)


@pytest.mark.parametrize("s", [0.6, 1.25])
def test_estimate_does_not_move_with_global_illumination(s):
    A = synth.make_mixing(7).A
    fr = synth.make_frame(7, 24, 40, A, 4, 3.0, 10.0, 0.0, "f32").rgb
    grid = dict(n0=32, n1=32, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)
    base = oracle.estimate(fr, A, grid, 2, 1e-3, illumination=True, nthreads=NTH)
    lit = oracle.estimate((fr * s).astype(np.float32), A, grid, 2, 1e-3, illumination=True, nthreads=NTH)
    # float32 rounding of the scaled intensities is the only difference (|d log I| <= 6e-8)
    np.testing.assert_allclose(lit["thb"], base["thb"], rtol=1e-4, atol=1e-3)
    plain = oracle.estimate(fr, A, grid, 2, 1e-3, nthreads=NTH)
    plain_lit = oracle.estimate((fr * s).astype(np.float32), A, grid, 2, 1e-3, nthreads=NTH)
    assert np.abs(plain_lit["thb"] - plain["thb"]).max() > 1.0


def test_noiseless_patch_under_an_offset_recovers_its_node():
    A = synth.make_mixing(1).A
    n0, n1 = 31, 21
    c_star = np.array([np.linspace(0, 150, n0)[12], np.linspace(0, 100, n1)[7]])
    I = np.exp(-(A @ c_star + 0.4)).astype(np.float64)
    frame = np.broadcast_to(I, (16, 16, 3)).astype(np.float32)
    P = np.eye(3) - 1.0 / 3.0
    spacing = np.linalg.norm(P @ A @ np.array([150 / 30, 0.0]))
    grid = dict(n0=n0, n1=n1, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.25 * spacing)
    out = oracle.estimate(frame, A, grid, 2, 1e-3, illumination=True)
    np.testing.assert_allclose(out["hbo2"], c_star[0], atol=1e-3)
    np.testing.assert_allclose(out["hb"], c_star[1], atol=1e-3)
