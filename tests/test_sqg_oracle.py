"""Pins of the FP64 SQG oracle: the textbook Eady growth rate, conservation
of boundary theta variance by the nonlinear advection, and analytic spectral
derivatives."""
import numpy as np
import pytest

from oracle import sqg_oracle as sq


def test_eady_growth_rate_matches_textbook():
    """A single small-amplitude mode grows at the analytic Eady rate."""
    p = sq.SQGParams(n=24, L=20.0, dt=0.02, diffusion=False)  # 2/3 rule keeps |index| < 8
    for idx in [3, 5, 7]:
        Kmode = 2 * np.pi / p.L * idx
        x = np.arange(p.n) * p.L / p.n
        X = np.broadcast_to(x[None, :], (p.n, p.n))
        theta = 1e-9 * np.stack([np.cos(Kmode * X), 0.3 * np.sin(Kmode * X)])
        # the decaying normal mode has the same (zero) phase speed: wait until
        # it has died out (t = 30), then measure over t = 30 .. 40
        out = sq.run(theta, 1500, p)
        a1 = np.abs(np.fft.rfft2(out[0]))[0, idx]
        out2 = sq.run(out, 500, p)
        a2 = np.abs(np.fft.rfft2(out2[0]))[0, idx]
        sigma = np.log(a2 / a1) / (500 * p.dt)
        assert sigma == pytest.approx(sq.eady_growth_rate(Kmode, p), rel=2e-3, abs=2e-4)


def test_linear_eady_neutral_short_waves():
    """Waves shorter than the Eady cut-off (mu > 2.399) do not grow."""
    p = sq.SQGParams(n=32, L=20.0, dt=0.01, diffusion=False)
    idx = 10  # mu = 3.14
    Kmode = 2 * np.pi / p.L * idx
    assert sq.eady_growth_rate(Kmode, p) == 0.0
    x = np.arange(p.n) * p.L / p.n
    X = np.broadcast_to(x[None, :], (p.n, p.n))
    theta = 1e-7 * np.stack([np.cos(Kmode * X), np.sin(Kmode * X)])
    out = sq.run(theta, 300, p)
    assert np.abs(out).max() < 2.0 * np.abs(theta).max()


def test_theta_variance_conserved_without_shear_and_diffusion():
    """With Lambda = 0 and no diffusion the dealiased advection conserves the
    theta variance of each boundary (the Jacobian integrates to zero against
    theta); RK4 leaves a tiny error."""
    p = sq.SQGParams(n=32, L=20.0, dt=0.005, shear=0.0, diffusion=False)
    g = np.random.default_rng(0)
    th = sq.to_spectral(g.standard_normal((2, p.n, p.n)))
    _, _, _, keep = sq.wavenumbers(p)
    th = th * keep  # start inside the dealiased band
    v0 = [np.sum(np.abs(sq.to_grid(th, p.n)[lev]) ** 2) for lev in range(2)]
    for _ in range(20):
        th = sq.rk4_step(th, p)
    v1 = [np.sum(np.abs(sq.to_grid(th, p.n)[lev]) ** 2) for lev in range(2)]
    for a, b in zip(v0, v1):
        assert b == pytest.approx(a, rel=1e-6)
    # ... and the shear makes it grow (baroclinic instability feeds it)
    p2 = sq.SQGParams(n=32, L=20.0, dt=0.01, diffusion=False)
    th2 = th.copy()
    for _ in range(200):
        th2 = sq.rk4_step(th2, p2)
    assert np.sum(sq.to_grid(th2, p.n) ** 2) > 1.05 * sum(v1)


def test_spectral_derivatives_and_jacobian_analytic():
    """psi = sin(a x) cos(b y), theta = cos(c x): the pseudo-spectral
    advection term equals the analytic one."""
    p = sq.SQGParams(n=32, L=2 * np.pi, shear=0.0, diffusion=False, dealias=False)
    x = np.arange(p.n) * p.L / p.n
    Y, X = np.meshgrid(x, x, indexing="ij")
    theta = np.stack([np.cos(2 * X) * np.sin(Y), np.cos(3 * Y)])
    th = sq.to_spectral(theta)
    kx, ky, K, _ = sq.wavenumbers(p)
    dx = sq.to_grid(np.stack([1j * kx * th[0], 1j * kx * th[1]]), p.n)
    dy = sq.to_grid(np.stack([1j * ky * th[0], 1j * ky * th[1]]), p.n)
    np.testing.assert_allclose(dx[0], -2 * np.sin(2 * X) * np.sin(Y), atol=1e-12)
    np.testing.assert_allclose(dy[0], np.cos(2 * X) * np.cos(Y), atol=1e-12)
    np.testing.assert_allclose(dy[1], -3 * np.sin(3 * Y), atol=1e-12)
    # inversion of a single mode against the closed form
    psi = sq.invert(th, p)
    Km = np.sqrt(5.0)
    c, s = np.cosh(Km), np.sinh(Km)
    g0 = sq.to_grid(np.stack([th[0], np.zeros_like(th[0])]), p.n)
    psi0 = sq.to_grid(sq.invert(np.stack([th[0], np.zeros_like(th[0])]), p), p.n)
    np.testing.assert_allclose(psi0[0], -c / (Km * s) * g0[0], atol=1e-12)
    np.testing.assert_allclose(psi0[1], -1.0 / (Km * s) * g0[0], atol=1e-12)


def test_relaxation_decay_rate():
    """Without shear the relaxation alone damps a mode at rate 1/tau_relax
    (single mode: the advection term vanishes)."""
    p = sq.SQGParams(n=16, L=20.0, dt=0.02, shear=0.0, diffusion=False, tau_relax=5.0)
    x = np.arange(p.n) * p.L / p.n
    X = np.broadcast_to(x[None, :], (p.n, p.n))
    theta = np.stack([np.cos(2 * np.pi / p.L * 2 * X), np.zeros((p.n, p.n))])
    out = sq.run(theta, 250, p)
    ratio = np.abs(out[0]).max() / np.abs(theta[0]).max()
    assert ratio == pytest.approx(np.exp(-250 * p.dt / p.tau_relax), rel=1e-6)


def test_spectral_transform_matches_naive_dft():
    """The oracle's grid <-> spectral transforms against a naive DFT on 8 x 8."""
    g = np.random.default_rng(3)
    th = g.standard_normal((2, 8, 8))
    spec = sq.to_spectral(th)
    j = np.arange(8)
    W = np.exp(-2j * np.pi * np.outer(j, j) / 8)
    for lev in range(2):
        naive = W @ th[lev] @ W.T          # sum over y, x of theta e^{-2 pi i (k_y y + k_x x)/8}
        np.testing.assert_allclose(spec[lev], naive[:, :5], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(sq.to_grid(spec, 8), th, rtol=1e-12, atol=1e-12)
