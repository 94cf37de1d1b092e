"""FP64 CPU oracle of the two-level surface quasi-geostrophic (SQG) model.

TEST INFRASTRUCTURE ONLY (the GPU integrator in the CUDA library is checked
against it; nothing in the library imports it).

The model follows the description of the paper's forecast model (Sec. II-B):
a nonlinear Eady model on an f-plane with uniform stratification N and
uniform vertical shear of the mean flow between rigid lids at z = 0 and
z = H, interior potential vorticity zero, so the dynamics are carried by the
potential temperature theta on the two boundaries; doubly periodic,
pseudo-spectral (FFT) space discretisation, fourth-order Runge-Kutta in time
with the 2/3 dealiasing rule, hyperdiffusion treated implicitly.

Units: theta is scaled so that d(psi)/dz = theta on each boundary.  The
interior streamfunction solves psi_xx + psi_yy + (f/N)^2 psi_zz = 0; for a
horizontal wavenumber K, m = (N/f) K and mu = m H:

    psi_0 = (theta_1 - theta_0 cosh mu) / (m sinh mu)
    psi_H = (theta_1 cosh mu - theta_0) / (m sinh mu)

Mean flow U(z) = Lambda (z - H/2) (thermal wind: mean theta gradient
d(theta_bar)/dy = -Lambda).  On each boundary l:

    d theta_l / dt = -(U_l + u_l) d theta_l/dx - v_l d theta_l/dy + Lambda v_l
                     - nu del^8 theta_l,     u = -d psi/dy,  v = d psi/dx.

The hyperdiffusion is applied after each RK4 step as the backward-Euler
factor 1 / (1 + dt nu K^8) (operator splitting); nu is set by an e-folding
time tau_diss at the largest retained wavenumber.

Large-scale sink (a reading: the paper names none, but a flow forced only by
the uniform shear has no statistical equilibrium without one): Newtonian
relaxation -theta / tau_relax on both lids (tau_relax = 0 disables it).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class SQGParams:
    n: int = 128            # grid points per side
    L: float = 20.0         # domain side (units of the deformation radius N H / f)
    H: float = 1.0          # depth between the lids
    N_over_f: float = 1.0   # buoyancy frequency over Coriolis parameter
    shear: float = 1.0      # Lambda = dU/dz
    dt: float = 0.025       # time step
    tau_diss: float = 0.1   # e-folding time of the hyperdiffusion at the cut-off wavenumber
    tau_relax: float = 0.0  # Newtonian relaxation time of theta (0: none)
    diffusion: bool = True
    dealias: bool = True


def wavenumbers(p: SQGParams):
    """kx [n], ky [n//2+1] (rfft layout over the last axis), K, dealias mask."""
    k1 = 2.0 * np.pi / p.L * np.fft.fftfreq(p.n, d=1.0 / p.n)
    kr = 2.0 * np.pi / p.L * np.fft.rfftfreq(p.n, d=1.0 / p.n)
    kx = kr[None, :] * np.ones((p.n, 1))     # x along the last axis
    ky = k1[:, None] * np.ones((1, kr.size))  # y along the first axis
    K = np.sqrt(kx ** 2 + ky ** 2)
    kmax = 2.0 * np.pi / p.L * (p.n // 2)
    keep = (np.abs(kx) < (2.0 / 3.0) * kmax) & (np.abs(ky) < (2.0 / 3.0) * kmax)
    return kx, ky, K, keep


def invert(theta_hat, p: SQGParams):
    """Boundary streamfunctions psi_hat[2] from theta_hat[2] (zero-PV interior)."""
    _, _, K, _ = wavenumbers(p)
    m = p.N_over_f * K
    mu = m * p.H
    psi = np.zeros_like(theta_hat)
    nz = K > 0
    s = np.sinh(mu[nz])
    c = np.cosh(mu[nz])
    t0, t1 = theta_hat[0][nz], theta_hat[1][nz]
    psi[0][nz] = (t1 - t0 * c) / (m[nz] * s)
    psi[1][nz] = (t1 * c - t0) / (m[nz] * s)
    return psi


def tendency(theta_hat, p: SQGParams):
    """d theta_hat / dt without the hyperdiffusion (dealiased)."""
    kx, ky, K, keep = wavenumbers(p)
    psi = invert(theta_hat, p)
    U = (np.array([0.0, p.H]) - 0.5 * p.H) * p.shear
    out = np.zeros_like(theta_hat)
    for lev in range(2):
        th_x = np.fft.irfft2(1j * kx * theta_hat[lev], s=(p.n, p.n))
        th_y = np.fft.irfft2(1j * ky * theta_hat[lev], s=(p.n, p.n))
        u = np.fft.irfft2(-1j * ky * psi[lev], s=(p.n, p.n))
        v = np.fft.irfft2(1j * kx * psi[lev], s=(p.n, p.n))
        rhs = -(U[lev] + u) * th_x - v * th_y + p.shear * v
        r = np.fft.rfft2(rhs)
        if p.dealias:
            r = r * keep
        if p.tau_relax > 0.0:
            r = r - theta_hat[lev] / p.tau_relax
        out[lev] = r
    return out


def diffusion_factor(p: SQGParams):
    _, _, K, _ = wavenumbers(p)
    kmax = 2.0 * np.pi / p.L * (p.n // 2)
    nu = 1.0 / (p.tau_diss * kmax ** 8)
    return 1.0 / (1.0 + p.dt * nu * K ** 8)


def rk4_step(theta_hat, p: SQGParams):
    dt = p.dt
    k1 = tendency(theta_hat, p)
    k2 = tendency(theta_hat + 0.5 * dt * k1, p)
    k3 = tendency(theta_hat + 0.5 * dt * k2, p)
    k4 = tendency(theta_hat + dt * k3, p)
    out = theta_hat + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    if p.diffusion:
        out = out * diffusion_factor(p)
    return out


def to_spectral(theta):
    return np.stack([np.fft.rfft2(theta[0]), np.fft.rfft2(theta[1])])


def to_grid(theta_hat, n):
    return np.stack([np.fft.irfft2(theta_hat[0], s=(n, n)), np.fft.irfft2(theta_hat[1], s=(n, n))])


def run(theta, nsteps: int, p: SQGParams):
    """Integrate grid-point theta [2][n][n] for nsteps RK4 steps (FP64)."""
    th = to_spectral(np.asarray(theta, dtype=np.float64))
    for _ in range(nsteps):
        th = rk4_step(th, p)
    return to_grid(th, p.n)


def eady_growth_rate(K, p: SQGParams):
    """Textbook Eady growth rate for total wavenumber K (e.g. Vallis, Atmospheric
    and Oceanic Fluid Dynamics, Eady problem): with mu = K N H / f,
    sigma = k c_i = (f / N) Lambda sqrt((mu/2 - tanh(mu/2)) (coth(mu/2) - mu/2)),
    maximal (0.31 f Lambda / N) near mu = 1.61; zero where the square root is
    not real (short waves are neutral)."""
    mu = np.asarray(K, dtype=np.float64) * p.N_over_f * p.H
    a = mu / 2.0 - np.tanh(mu / 2.0)
    b = 1.0 / np.tanh(mu / 2.0) - mu / 2.0
    prod = np.where(a * b > 0, a * b, 0.0)
    return p.shear / p.N_over_f * np.sqrt(prod)
