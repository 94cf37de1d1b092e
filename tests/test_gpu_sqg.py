"""The GPU SQG integrator against the FP64 SQG oracle (Sec. II-B forecast model)."""
import numpy as np
import pytest

from oracle import sqg_oracle as sq

pytestmark = pytest.mark.gpu


def _band_limited(g, batch, n, L, amp=1.0):
    """Random theta [batch][2][n][n] inside the 2/3-dealiased band, smooth."""
    p = sq.SQGParams(n=n, L=L)
    kx, ky, K, keep = sq.wavenumbers(p)
    out = np.empty((batch, 2, n, n))
    for b in range(batch):
        for lev in range(2):
            spec = np.fft.rfft2(g.standard_normal((n, n))) * keep * np.exp(-(K / (0.3 * K.max())) ** 2)
            f = np.fft.irfft2(spec, s=(n, n))
            out[b, lev] = amp * f / f.std()
    return out


@pytest.mark.parametrize("diffusion,relax", [(False, 0.0), (True, 0.0), (True, 10.0)])
def test_sqg_gpu_matches_oracle(diffusion, relax):
    import torch
    from paper_2407_12168_gb300 import ensf
    n, L, B, steps = 64, 20.0, 3, 40
    g = np.random.default_rng(5)
    theta0 = _band_limited(g, B, n, L)
    sim = ensf.SQG(B, n=n, L=L, dt=0.025, tau_diss=0.1, diffusion=diffusion, tau_relax=relax)
    th = torch.from_numpy(theta0.astype(np.float32)).cuda()
    sim.run(th, steps)
    got = th.cpu().numpy()
    p = sq.SQGParams(n=n, L=L, dt=0.025, tau_diss=0.1, diffusion=diffusion, tau_relax=relax)
    for b in range(B):
        ref = sq.run(theta0[b].astype(np.float32).astype(np.float64), steps, p)
        rel = np.linalg.norm(got[b] - ref) / np.linalg.norm(ref)
        assert rel < 2e-5, rel


def test_sqg_gpu_long_run_stays_bounded():
    """A long spin-up from small noise develops turbulence (theta grows by
    baroclinic instability); hyperdiffusion and relaxation keep it bounded."""
    import torch
    from paper_2407_12168_gb300 import ensf
    n, L = 64, 20.0
    g = np.random.default_rng(6)
    th = torch.from_numpy((0.1 * _band_limited(g, 2, n, L)).astype(np.float32)).cuda()
    sim = ensf.SQG(2, n=n, L=L, dt=0.025, tau_diss=0.1, tau_relax=5.0)
    rms = []
    for _ in range(16):
        sim.run(th, 1000)
        rms.append(float(th.pow(2).mean().sqrt()))
    assert np.all(np.isfinite(rms))
    assert rms[-1] > 2 * 0.1
    assert rms[-1] < 10.0
    # statistical equilibrium: the last third varies by less than a factor 2
    assert max(rms[-4:]) < 2.0 * min(rms[-4:])
