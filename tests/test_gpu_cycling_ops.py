"""GPU parity of the cycling companions against the oracle: relaxation of
the analysis to the prior (Sec. IV-A) and the imperfect-model error of the
twin experiment (Sec. IV-A)."""
import numpy as np
import pytest

from oracle import oracle as o

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("mode", ["spread", "perturbations"])
@pytest.mark.parametrize("factor", [0.0, 0.3, 1.0])
def test_relax_spread_matches_oracle(mode, factor):
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    g = np.random.default_rng(21)
    n, d = 20, 3 * 1024 + 5
    prior = (g.standard_normal((n, d)) * g.uniform(0.5, 2.0, d) + 1.0).astype(np.float32)
    z = (g.standard_normal((n, d)) * g.uniform(0.05, 0.3, d) - 0.5).astype(np.float32)
    z[:, 3] = 0.125            # no analysis spread in one variable
    ref = o.relax_spread(prior, z, factor, mode)
    zd = torch.from_numpy(z).cuda()
    ensf.relax_spread(torch.from_numpy(prior).cuda(), zd, factor, mode)
    out = zd.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(out, ref, rtol=2e-6, atol=2e-6)


def test_model_error_matches_oracle():
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    g = np.random.default_rng(22)
    B, d = 6, 4099             # a ragged particle quad and a ragged column tail
    state = g.standard_normal((B, d)).astype(np.float32)
    coef = [0.2 * 0.7, 0.0, 0.4 * 0.7, 0.5 * 0.7]
    ref = o.model_error(state, coef, seed=77, cycle=12)
    sd = torch.from_numpy(state).cuda()
    ensf.model_error(sd, coef, seed=77, cycle=12)
    np.testing.assert_allclose(sd.cpu().numpy().astype(np.float64), ref, rtol=1e-5, atol=1e-5)
    # a 1-D state is one member
    one = torch.from_numpy(state[0].copy()).cuda()
    ensf.model_error(one, coef, seed=77, cycle=12)
    np.testing.assert_allclose(one.cpu().numpy().astype(np.float64), ref[0], rtol=1e-5, atol=1e-5)


def test_model_error_rejects_bad_arguments():
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    s = torch.zeros(2, 16, device="cuda")
    with pytest.raises(ensf.EnsfError):
        ensf.model_error(s, [], seed=1, cycle=0)
    with pytest.raises(ensf.EnsfError):
        ensf.model_error(s, [0.1] * 9, seed=1, cycle=0)
