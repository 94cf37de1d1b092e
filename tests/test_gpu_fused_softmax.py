"""The row softmax fused into the pair Gram's epilogue (last-arriver counters,
no waits) against the separate tiled softmax launch: the same arithmetic in
the same order, so whole analyses agree bit for bit -- over several 128-row
bands and 256-column tiles, split counts from one to many, both noise
placements -- and the fused form launches no softmax kernel."""
import numpy as np
import pytest

from oracle import oracle as o
from paper_2407_12168_gb300 import inputs

from .parity_util import compare_members, conditioning, describe, run_oracle

pytestmark = pytest.mark.gpu


def _run(p, fused, splits, noise_inline=0, repeat=1):
    import torch
    from paper_2407_12168_gb300 import ensf
    f = ensf.Filter(p.n, p.d, gram="split", wx="bf16", check_finite=True)
    f.set_tuning(p.n, p.d, 256, 3, gram_splits=splits, gram_cta_pair=1, wx_tile_n=256, noise_inline=noise_inline,
                 gram_fused_softmax=1 if fused else 0)
    args = (torch.from_numpy(p.prior).cuda(), torch.from_numpy(p.y).cuda(),
            None if p.mask is None else torch.from_numpy(p.mask).cuda(), p.sigma_obs, p.K, p.eps, p.obs_op)
    f.profile_enable(True)
    outs = [f.analysis(*args, seed=p.seed, offset=p.offset).cpu().numpy() for _ in range(repeat)]
    prof = f.profile_read()
    f.profile_enable(False)
    assert f.status_sync() == 0
    return outs, prof


@pytest.mark.parametrize("n,splits", [(256, 1), (512, 3), (512, 8), (768, 16)])
@pytest.mark.parametrize("noise_inline", [0, 1])
def test_fused_softmax_is_bitwise_the_separate_launch(n, splits, noise_inline):
    p = inputs.small_case(seed=81 + n, n=n, grid=32, layers=2, K=4, obs_op=1, obs_frac=0.5, sigma_obs=0.4)
    (a,), pa = _run(p, False, splits, noise_inline)
    (b, b2), pb = _run(p, True, splits, noise_inline, repeat=2)
    assert np.array_equal(a, b)
    assert np.array_equal(b, b2)   # deterministic, whatever order the CTAs arrive in
    assert pa["softmax_rows"][0] == 4 and "softmax_rows" not in pb


def test_fused_softmax_matches_oracle():
    p = inputs.small_case(seed=85, n=512, grid=32, layers=2, K=8, obs_op=0, obs_frac=1.0, sigma_obs=0.8)
    ref = run_oracle(p)
    (got,), _ = _run(p, True, 4)
    cond = conditioning(p, ref, prec="bf16")
    rel, tie, bad = compare_members(got.astype(np.float64), ref, cond, 1e-2)
    assert not bad.any(), describe(rel, tie, bad)
    assert tie.sum() <= max(1, p.n // 20), describe(rel, tie, bad)
    _, r_ref = o.mean_rmse(ref, p.truth)
    _, r_got = o.mean_rmse(got, p.truth)
    assert r_got == pytest.approx(r_ref, rel=1e-2)
