"""The TMA-staged W X epilogue (particles moved through shared memory by TMA,
noise evaluated in the epilogue) against the epilogue that reads and writes
the particles with per-thread global accesses: the same arithmetic, so whole
analyses must agree bit for bit -- on ragged shapes (N not a multiple of the
16-particle chunk or of the tile, d not a multiple of the 128-column tile),
for every particle-plane layout the next Gram may need (BF16 hi + lo for
the split Gram, hi only for the BF16 Gram, none for a CUDA-core Gram) and
every W X tile width -- and match the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as o
from paper_2407_12168_gb300 import inputs

from .parity_util import compare_members, conditioning, describe, run_oracle

pytestmark = pytest.mark.gpu

CASES = [
    # (seed, n, grid, layers, K, obs_op, obs_frac, sigma)
    (71, 70, 44, 1, 6, 1, 0.6, 0.4),     # n: 4 chunks + a ragged 6; d = 1936: a ragged 128-column tile
    (72, 256, 32, 2, 5, 0, 1.0, 0.6),    # whole 256-particle tiles
    (73, 300, 20, 2, 4, 1, 0.5, 0.4),    # a second, ragged particle tile; d = 800
    (74, 33, 64, 2, 5, 1, 0.25, 0.3),    # n = 33, d = 8192
]


def _run(p, gram, wx, unstaged, wx_tile=0):
    import torch
    from paper_2407_12168_gb300 import ensf
    f = ensf.Filter(p.n, p.d, gram=gram, wx=wx, inline_noise=True, wx_unstaged=unstaged, check_finite=True)
    if wx_tile and gram != "fp32":
        f.set_tuning(p.n, p.d, 128 if p.n <= 128 else 256, 3 if p.n <= 128 else 2, wx_tile_n=wx_tile,
                     noise_inline=1)
    out = f.analysis(torch.from_numpy(p.prior).cuda(), torch.from_numpy(p.y).cuda(),
                     None if p.mask is None else torch.from_numpy(p.mask).cuda(), p.sigma_obs, p.K, p.eps,
                     p.obs_op, seed=p.seed, offset=p.offset)
    assert f.status_sync() == 0
    return out.cpu().numpy()


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("gram", ["split", "bf16", "fp32"])
def test_staged_epilogue_is_bitwise_the_unstaged_one(case, gram):
    seed, n, grid, layers, K, obs_op, frac, sigma = case
    p = inputs.small_case(seed=seed, n=n, grid=grid, layers=layers, K=K, obs_op=obs_op, obs_frac=frac,
                          sigma_obs=sigma)
    a = _run(p, gram, "bf16", unstaged=False)
    b = _run(p, gram, "bf16", unstaged=True)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("wx_tile", [64, 128, 256])
def test_staged_epilogue_tile_widths(wx_tile):
    p = inputs.small_case(seed=75, n=140, grid=36, layers=2, K=4, obs_op=1, obs_frac=0.5, sigma_obs=0.4)
    a = _run(p, "split", "bf16", unstaged=False, wx_tile=wx_tile)
    b = _run(p, "split", "bf16", unstaged=True, wx_tile=wx_tile)
    assert np.array_equal(a, b)


def test_staged_epilogue_matches_oracle():
    p = inputs.small_case(seed=76, n=70, grid=44, layers=1, K=10, obs_op=1, obs_frac=0.6, sigma_obs=0.4)
    ref = run_oracle(p)
    got = _run(p, "split", "bf16", unstaged=False)
    cond = conditioning(p, ref, prec="bf16")
    rel, tie, bad = compare_members(got, ref, cond, 1e-2)
    assert not bad.any(), describe(rel, tie, bad)
    # near-tie members (their oracle result moves under log-kernel errors of
    # the BF16 path's size) are counted, bounded at a few per cent as in the
    # other parity tests, and never dropped from the RMSE check below
    assert tie.sum() <= max(1, p.n // 20), describe(rel, tie, bad)
    _, r_ref = o.mean_rmse(ref, p.truth)
    _, r_got = o.mean_rmse(got, p.truth)
    assert r_got == pytest.approx(r_ref, rel=1e-2)


def test_batched_staged_epilogue_is_bitwise_the_unstaged_one():
    """The batched W X of many uneven filters with the TMA-staged epilogue
    (per-filter staging maps in the device table) against the batched
    per-thread epilogue: bitwise, for every filter, BF16 and split Gram."""
    import torch
    from paper_2407_12168_gb300 import ensf
    cases = [(91, 33, 36, 1, 1, 0.5, 0.4), (92, 130, 32, 2, 0, 1.0, 0.6), (93, 64, 44, 1, 1, 0.25, 0.3),
             (94, 200, 20, 2, 1, 0.6, 0.4), (95, 16, 64, 2, 0, 0.5, 1.0)]
    probs = [inputs.small_case(seed=c[0], n=c[1], grid=c[2], layers=c[3], K=5, obs_op=c[4], obs_frac=c[5],
                               sigma_obs=c[6]) for c in cases]
    for gram in ("split", "bf16"):
        outs = []
        for unstaged in (False, True):
            f = ensf.Filter(256, 8192, gram=gram, wx="bf16", wx_unstaged=unstaged)
            filters = [dict(prior=torch.from_numpy(p.prior).cuda(), y=torch.from_numpy(p.y).cuda(),
                            mask=torch.from_numpy(p.mask).cuda() if p.mask is not None else None,
                            sigma_obs=p.sigma_obs, obs_op=p.obs_op, seed=p.seed) for p in probs]
            outs.append([o.cpu().numpy() for o in f.analysis_batched(filters, 5, 0.05)])
            assert f.status_sync() == 0
        for a, b in zip(*outs):
            assert np.array_equal(a, b)
