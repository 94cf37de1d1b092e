"""The persistent small-filter path (ENSF_FLAG_PERSISTENT: all K steps in one
cooperative launch with bounded grid barriers) against the oracle, and the
failure-detection self-test of the library's bounded waits."""
import numpy as np
import pytest

from paper_2407_12168_gb300 import inputs
from tests.parity_util import TOL_FP32, compare_members, conditioning, describe, run_oracle

pytestmark = pytest.mark.gpu


def _run(p, noise_buf=None, graph=False, filt=None):
    import torch
    from paper_2407_12168_gb300 import ensf
    f = filt or ensf.Filter(p.n, p.d, gram="fp32", wx="fp32", check_finite=True, persistent=True, graph=graph)
    prior = torch.from_numpy(p.prior).cuda()
    y = torch.from_numpy(p.y).cuda()
    mask = torch.from_numpy(p.mask).cuda() if p.mask is not None else None
    nb = torch.from_numpy(noise_buf).cuda() if noise_buf is not None else None
    stream = torch.cuda.Stream() if graph else None
    if stream is not None:
        with torch.cuda.stream(stream):
            out = f.analysis(prior, y, mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed, noise=nb)
        stream.synchronize()
    else:
        out = f.analysis(prior, y, mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed, noise=nb)
    assert f.status_sync() == 0
    return out.cpu().numpy()


@pytest.mark.parametrize("case", [
    dict(seed=71, n=1, grid=8, K=5, obs_op=0, sigma_obs=0.6),
    dict(seed=72, n=33, grid=36, K=8, obs_op=1, obs_frac=0.5, sigma_obs=0.4),
    dict(seed=77, n=64, grid=32, K=6, obs_op=1, obs_frac=0.5, sigma_obs=0.4),
    dict(seed=73, n=70, grid=44, K=6, obs_op=0, obs_frac=0.25, sigma_obs=0.5),
    dict(seed=74, n=128, grid=24, layers=2, K=6, obs_op=1, obs_frac=0.5, sigma_obs=0.5),
])
def test_persistent_small_cases_match_oracle(case):
    p = inputs.small_case(**case)
    ref = run_oracle(p)
    cond = conditioning(p, ref, prec="fp32")
    rel, tie, bad = compare_members(_run(p), ref, cond, TOL_FP32)
    assert not bad.any(), describe(rel, tie, bad)
    assert tie.sum() <= max(1, p.n // 20), describe(rel, tie, bad)


def test_persistent_plain_64_full():
    """The 2 x 64 x 64 accuracy setup (N = 20, K = 100, identity, sigma 1)."""
    p = inputs.plain_64()
    ref = run_oracle(p)
    cond = conditioning(p, ref, prec="fp32")
    rel, tie, bad = compare_members(_run(p), ref, cond, TOL_FP32)
    assert not bad.any(), describe(rel, tie, bad)
    assert tie.sum() == 0, describe(rel, tie, bad)


def test_persistent_with_noise_buffer_and_in_a_graph():
    import torch
    from paper_2407_12168_gb300 import ensf
    p = inputs.small_case(seed=75, n=20, grid=16, K=5, obs_op=1, obs_frac=0.5, sigma_obs=0.5)
    nb = inputs.noise_buffer(7, p.K, p.n, p.d)
    ref = run_oracle(p, noise_buf=nb)
    rel, tie, bad = compare_members(_run(p, noise_buf=nb), ref, conditioning(p, ref, noise_buf=nb, prec="fp32"),
                                    TOL_FP32)
    assert not bad.any(), describe(rel, tie, bad)
    f = ensf.Filter(p.n, p.d, gram="fp32", wx="fp32", persistent=True, graph=True)
    a = _run(p, graph=True, filt=f)
    b = _run(p, graph=True, filt=f)     # replayed (updated) graph
    c = _run(p)                          # eager
    np.testing.assert_array_equal(a, c)
    np.testing.assert_array_equal(b, c)


def test_bounded_waits_report_timeouts_and_leave_the_context_usable():
    """Failure detection without a fault: an mbarrier wait and a grid barrier
    that can never complete both end with ENSF_ETIMEOUT after their time
    limit; a normal analysis then runs."""
    from paper_2407_12168_gb300 import ensf
    assert ensf.selftest_timeouts() == [ensf.ETIMEOUT, ensf.ETIMEOUT]
    p = inputs.small_case(seed=76, n=8, grid=8, K=3)
    ref = run_oracle(p)
    rel, tie, bad = compare_members(_run(p), ref, np.zeros(p.n), TOL_FP32)
    assert not bad.any(), describe(rel, tie, bad)
