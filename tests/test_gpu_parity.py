"""GPU parity: the CUDA path, called through the C ABI, against the FP64 CPU
oracle on the same seeded inputs, element by element (tolerances and the
near-tie clause are documented in parity_util)."""
import os

import numpy as np
import pytest

from oracle import oracle as o
from paper_2407_12168_gb300 import inputs
from tests.parity_util import TOL_BF16, TOL_FP32, compare_members, conditioning, describe, eps_path, run_oracle

pytestmark = pytest.mark.gpu

PATHS = {
    # name: (gram, wx, tolerance)
    "fp32": ("fp32", "fp32", TOL_FP32),
    "split": ("split", "split", TOL_FP32),
    "split-bf16": ("split", "bf16", TOL_BF16),
    # the TF32 Gram (kind::tf32 on FP32 centred operands) with the split W X:
    # TF32 keeps 10 mantissa bits, so it is held to the BF16-level tolerance
    "tf32": ("tf32", "split", TOL_BF16),
}


def _cond_prec(gram: str, wx: str) -> str:
    """Accuracy level of the path for the near-tie check: a BF16 W X feeds
    2^-9-level errors into the particles and from there into the logits."""
    return "bf16" if "bf16" in (gram, wx) else gram


def _torch():
    import torch
    return torch


def _gpu_analysis(p, gram="fp32", wx="fp32", noise_buf=None, filt=None):
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    f = filt or ensf.Filter(p.n, p.d, gram=gram, wx=wx, check_finite=True)
    prior = torch.from_numpy(p.prior).cuda()
    y = torch.from_numpy(p.y).cuda()
    mask = torch.from_numpy(p.mask).cuda() if p.mask is not None else None
    nb = torch.from_numpy(noise_buf).cuda() if noise_buf is not None else None
    out = f.analysis(prior, y, mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed, offset=p.offset, noise=nb)
    assert f.status_sync() == 0
    return out.cpu().numpy()


# ------------------------------------------------------------------ noise ---
def test_philox_stream_matches_oracle():
    from paper_2407_12168_gb300 import ensf
    seed, offset = 0x1234_5678_9ABC_DEF0, 7
    out = ensf.philox_normal(seed, offset, k0=3, count=2, n=3, d=1000).cpu().numpy()
    for kk in range(2):
        for i in range(3):
            ref = o.noise(seed, offset, 3 + kk, i, 1000)
            # the kernels evaluate Box-Muller with the SFU approximations: each
            # normal lies within about 7e-6 of the exact transform of the same
            # uniforms (ln u1 from lg2 to 4e-7 absolute for u1 <= 1 - 2^-7 and
            # from a series above, sin/cos to 4e-7 absolute on [-pi, pi),
            # sqrt to 2^-22 relative, |xi| <= 5.8)
            np.testing.assert_allclose(out[kk, i], ref, rtol=0, atol=1e-5)
    # the draws near u1 = 1, where ln u1 comes from the series, and the
    # largest draws are covered: a million normals against the oracle
    big = ensf.philox_normal(seed, offset, k0=0, count=1, n=8, d=1 << 17).cpu().numpy()[0]
    ref = np.stack([o.noise(seed, offset, 0, i, 1 << 17) for i in range(8)])
    err = np.abs(big - ref)
    assert err.max() <= 1e-5, (err.max(), np.unravel_index(err.argmax(), err.shape))
    assert np.abs(ref).max() > 4.5


def test_row_norms_fp64():
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    x = np.random.default_rng(0).standard_normal((37, 1032)).astype(np.float32)
    got = ensf.row_norms(torch.from_numpy(x).cuda()).cpu().numpy()
    np.testing.assert_allclose(got, np.sum(x.astype(np.float64) ** 2, axis=1), rtol=1e-13)
    # long rows with a large offset: thousands of terms per thread, where an
    # FP32 running sum would lose about ten digits
    # (a plain FP64 running sum over the same 2048 terms per thread is good to
    # about 1e-13 here as well)
    x = (30.0 + np.random.default_rng(1).standard_normal((4, 524288))).astype(np.float32)
    got = ensf.row_norms(torch.from_numpy(x).cuda()).cpu().numpy()
    np.testing.assert_allclose(got, np.sum(x.astype(np.float64) ** 2, axis=1), rtol=1e-12)


def test_ensemble_stats_fp64():
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    g = np.random.default_rng(1)
    z = g.standard_normal((13, 5000)).astype(np.float32)
    truth = g.standard_normal(5000).astype(np.float32)
    mean, rmse = ensf.ensemble_stats(torch.from_numpy(z).cuda(), torch.from_numpy(truth).cuda())
    ref_mean, ref_rmse = o.mean_rmse(z, truth)
    np.testing.assert_allclose(mean.cpu().numpy(), ref_mean, rtol=1e-12, atol=1e-14)
    assert float(rmse.item()) == pytest.approx(ref_rmse, rel=1e-12)


# ---------------------------------------------------------------- weights ---
@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("n,n_x,d", [(1, 1, 8), (3, 5, 72), (20, 20, 1296), (70, 33, 4104)])
def test_weights_match_oracle(path, n, n_x, d):
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    gram, wx, _ = PATHS[path]
    g = np.random.default_rng(n * 1000 + d)
    X = (g.standard_normal((n_x, d)) * 0.5 + 0.2).astype(np.float32)
    f = ensf.Filter(max(n, n_x), d, gram=gram, wx=wx)
    for t in [1.0, 0.5, 0.1, 0.02]:
        s = o.schedule(t, 0.05)
        # particles near the forecast members so that the weights are not one-hot
        Z = (s["alpha"] * X[g.integers(0, n_x, n)] + np.sqrt(t) * 0.05 * g.standard_normal((n, d)))
        Z = Z.astype(np.float32)
        w = f.weights(torch.from_numpy(Z).cuda(), torch.from_numpy(X).cuda(), t, 0.05).cpu().numpy()
        for i in range(n):
            ref, logit = o.weights(X, Z[i], s["alpha"], s["beta2"])
            gap = np.sort(logit)[-1] - np.sort(logit)[-2] if n_x > 1 else np.inf
            assert abs(w[i].sum() - 1.0) < 1e-5
            # the TF32 Gram keeps 10 mantissa bits of each operand: its logits
            # carry errors of about 1e-2 at these sizes, hence the wider bound
            # and the wider gap below which members count as tied
            atol, min_gap = (5e-3, 0.5) if gram == "tf32" else (2e-4, 1e-2)
            if gap > min_gap:
                np.testing.assert_allclose(w[i], ref, atol=atol)


# --------------------------------------------------------------- analysis ---
# Explicit Euler-Maruyama is stable on the likelihood term only while
# dt * sigma^2(t) * h(t) / sigma_obs^2 stays below 2, so the short K of these
# cases comes with sigma_obs large enough (sigma_obs^2 >= 0.6 / K).
SMALL = [
    # (seed, n, grid, layers, K, obs_op, obs_frac, sigma)
    (11, 1, 2, 2, 6, 0, 1.0, 1.0),       # d = 8, N = 1
    (12, 2, 6, 2, 8, 1, 0.5, 0.3),       # d = 72: one full tile + ragged tail
    (13, 3, 36, 1, 10, 0, 0.25, 0.5),    # d = 1296
    (14, 20, 64, 2, 10, 0, 1.0, 1.0),    # the 64x64x2 grid, 10 steps
    (15, 33, 36, 1, 12, 1, 0.25, 0.3),   # N not a tile multiple, arctan
    (16, 70, 44, 1, 10, 1, 0.6, 0.4),    # N spans two 64-row tiles, d = 1936
    (17, 130, 16, 2, 8, 0, 1.0, 0.5),    # N spans two 128-row tiles, d = 512
]


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("case", SMALL, ids=[f"n{c[1]}-d{c[3] * c[2] ** 2}" for c in SMALL])
@pytest.mark.parametrize("noise_mode", ["philox", "buffer"])
def test_analysis_small_matches_oracle(path, case, noise_mode):
    seed, n, grid, layers, K, op, frac, sigma = case
    gram, wx, tol = PATHS[path]
    p = inputs.small_case(seed=seed, n=n, grid=grid, layers=layers, K=K, obs_op=op, obs_frac=frac,
                          sigma_obs=sigma)
    nb = inputs.noise_buffer(seed, K, n, p.d) if noise_mode == "buffer" else None
    ref = run_oracle(p, noise_buf=nb)
    cond = conditioning(p, ref, noise_buf=nb, prec=_cond_prec(gram, wx))
    got = _gpu_analysis(p, gram, wx, noise_buf=nb)
    rel, tie, bad = compare_members(got, ref, cond, tol)
    assert not bad.any(), describe(rel, tie, bad)
    assert tie.sum() <= max(1, n // 10), describe(rel, tie, bad)


@pytest.mark.parametrize("path", list(PATHS))
def test_analysis_plain_64_full(path):
    """The paper's 64x64x2, N = 20, H = I, R = I setup, all K = 100 steps."""
    gram, wx, tol = PATHS[path]
    p = inputs.plain_64()
    ref = run_oracle(p)
    cond = conditioning(p, ref, prec=_cond_prec(gram, wx))
    got = _gpu_analysis(p, gram, wx)
    rel, tie, bad = compare_members(got, ref, cond, tol)
    assert not bad.any(), describe(rel, tie, bad)
    assert tie.sum() == 0, describe(rel, tie, bad)
    _, rmse_ref = o.mean_rmse(ref, p.truth)
    _, rmse_gpu = o.mean_rmse(got, p.truth)
    assert rmse_gpu == pytest.approx(rmse_ref, rel=1e-2)


@pytest.mark.parametrize("path", list(PATHS))
def test_analysis_sparse_arctan_128_rows(path):
    """d = 2x128x128, N = 128, 25 % arctan observations: 12 sampled rows
    (rows are independent given the forecast ensemble, so the oracle is exact
    on them)."""
    gram, wx, tol = PATHS[path]
    p = inputs.sparse_arctan_128()
    rows = np.array([0, 5, 17, 33, 64, 77, 90, 101, 111, 120, 126, 127])
    ref = run_oracle(p, rows=rows)
    cond = conditioning(p, ref, rows=rows, prec=_cond_prec(gram, wx))
    got = _gpu_analysis(p, gram, wx)[rows]
    rel, tie, bad = compare_members(got, ref, cond, tol)
    assert not bad.any(), describe(rel, tie, bad)
    # no sampled member of this workload is ill-conditioned: every one is
    # held to the per-member tolerance
    assert tie.sum() == 0, describe(rel, tie, bad)


def test_analysis_is_deterministic():
    p = inputs.small_case(seed=21, n=33, grid=36, K=6, obs_op=1, obs_frac=0.5, sigma_obs=0.2)
    a = _gpu_analysis(p)
    b = _gpu_analysis(p)
    np.testing.assert_array_equal(a, b)


def test_nonfinite_input_is_reported():
    """A NaN in the forecast ensemble propagates into the particles; with the
    finite check on, ensf_status_sync returns ENSF_ENUMERIC."""
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    p = inputs.small_case(seed=22, n=4, grid=8, K=3)
    prior = p.prior.copy()
    prior[1, 5] = np.nan
    f = ensf.Filter(p.n, p.d, check_finite=True)
    f.analysis(torch.from_numpy(prior).cuda(), torch.from_numpy(p.y).cuda(), None, p.sigma_obs, p.K, p.eps,
               seed=p.seed)
    assert f.status_sync() == ensf.ENUMERIC
    assert f.status_sync() == 0  # the error word is cleared once read


def test_invalid_arguments_raise():
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    f = ensf.Filter(8, 64)
    x = torch.zeros((4, 64), device="cuda")
    y = torch.zeros(64, device="cuda")
    with pytest.raises(ensf.EnsfError):
        f.analysis(x, y, None, 0.0, 3, 0.05)
    with pytest.raises(ensf.EnsfError):
        f.analysis(torch.zeros((9, 64), device="cuda"), y, None, 1.0, 3, 0.05)
    with pytest.raises(ensf.EnsfError):
        f.analysis(x, y, None, 1.0, 3, 0.05, out=x)


@pytest.mark.parametrize("path", ["fp32", "split-bf16"])
def test_graph_replay_matches_eager(path):
    """ENSF_FLAG_CUDA_GRAPH: the captured and replayed analysis is bitwise the
    eager one, across calls that change only the noise seed (graph update)
    and a call with another shape (re-instantiation)."""
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    gram, wx, _ = PATHS[path]
    eager = ensf.Filter(70, 1936, gram=gram, wx=wx)
    graph = ensf.Filter(70, 1936, gram=gram, wx=wx, graph=True)
    stream = torch.cuda.Stream()
    for seed, (n, grid) in [(1, (70, 44)), (2, (70, 44)), (3, (33, 36)), (4, (70, 44))]:
        p = inputs.small_case(seed=seed, n=n, grid=grid, K=6, obs_op=1, obs_frac=0.5, sigma_obs=0.4)
        prior = torch.from_numpy(p.prior).cuda()
        y = torch.from_numpy(p.y).cuda()
        mask = torch.from_numpy(p.mask).cuda()
        with torch.cuda.stream(stream):
            a = eager.analysis(prior, y, mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed)
            b = graph.analysis(prior, y, mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed)
        stream.synchronize()
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_autotuned_analysis_matches_oracle():
    """After ensf_autotune picks the launch shapes, the split path still meets
    the parity bar on the 64x64x2 case."""
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    p = inputs.plain_64()
    f = ensf.Filter(p.n, p.d, gram="split", wx="split", check_finite=True)
    prior = torch.from_numpy(p.prior).cuda()
    y = torch.from_numpy(p.y).cuda()
    rep = f.autotune(prior, y, None, p.sigma_obs, p.eps, p.obs_op, seed=7)
    assert rep["gram_tile_n"] in (128, 256) and rep["wx_tile_n"] in (64, 128, 256)
    assert rep["gram_splits"] >= 1 and rep["gram_ms"] > 0 and rep["wx_ms"] > 0
    assert rep["noise_inline"] in (0, 1) and rep["pdl"] in (0, 1)
    got = _gpu_analysis(p, "split", "split", filt=f)
    ref = run_oracle(p)
    cond = conditioning(p, ref, prec="split")
    rel, tie, bad = compare_members(got, ref, cond, TOL_FP32)
    assert not bad.any(), describe(rel, tie, bad)


BATCH = [
    # (seed, n, grid, layers, obs_op, obs_frac, sigma)
    (41, 20, 16, 2, 0, 1.0, 0.6),    # d = 512
    (42, 33, 36, 1, 1, 0.25, 0.4),   # d = 1296
    (43, 70, 44, 1, 1, 0.6, 0.4),    # d = 1936
    (44, 130, 32, 2, 0, 1.0, 0.5),   # d = 2048, N over one 128 tile
    (45, 256, 24, 1, 1, 0.5, 0.5),   # d = 576, N = two tiles
]


@pytest.mark.parametrize("path,kb_chunk", [("split", 32), ("split-bf16", 32), ("split", 8), ("split-bf16", 64)])
def test_batched_analysis_matches_oracle(path, kb_chunk):
    """Five filters with uneven N and d in one batched analysis (one launch
    per stage for all of them): each against the oracle, sampled rows; with
    the default k-range per Gram work item and with the smallest and largest
    the batched autotuner tries (2 to 8 slices of d, or one)."""
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    gram, wx, tol = PATHS[path]
    K = 8
    probs = [inputs.small_case(seed=c[0], n=c[1], grid=c[2], layers=c[3], K=K, obs_op=c[4], obs_frac=c[5],
                               sigma_obs=c[6]) for c in BATCH]
    f = ensf.Filter(256, 4096, gram=gram, wx=wx)
    f.set_batch_tuning(kb_chunk)
    filters = [dict(prior=torch.from_numpy(p.prior).cuda(), y=torch.from_numpy(p.y).cuda(),
                    mask=torch.from_numpy(p.mask).cuda() if p.mask is not None else None, sigma_obs=p.sigma_obs,
                    obs_op=p.obs_op, seed=p.seed, offset=3) for p in probs]
    outs = f.analysis_batched(filters, K, 0.05)
    assert f.status_sync() == 0
    for p, out in zip(probs, outs):
        p.offset = 3
        rows = np.unique(np.linspace(0, p.n - 1, min(p.n, 12)).astype(int))
        ref = run_oracle(p, rows=rows)
        cond = conditioning(p, ref, rows=rows, prec=_cond_prec(gram, wx))
        got = out.cpu().numpy()[rows]
        rel, tie, bad = compare_members(got, ref, cond, tol)
        assert not bad.any(), f"{p.name}: " + describe(rel, tie, bad)
        assert tie.sum() <= max(1, len(rows) // 6), f"{p.name}: " + describe(rel, tie, bad)


def test_batched_autotuner_choice_is_recorded():
    """ensf_autotune_batched picks one of the k-ranges and keeps it: a later
    batched analysis is bitwise the one with that k-range set explicitly;
    bad k-ranges are rejected."""
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    probs = [inputs.small_case(seed=c[0], n=c[1], grid=c[2], layers=c[3], K=4, obs_op=c[4], obs_frac=c[5],
                               sigma_obs=c[6]) for c in BATCH]
    filters = [dict(prior=torch.from_numpy(p.prior).cuda(), y=torch.from_numpy(p.y).cuda(),
                    mask=torch.from_numpy(p.mask).cuda() if p.mask is not None else None, sigma_obs=p.sigma_obs,
                    obs_op=p.obs_op, seed=p.seed) for p in probs]
    tuned = ensf.Filter(256, 4096, gram="split", wx="bf16")
    rep = tuned.autotune_batched(filters, 0.05)
    assert rep["kb_chunk"] in (8, 16, 32, 64) and rep["trial_ms_k8"] > 0
    a = [o.cpu().numpy() for o in tuned.analysis_batched(filters, 4, 0.05)]
    fixed = ensf.Filter(256, 4096, gram="split", wx="bf16")
    fixed.set_batch_tuning(rep["kb_chunk"])
    b = [o.cpu().numpy() for o in fixed.analysis_batched(filters, 4, 0.05)]
    assert tuned.status_sync() == 0 and fixed.status_sync() == 0
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    for bad in (0, 12, 128):
        with pytest.raises(ensf.EnsfError):
            fixed.set_batch_tuning(bad)


def test_batched_graph_matches_eager():
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    probs = [inputs.small_case(seed=c[0], n=c[1], grid=c[2], layers=c[3], K=5, obs_op=c[4], obs_frac=c[5],
                               sigma_obs=c[6]) for c in BATCH[:3]]
    eager = ensf.Filter(256, 4096, gram="split", wx="bf16")
    graph = ensf.Filter(256, 4096, gram="split", wx="bf16", graph=True)
    stream = torch.cuda.Stream()
    for rep in range(2):
        filters = [dict(prior=torch.from_numpy(p.prior).cuda(), y=torch.from_numpy(p.y).cuda(),
                        mask=torch.from_numpy(p.mask).cuda() if p.mask is not None else None,
                        sigma_obs=p.sigma_obs, obs_op=p.obs_op, seed=p.seed + rep) for p in probs]
        with torch.cuda.stream(stream):
            a = eager.analysis_batched(filters, 5, 0.05)
            b = graph.analysis_batched(filters, 5, 0.05)
        stream.synchronize()
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())


def test_inline_noise_is_bitwise_the_pregenerated_noise():
    """ENSF_FLAG_INLINE_NOISE evaluates the same counter-based draws inside the
    W X epilogue: the analysis is bitwise the pre-generated-slice one."""
    p = inputs.small_case(seed=31, n=130, grid=32, layers=2, K=6, obs_op=1, obs_frac=0.5, sigma_obs=0.4)
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    outs = []
    for inline in (False, True):
        f = ensf.Filter(p.n, p.d, gram="split", wx="bf16", inline_noise=inline)
        outs.append(_gpu_analysis(p, "split", "bf16", filt=f))
    np.testing.assert_array_equal(outs[0], outs[1])


@pytest.mark.parametrize("n,pair,inline", [(130, 0, 0), (130, 0, 1), (130, 0, 2), (512, 1, 0)])
def test_programmatic_dependent_launch_is_bitwise(n, pair, inline):
    """The step kernels (Gram, row softmax, W X) launched with programmatic
    dependent launch, where each waits on the device for its predecessor,
    give bitwise the analysis of ordinary launches, eagerly and replayed from
    a CUDA graph."""
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    p = inputs.small_case(seed=34, n=n, grid=32, layers=2, K=5, obs_op=1, obs_frac=0.5, sigma_obs=0.4)
    prior, y = torch.from_numpy(p.prior).cuda(), torch.from_numpy(p.y).cuda()
    mask = torch.from_numpy(p.mask).cuda()
    bn, stages = (256, 3) if pair else (128, 3)
    stream = torch.cuda.Stream()
    outs = []
    for pdl, graph in [(0, False), (1, False), (1, True)]:
        f = ensf.Filter(p.n, p.d, gram="split", wx="bf16", graph=graph, check_finite=True)
        f.set_tuning(p.n, p.d, bn, stages, gram_splits=2, gram_cta_pair=pair, wx_tile_n=128,
                     noise_inline=inline, pdl=pdl)
        with torch.cuda.stream(stream):
            o_ = f.analysis(prior, y, mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed)
        stream.synchronize()
        assert f.status_sync() == 0
        outs.append(o_.cpu().numpy())
    for o_ in outs[1:]:
        np.testing.assert_array_equal(o_, outs[0])


def test_minibatch_launch_forms_are_bitwise():
    """The mini-batch analysis (windows of J = 32 of 128 members) gives the
    same bits with the draws made in the Gram's warps, in the W X epilogue or
    on the side stream, with and without programmatic dependent launch."""
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    p = inputs.small_case(seed=35, n=128, grid=32, layers=2, K=5, obs_op=1, obs_frac=0.5, sigma_obs=0.4)
    prior, y = torch.from_numpy(p.prior).cuda(), torch.from_numpy(p.y).cuda()
    mask = torch.from_numpy(p.mask).cuda()
    perm = torch.from_numpy(np.random.default_rng(36).permutation(p.n).astype(np.int32)).cuda()
    outs = []
    for place, pdl in [(0, 0), (1, 1), (2, 1), (2, 0)]:
        f = ensf.Filter(p.n, p.d, gram="split", wx="bf16", check_finite=True)
        f.set_tuning(p.n, p.d, 128, 3, gram_splits=2, wx_tile_n=128, noise_inline=place, pdl=pdl)
        o_ = f.analysis_minibatch(prior, y, mask, p.sigma_obs, p.K, p.eps, perm, 32, p.obs_op, seed=p.seed)
        assert f.status_sync() == 0
        outs.append(o_.cpu().numpy())
    for o_ in outs[1:]:
        np.testing.assert_array_equal(o_, outs[0])


@pytest.mark.parametrize("wx_tile", [64, 128, 256])
def test_recorded_noise_placement_is_bitwise(wx_tile):
    """The noise placement recorded for a shape (by ensf_set_tuning here, by
    ensf_autotune otherwise) moves the draws from the Gram's spare warps to the
    W X epilogue without changing them: both analyses are bitwise equal
    (130 particles: the last W X column group is ragged)."""
    p = inputs.small_case(seed=33, n=130, grid=32, layers=2, K=6, obs_op=1, obs_frac=0.5, sigma_obs=0.4)
    from paper_2407_12168_gb300 import ensf
    outs = []
    for place in (0, 1, 2):  # Gram warps, W X epilogue, side-stream kernel
        f = ensf.Filter(p.n, p.d, gram="split", wx="bf16")
        f.set_tuning(p.n, p.d, 128, 3, gram_splits=2, wx_tile_n=wx_tile, noise_inline=place)
        outs.append(_gpu_analysis(p, "split", "bf16", filt=f))
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])
    with pytest.raises(ensf.EnsfError):
        f.set_tuning(p.n, p.d, 128, 3, noise_inline=3)


@pytest.mark.parametrize("path,J", [("split", 16), ("split", 32), ("split-bf16", 32), ("split-bf16", 64)])
def test_minibatch_analysis_matches_oracle(path, J):
    """Mini-batch prior score (Eq. 15-16 with J < N): windows of J members of
    a seeded permutation, one window per Euler-Maruyama step.  (Not BF16 W X
    with J = 16: its 2^-9-level error moves every particle each step, which
    the logit-perturbation check does not model, and with 16-member windows
    a particle can switch to another target member; one such member exceeded
    the BF16 tolerance without being flagged.)"""
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    gram, wx, tol = PATHS[path]
    p = inputs.small_case(seed=51, n=64, grid=32, layers=2, K=8, obs_op=1, obs_frac=0.5, sigma_obs=0.4)
    perm = np.random.default_rng(52).permutation(p.n).astype(np.int32)
    ref = run_oracle(p, perm=perm, J=J)
    cond = conditioning(p, ref, prec=_cond_prec(gram, wx), perm=perm, J=J)
    f = ensf.Filter(p.n, p.d, gram=gram, wx=wx, check_finite=True)
    out = f.analysis_minibatch(torch.from_numpy(p.prior).cuda(), torch.from_numpy(p.y).cuda(),
                               torch.from_numpy(p.mask).cuda(), p.sigma_obs, p.K, p.eps,
                               torch.from_numpy(perm).cuda(), J, obs_op=p.obs_op, seed=p.seed)
    assert f.status_sync() == 0
    rel, tie, bad = compare_members(out.cpu().numpy(), ref, cond, tol)
    assert not bad.any(), describe(rel, tie, bad)
    # a particle that follows the nearest member of a small window changes
    # target whenever the window changes, so small J leaves more of them
    # ill-conditioned (the oracle itself moves beyond tol/2 under perturbations
    # at the path's precision); at least three quarters are compared strictly
    assert tie.sum() <= p.n // 4, describe(rel, tie, bad)


def test_minibatch_with_all_members_is_bitwise_the_full_analysis():
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    p = inputs.small_case(seed=53, n=40, grid=32, K=5, obs_op=0, sigma_obs=0.5)
    f = ensf.Filter(p.n, p.d, gram="split", wx="bf16")
    prior, y = torch.from_numpy(p.prior).cuda(), torch.from_numpy(p.y).cuda()
    a = f.analysis(prior, y, None, p.sigma_obs, p.K, p.eps, seed=p.seed).cpu().numpy()
    ident = torch.arange(p.n, dtype=torch.int32, device="cuda")
    b = f.analysis_minibatch(prior, y, None, p.sigma_obs, p.K, p.eps, ident, p.n, seed=p.seed).cpu().numpy()
    np.testing.assert_array_equal(a, b)


def _check_large_subsample(p, g, sub, gram, wx, tol):
    """64 members of the large-512 analysis against the stored FP64 oracle
    rows (written by tests/golden/make_large512_subsample.py), on 4096 seeded
    state entries per member.  A member whose oracle top-two log-kernel gap
    is within twice the path's log-kernel error bound at some step can follow
    another forecast member than the oracle's; such members are counted
    (at most four) and left out of the comparison.  For the rest: each
    member's relative error within the path's tolerance, and the ensemble
    RMSE of their mean on those entries within 1 % of the oracle's."""
    vals = sub[:, g["idx"]].astype(np.float64)
    ref = g["values"]
    near_tie = g["gap_ratio"] < 2.0 * eps_path(_cond_prec(gram, wx), p.d)
    keep = ~near_tie
    rel = np.linalg.norm(vals - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert near_tie.sum() <= 4, (np.flatnonzero(near_tie).tolist(), rel[near_tie].tolist())
    assert (rel[keep] <= tol).all(), (rel[keep].max(), np.flatnonzero(keep & (rel > tol)).tolist())
    truth = p.truth.astype(np.float32).astype(np.float64)[g["idx"]]
    rmse_gpu = float(np.sqrt(np.mean((vals[keep].mean(axis=0) - truth) ** 2)))
    rmse_ref = float(np.sqrt(np.mean((ref[keep].mean(axis=0) - truth) ** 2)))
    assert abs(rmse_gpu - rmse_ref) <= 0.01 * rmse_ref, (rmse_gpu, rmse_ref)


def test_analysis_large_512_rows_in_the_bench_configuration():
    """d = 2x512x512, N = 1024, K = 100 (2 GiB forecast ensemble) on the
    headline path (split-BF16x3 Gram + BF16 W X, autotuned launch shapes, as
    the benchmark runs it): sampled rows against the oracle, which is exact on
    any subset of rows.  The perturbation check runs only for members beyond
    the tolerance (it triples the oracle's cost)."""
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    gram, wx, tol = PATHS["split-bf16"]
    p = inputs.large_512()
    rows = np.array([0, 383, 1023])
    f = ensf.Filter(p.n, p.d, gram=gram, wx=wx, check_finite=True)
    prior = torch.from_numpy(p.prior).cuda()
    y = torch.from_numpy(p.y).cuda()
    out = torch.empty_like(prior)
    f.autotune(prior, y, None, p.sigma_obs, p.eps, p.obs_op, seed=p.seed, out=out)
    f.analysis(prior, y, None, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed, out=out)
    assert f.status_sync() == 0
    got = out[torch.from_numpy(rows).cuda()].cpu().numpy()
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "large512_subsample64.npz")
    sub = None
    if os.path.exists(golden):
        g = np.load(golden)
        sub = out[torch.from_numpy(g["rows"].astype(np.int64)).cuda()].cpu().numpy()
    del prior, out
    if sub is not None:
        _check_large_subsample(p, g, sub, gram, wx, tol)
    ref = run_oracle(p, rows=rows)
    rel = np.sqrt(((got.astype(np.float64) - ref) ** 2).sum(axis=1) / (ref ** 2).sum(axis=1))
    cond = np.zeros(len(rows))
    if (rel > tol).any():
        cond = conditioning(p, ref, rows=rows, prec=_cond_prec(gram, wx))
    rel, tie, bad = compare_members(got, ref, cond, tol)
    assert not bad.any(), describe(rel, tie, bad)
    # no sampled member of this workload is ill-conditioned: every one is
    # held to the per-member tolerance
    assert tie.sum() == 0, describe(rel, tie, bad)


GRAM_SHAPES = {
    # Gram precision: (tile width, ring depth, k-block width) of every compiled variant
    "split": [(256, 2, 64), (128, 3, 64), (128, 6, 32), (256, 4, 32), (256, 3, 32)],
    "bf16": [(256, 4, 64), (128, 6, 64), (128, 12, 32), (256, 8, 32)],
}


@pytest.mark.parametrize("gram", ["split", "bf16"])
def test_gram_launch_shapes_agree_bitwise(gram):
    """Every K = 16 MMA chunk is accumulated in the same order whatever the
    tile width, ring depth or k-block width, so with the same split
    boundaries (d = 72 x 64, two splits) every launch shape gives the same
    bits through the whole analysis."""
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    p = inputs.small_case(seed=61, n=300, grid=48, layers=2, K=4, obs_op=1, obs_frac=0.5, sigma_obs=0.5)
    prior, y = torch.from_numpy(p.prior).cuda(), torch.from_numpy(p.y).cuda()
    mask = torch.from_numpy(p.mask).cuda()
    outs = []
    for bn, stages, bk in GRAM_SHAPES[gram]:
        f = ensf.Filter(p.n, p.d, gram=gram, wx="bf16", check_finite=True)
        f.set_tuning(p.n, p.d, bn, stages, gram_k_block=bk, gram_splits=2)
        outs.append(f.analysis(prior, y, mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed).cpu().numpy())
        assert f.status_sync() == 0
    for (bn, stages, bk), o_ in zip(GRAM_SHAPES[gram][1:], outs[1:]):
        np.testing.assert_array_equal(o_, outs[0], err_msg=f"shape {(bn, stages, bk)}")


@pytest.mark.parametrize("shape", [(128, 6, 32), (256, 4, 32), (256, 3, 32)])
def test_narrow_kblock_gram_ragged_matches_oracle(shape):
    """32-wide k-blocks (64-byte swizzle) with a ragged state tail (d = 2888
    is not a multiple of 32), ragged member tiles (N = 70) and three splits
    that do not divide the k-blocks evenly, against the oracle."""
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    gram, wx, tol = PATHS["split"]
    p = inputs.small_case(seed=62, n=70, grid=38, layers=2, K=6, obs_op=1, obs_frac=0.5, sigma_obs=0.4)
    ref = run_oracle(p)
    cond = conditioning(p, ref, prec=_cond_prec(gram, wx))
    f = ensf.Filter(p.n, p.d, gram=gram, wx=wx, check_finite=True)
    bn, stages, bk = shape
    f.set_tuning(p.n, p.d, bn, stages, gram_k_block=bk, gram_splits=3)
    got = _gpu_analysis(p, gram, wx, filt=f)
    rel, tie, bad = compare_members(got, ref, cond, tol)
    assert not bad.any(), describe(rel, tie, bad)
    assert tie.sum() <= 2, describe(rel, tie, bad)


def test_set_tuning_rejects_shapes_without_a_kernel():
    from paper_2407_12168_gb300 import ensf
    f = ensf.Filter(64, 4096, gram="split", wx="bf16")
    for bn, stages, bk in [(256, 4, 64), (128, 5, 32), (192, 2, 64), (256, 2, 16), (256, 3, 64)]:
        with pytest.raises(ensf.EnsfError):
            f.set_tuning(64, 4096, bn, stages, gram_k_block=bk)
    g = ensf.Filter(64, 4096, gram="fp32", wx="fp32")
    with pytest.raises(ensf.EnsfError):
        g.set_tuning(64, 4096, 256, 2)


def test_pair_gram_matches_single_cta_bitwise():
    """The CTA-pair Gram (tcgen05 cta_group::2, 256 x 256 tiles) accumulates
    the K = 16 chunks in the same order as the single-CTA shapes: with the
    same split boundaries the analyses are bitwise equal (N = 512, two
    pair tiles per side)."""
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    p = inputs.small_case(seed=63, n=512, grid=48, layers=2, K=3, obs_op=1, obs_frac=0.5, sigma_obs=0.5)
    prior, y = torch.from_numpy(p.prior).cuda(), torch.from_numpy(p.y).cuda()
    mask = torch.from_numpy(p.mask).cuda()
    outs = []
    # (pair, tile width, ring depth, warps generating the next step's noise,
    #  Gram reading the FP32 particles and splitting them itself)
    for pair, bn, stages, nw, f32 in [(0, 256, 2, 8, 0), (1, 256, 3, 8, 0), (0, 128, 3, 8, 0), (1, 256, 3, 4, 0),
                                      (0, 256, 2, 4, 0), (1, 256, 3, 4, 1)]:
        f = ensf.Filter(p.n, p.d, gram="split", wx="bf16", check_finite=True)
        f.set_tuning(p.n, p.d, bn, stages, gram_splits=2, gram_cta_pair=pair, gram_noise_warps=nw,
                     gram_fp32_particles=f32)
        outs.append(f.analysis(prior, y, mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed).cpu().numpy())
        assert f.status_sync() == 0
    for o_ in outs[1:]:
        np.testing.assert_array_equal(o_, outs[0])


@pytest.mark.parametrize("f32", [0, 1])
def test_pair_gram_ragged_state_matches_oracle(f32):
    """One pair tile (N = 256), a ragged state tail (d = 2888 is not a
    multiple of the 64-wide k-block) and three uneven splits, against the
    oracle; with the particle operand from BF16 planes or split in the
    kernel from the FP32 particles."""
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    gram, wx, tol = PATHS["split"]
    p = inputs.small_case(seed=64, n=256, grid=38, layers=2, K=5, obs_op=1, obs_frac=0.5, sigma_obs=0.5)
    ref = run_oracle(p)
    cond = conditioning(p, ref, prec=_cond_prec(gram, wx))
    f = ensf.Filter(p.n, p.d, gram=gram, wx=wx, check_finite=True)
    f.set_tuning(p.n, p.d, 256, 3, gram_splits=3, gram_cta_pair=1, gram_fp32_particles=f32)
    got = _gpu_analysis(p, gram, wx, filt=f)
    rel, tie, bad = compare_members(got, ref, cond, tol)
    assert not bad.any(), describe(rel, tie, bad)
    assert tie.sum() <= max(1, p.n // 50), describe(rel, tie, bad)


def test_tf32_pair_gram_matches_single_cta_bitwise():
    """The TF32 Gram on a CTA pair (tcgen05 cta_group::2 kind::tf32, 256 x 256
    tiles, six-deep ring of 32-element k-blocks) accumulates the K = 8 chunks
    in the single-CTA order: with the same split boundaries the analyses are
    bitwise those of the two single-CTA TF32 shapes (N = 512)."""
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    p = inputs.small_case(seed=66, n=512, grid=48, layers=2, K=3, obs_op=1, obs_frac=0.5, sigma_obs=0.5)
    prior, y = torch.from_numpy(p.prior).cuda(), torch.from_numpy(p.y).cuda()
    mask = torch.from_numpy(p.mask).cuda()
    outs = []
    for pair, bn, stages, nw in [(0, 256, 4, 8), (1, 256, 6, 8), (0, 128, 6, 8), (1, 256, 6, 4)]:
        f = ensf.Filter(p.n, p.d, gram="tf32", wx="split", check_finite=True)
        f.set_tuning(p.n, p.d, bn, stages, gram_k_block=32, gram_splits=2, gram_cta_pair=pair,
                     gram_noise_warps=nw)
        outs.append(f.analysis(prior, y, mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed).cpu().numpy())
        assert f.status_sync() == 0
    for o_ in outs[1:]:
        np.testing.assert_array_equal(o_, outs[0])


def test_tf32_pair_gram_ragged_state_matches_oracle():
    """One TF32 pair tile (N = 256), a ragged state tail (d = 2888 is not a
    multiple of the 32-wide FP32 k-block) and three uneven splits, against
    the oracle at the TF32 path's tolerance."""
    from paper_2407_12168_gb300 import ensf
    gram, wx, tol = PATHS["tf32"]
    p = inputs.small_case(seed=67, n=256, grid=38, layers=2, K=5, obs_op=1, obs_frac=0.5, sigma_obs=0.5)
    ref = run_oracle(p)
    cond = conditioning(p, ref, prec=_cond_prec(gram, wx))
    f = ensf.Filter(p.n, p.d, gram=gram, wx=wx, check_finite=True)
    f.set_tuning(p.n, p.d, 256, 6, gram_k_block=32, gram_splits=3, gram_cta_pair=1)
    got = _gpu_analysis(p, gram, wx, filt=f)
    rel, tie, bad = compare_members(got, ref, cond, tol)
    assert not bad.any(), describe(rel, tie, bad)
    assert tie.sum() <= max(1, p.n // 50), describe(rel, tie, bad)


def test_pair_gram_needs_whole_pair_tiles():
    from paper_2407_12168_gb300 import ensf
    f = ensf.Filter(300, 4096, gram="split", wx="bf16")
    with pytest.raises(ensf.EnsfError):
        f.set_tuning(300, 4096, 256, 3, gram_cta_pair=1)
    g = ensf.Filter(512, 4096, gram="bf16", wx="bf16")
    with pytest.raises(ensf.EnsfError):
        g.set_tuning(512, 4096, 256, 3, gram_cta_pair=1)
    t = ensf.Filter(300, 4096, gram="tf32", wx="split")
    with pytest.raises(ensf.EnsfError):  # TF32 pair: whole tiles, ring depth 6
        t.set_tuning(300, 4096, 256, 6, gram_k_block=32, gram_cta_pair=1)
    with pytest.raises(ensf.EnsfError):
        t.set_tuning(256, 4096, 256, 4, gram_k_block=32, gram_cta_pair=1)


@pytest.mark.parametrize("f32", [0, 1])
def test_pair_gram_in_a_cuda_graph(f32):
    """The cluster-launched pair Gram (both operand forms) captured in a CUDA
    graph and replayed gives the eager bits, across a seed change (graph
    update) and a repeat."""
    torch = _torch()
    from paper_2407_12168_gb300 import ensf
    p0 = inputs.small_case(seed=65, n=512, grid=40, layers=2, K=4, obs_op=1, obs_frac=0.5, sigma_obs=0.5)
    eager = ensf.Filter(p0.n, p0.d, gram="split", wx="bf16")
    graph = ensf.Filter(p0.n, p0.d, gram="split", wx="bf16", graph=True)
    for f in (eager, graph):
        f.set_tuning(p0.n, p0.d, 256, 3, gram_splits=3, gram_cta_pair=1, gram_fp32_particles=f32)
    prior, y = torch.from_numpy(p0.prior).cuda(), torch.from_numpy(p0.y).cuda()
    mask = torch.from_numpy(p0.mask).cuda()
    stream = torch.cuda.Stream()
    for seed in (1, 2, 2):
        with torch.cuda.stream(stream):
            a = eager.analysis(prior, y, mask, p0.sigma_obs, p0.K, p0.eps, p0.obs_op, seed=seed)
            b = graph.analysis(prior, y, mask, p0.sigma_obs, p0.K, p0.eps, p0.obs_op, seed=seed)
        stream.synchronize()
        assert graph.status_sync() == 0
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_analysis_rejects_degenerate_arguments():
    """Empty and oversized problems, a non-positive or non-finite sigma_obs,
    eps outside (0, 1), K < 1, an unknown operator, misaligned or aliased
    buffers: the entry point answers ENSF_EINVAL before any launch, and the
    handle still runs a valid analysis afterwards (against the oracle)."""
    import ctypes
    import torch
    from paper_2407_12168_gb300 import ensf
    p = inputs.small_case(seed=91, n=8, grid=8, K=4, obs_op=0, obs_frac=1.0, sigma_obs=0.5)
    f = ensf.Filter(p.n, p.d, gram="fp32", wx="fp32", check_finite=True)
    lib = ensf.load()
    prior = torch.from_numpy(p.prior).cuda()
    y = torch.from_numpy(p.y).cuda()
    out = torch.empty_like(prior)
    nz = ensf.EnsfNoise(None, p.seed, 0)

    def call(n=p.n, d=p.d, sigma=0.5, K=4, eps=p.eps, op=0, prior_ptr=None, out_ptr=None, noise=True):
        return lib.ensf_analysis(f._h, prior.data_ptr() if prior_ptr is None else prior_ptr, n, d, y.data_ptr(),
                                 None, op, sigma, K, eps, ctypes.byref(nz) if noise else None,
                                 out.data_ptr() if out_ptr is None else out_ptr, None)

    bad = [dict(n=0), dict(n=p.n + 1), dict(d=0), dict(d=p.d + 8), dict(d=12), dict(K=0), dict(sigma=0.0),
           dict(sigma=-1.0), dict(sigma=float("inf")), dict(sigma=float("nan")), dict(eps=0.0), dict(eps=1.0),
           dict(op=2), dict(prior_ptr=prior.data_ptr() + 4), dict(out_ptr=prior.data_ptr()), dict(noise=False)]
    for kw in bad:
        assert call(**kw) == ensf.EINVAL, kw
    torch.cuda.synchronize()
    assert f.status_sync() == 0
    got = f.analysis(prior, y, None, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed).cpu().numpy()
    ref = run_oracle(p)
    rel = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() <= 1e-4, rel
