"""The d-sharded analysis entry points (ensf_shard_*) on one GPU.

Two or four slices of the state columns run in lockstep in one process, each
on its own handle, on one stream: every slice's preparation, the norms
summed over the slices, then per step every slice's partial Grams written
into its own block of one gathered buffer (what the all-gather of a
multi-GPU run delivers) and every slice's update from all of them.  No
kernel waits for another.  Reassembled, the slices must match the FP64
oracle's unsharded analysis at the path's per-member tolerance (the noise
is drawn at global columns, so a wrong column offset fails), and the
unsharded GPU analysis with the same split-K boundaries far more tightly."""
import numpy as np
import pytest

from oracle import oracle as o
from paper_2407_12168_gb300 import inputs

from .parity_util import compare_members, conditioning, describe, run_oracle

pytestmark = pytest.mark.gpu

PATHS = {"fp32": ("fp32", "fp32", 1e-4), "split-bf16": ("split", "bf16", 1e-2), "split": ("split", "split", 1e-4)}


def _lockstep(p, gram, wx, world, S_local=None, inline_noise=False, noise=None):
    import torch
    from paper_2407_12168_gb300 import ensf, sharded
    parts = sharded.split_columns(p.d, world)
    prior = torch.from_numpy(p.prior).cuda()
    y = torch.from_numpy(p.y).cuda()
    mask = None if p.mask is None else torch.from_numpy(p.mask).cuda()
    filt, descs = [], []
    for c0, dl in parts:
        f = ensf.Filter(p.n, dl, gram=gram, wx=wx, check_finite=True, inline_noise=inline_noise)
        if S_local is not None:
            f.set_tuning(p.n, dl, 256 if p.n > 128 else 128, 2 if p.n > 128 else 3, gram_splits=S_local)
        nz = None if noise is None else noise[:, :, c0:c0 + dl].contiguous()
        descs.append(f.shard(prior[:, c0:c0 + dl].contiguous(), y[c0:c0 + dl].contiguous(),
                             None if mask is None else mask[c0:c0 + dl].contiguous(), p.sigma_obs, p.K, p.eps, c0,
                             obs_op=p.obs_op, seed=p.seed, offset=p.offset, noise=nz))
        filt.append(f)
    S = [f.shard_splits(p.n, dl) for f, (_, dl) in zip(filt, parts)]
    assert len(set(S)) == 1
    S = S[0]
    norms_parts = torch.zeros((world, p.n), dtype=torch.float64, device="cuda")
    for r, f in enumerate(filt):
        f.shard_prep(descs[r], norms_parts[r])
    norms = norms_parts.sum(dim=0)
    gathered = torch.zeros((world * S, p.n, p.n), dtype=torch.float32, device="cuda")
    for k in range(p.K):
        for r, f in enumerate(filt):
            f.shard_gram(descs[r], k, gathered[r * S:(r + 1) * S])
        for r, f in enumerate(filt):
            f.shard_update(descs[r], k, gathered, norms)
    torch.cuda.synchronize()
    for f in filt:
        assert f.status_sync() == 0
    out = np.zeros((p.n, p.d))
    for (c0, dl), dsc in zip(parts, descs):
        out[:, c0:c0 + dl] = dsc.out_tensor.cpu().numpy()
    return out, S


def _unsharded(p, gram, wx, splits=None, noise=None):
    import torch
    from paper_2407_12168_gb300 import ensf
    f = ensf.Filter(p.n, p.d, gram=gram, wx=wx)
    if splits is not None:
        f.set_tuning(p.n, p.d, 256 if p.n > 128 else 128, 2 if p.n > 128 else 3, gram_splits=splits)
    out = f.analysis(torch.from_numpy(p.prior).cuda(), torch.from_numpy(p.y).cuda(),
                     None if p.mask is None else torch.from_numpy(p.mask).cuda(), p.sigma_obs, p.K, p.eps,
                     p.obs_op, seed=p.seed, offset=p.offset, noise=noise)
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("world", [2, 4])
def test_sharded_lockstep_matches_oracle(path, world):
    gram, wx, tol = PATHS[path]
    p = inputs.small_case(seed=51, n=40, grid=64, layers=2, K=12, obs_op=1, obs_frac=0.25, sigma_obs=0.3)
    ref = run_oracle(p)
    got, _ = _lockstep(p, gram, wx, world)
    cond = conditioning(p, ref, prec="bf16" if "bf16" in (gram, wx) else gram)
    rel, tie, bad = compare_members(got, ref, cond, tol)
    assert not bad.any(), describe(rel, tie, bad)
    assert tie.sum() <= 1, describe(rel, tie, bad)
    _, r_ref = o.mean_rmse(ref, p.truth)
    _, r_got = o.mean_rmse(got, p.truth)
    assert r_got == pytest.approx(r_ref, rel=1e-2)


def test_sharded_lockstep_with_aligned_splits_tracks_unsharded_gpu():
    """Slices of 2 x 4096 columns with 4 split-K ranges each line up with the
    unsharded analysis's 8 ranges over 8192 columns: the Gram partials are the
    same numbers, and only the FP64 norm sums are associated differently."""
    p = inputs.small_case(seed=52, n=64, grid=64, layers=2, K=10, obs_op=0, obs_frac=1.0, sigma_obs=0.5)
    got, S = _lockstep(p, "split", "split", 2, S_local=4)
    assert S == 4
    ref = _unsharded(p, "split", "split", splits=8)
    rel = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() <= 1e-6, rel.max()


def test_sharded_noise_placements_and_buffer_agree():
    """The draws of a slice do not depend on where they are made (Gram warps,
    W X epilogue) and equal a caller buffer holding the same numbers."""
    import torch
    from paper_2407_12168_gb300 import ensf
    p = inputs.small_case(seed=53, n=32, grid=32, layers=2, K=6, obs_op=1, obs_frac=0.5, sigma_obs=0.3)
    a, _ = _lockstep(p, "split", "bf16", 2)
    b, _ = _lockstep(p, "split", "bf16", 2, inline_noise=True)
    assert np.array_equal(a, b)
    buf = torch.empty((p.K + 1, p.n, p.d), dtype=torch.float32, device="cuda")
    st = ensf.load().ensf_philox_normal(p.seed, p.offset, 0, p.K + 1, p.n, p.d, buf.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
    assert st == ensf.OK
    c, _ = _lockstep(p, "split", "bf16", 2, noise=buf)
    assert np.array_equal(a, c)
