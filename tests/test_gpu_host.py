"""Page-locked host buffers of ensf_host_alloc: registered with the CUDA
driver (asynchronous copies run from them), zeroed, round-tripped exactly,
released; and the analysis through them equals the analysis from device
inputs."""
import gc

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_host_buffer_round_trip():
    import torch
    from paper_2407_12168_gb300 import ensf
    t = ensf.host_empty((3, 1 << 20), torch.float32)
    assert ensf.host_registered(t)
    assert not ensf.host_registered(torch.empty(16))
    assert t.shape == (3, 1 << 20) and float(t.abs().max()) == 0.0
    frac = ensf.host_huge_fraction(t)
    assert 0.0 <= frac <= 1.0
    src = torch.arange(3 << 20, dtype=torch.float32).view(3, 1 << 20)
    t.copy_(src)
    d = torch.empty_like(t, device="cuda")
    d.copy_(t, non_blocking=True)
    back = ensf.host_empty(t.shape, torch.float32, huge_pages=False)
    assert ensf.host_registered(back)
    back.copy_(d, non_blocking=True)
    torch.cuda.synchronize()
    assert torch.equal(back, src)
    del t, back
    gc.collect()


def test_host_free_rejects_foreign_pointers():
    import ctypes

    import torch
    from paper_2407_12168_gb300 import ensf
    x = torch.empty(16, pin_memory=True)
    assert ensf.load().ensf_host_free(ctypes.c_void_p(x.data_ptr())) == ensf.EINVAL


def test_analysis_from_host_buffers_matches_device_inputs():
    import torch
    from paper_2407_12168_gb300 import ensf, inputs
    p = inputs.small_case(seed=61, n=24, grid=32, layers=2, K=6, obs_op=1, obs_frac=0.5, sigma_obs=0.3)
    f = ensf.Filter(p.n, p.d, gram="split", wx="bf16")
    ref = f.analysis(torch.from_numpy(p.prior).cuda(), torch.from_numpy(p.y).cuda(),
                     torch.from_numpy(p.mask).cuda(), p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed).cpu()
    h_prior = ensf.host_empty(p.prior.shape)
    h_prior.copy_(torch.from_numpy(p.prior))
    h_out = ensf.host_empty(p.prior.shape)
    d_prior = torch.empty(p.prior.shape, device="cuda")
    d_prior.copy_(h_prior, non_blocking=True)
    out = f.analysis(d_prior, torch.from_numpy(p.y).cuda(), torch.from_numpy(p.mask).cuda(), p.sigma_obs, p.K,
                     p.eps, p.obs_op, seed=p.seed)
    h_out.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    assert np.array_equal(h_out.numpy(), ref.numpy())


def test_pipelined_host_analyses_equal_one_by_one():
    """Filter.analyses_from_host (copies overlapped with the neighbouring
    analyses, two alternating device sets) gives every job exactly the
    result of its own analysis from device inputs."""
    import torch
    from paper_2407_12168_gb300 import ensf, inputs
    p = inputs.small_case(seed=62, n=32, grid=32, layers=2, K=5, obs_op=1, obs_frac=0.5, sigma_obs=0.3)
    f = ensf.Filter(p.n, p.d, gram="split", wx="bf16")
    d_prior, d_y, d_mask = (torch.from_numpy(a).cuda() for a in (p.prior, p.y, p.mask))
    jobs, refs = [], []
    for i in range(5):
        scale = 1.0 + 0.1 * i  # another forecast ensemble per job
        h_prior = ensf.host_empty(p.prior.shape)
        h_prior.copy_(torch.from_numpy(p.prior) * scale)
        h_y = ensf.host_empty(p.y.shape)
        h_y.copy_(torch.from_numpy(p.y))
        h_mask = ensf.host_empty(p.mask.shape, torch.uint8)
        h_mask.copy_(torch.from_numpy(p.mask))
        jobs.append(dict(prior=h_prior, y=h_y, mask=h_mask, out=ensf.host_empty(p.prior.shape), seed=p.seed + i))
        refs.append(f.analysis(d_prior * scale, d_y, d_mask, p.sigma_obs, p.K, p.eps, p.obs_op,
                               seed=p.seed + i).cpu())
    for sets in (2, 3):  # device sets rotating under the five jobs
        for j in jobs:
            j["out"].zero_()
        evs = f.analyses_from_host(jobs, p.sigma_obs, p.K, p.eps, p.obs_op, sets=sets)
        torch.cuda.synchronize()
        assert len(evs) == 5
        for j, ref in zip(jobs, refs):
            assert torch.equal(j["out"], ref), sets


def test_sm_copy_kernel_moves_host_and_device_bytes():
    import torch
    from paper_2407_12168_gb300 import ensf
    src = torch.randn(1 << 20, dtype=torch.float32, device="cuda")
    h = ensf.host_empty((1 << 20,))
    ensf.copy_sm(h, src, blocks=16)            # device -> page-locked host
    d = torch.empty_like(src)
    ensf.copy_sm(d, h, blocks=38)              # page-locked host -> device
    e = torch.empty_like(src)
    ensf.copy_sm(e, d, blocks=3)               # device -> device, ragged grid
    torch.cuda.synchronize()
    assert torch.equal(h, src.cpu()) and torch.equal(d, src) and torch.equal(e, src)
    with pytest.raises(ValueError):
        ensf.copy_sm(d[:5], src[:6])
    st = ensf.load().ensf_copy_sm(d.data_ptr() + 4, src.data_ptr(), 16, 1, None)
    assert st == ensf.EINVAL


def test_host_buffer_sits_on_the_devices_nearest_node():
    """ensf_host_alloc places a buffer's pages on the host NUMA node the
    driver reports as closest to the device (where it reports one), and the
    query answers for buffers placed either way."""
    import torch
    from paper_2407_12168_gb300 import ensf
    torch.cuda.init()
    near = ensf.host_empty((1 << 20,), torch.float32)
    anyn = ensf.host_empty((1 << 20,), torch.float32, near_device=False)
    node, dev_node = ensf.host_numa(near)
    node_any, dev_node2 = ensf.host_numa(anyn)
    assert dev_node == dev_node2
    assert node >= -1 and node_any >= -1
    if dev_node >= 0 and node >= 0:
        assert node == dev_node, (node, dev_node)
