"""The d-sharded analysis on CPU ranks (world size 2 over gloo).

Each rank holds a slice of the state columns of X, y and the mask and runs
the host loop of ``paper_2407_12168_gb300.sharded`` -- norms all-reduced
once, split-K partial Grams all-gathered every step, the same softmax on
every rank, W X and the update on its own columns -- with a compute backend
that evaluates the per-slice algebra in FP64 (a test double of the GPU
backend).  Checks: the weights every rank forms from the exchanged partials
equal the unsharded oracle's (Eq. 16); the analysis reassembled from the
slices equals the unsharded FP64 oracle analysis to 1e-12; a rank that leaves
between two steps is reported on the other rank, on the host, before that
rank enqueues the step's work."""
import os
import socket
import sys
import time

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class Fp64ShardBackend:
    """This rank's columns [col0, col0 + d_local) of the analysis, in FP64 on
    the CPU: the sharded form of Sec. III-A's step, term by term."""

    def __init__(self, n, d_local, d_total):
        self.n, self.d_local, self.d_total = n, d_local, d_total
        self.weights = {}  # step -> weights formed on this rank

    def splits(self):
        return 2  # two split-K partials per rank, so the gather order matters

    def zeros(self, shape, dtype):
        import torch
        return torch.zeros(shape, dtype=torch.float64)

    def describe(self, prior, y, mask, sigma_obs, K, eps, col0, obs_op, seed, offset, noise, out):
        return dict(X=np.asarray(prior, dtype=np.float64), y=np.asarray(y, dtype=np.float64),
                    mask=None if mask is None else np.asarray(mask, dtype=np.float64), sigma=sigma_obs, K=K,
                    eps=eps, col0=col0, obs_op=obs_op, seed=seed, offset=offset)

    def _xi(self, desc, k):
        from oracle import oracle as o
        c0, c1 = desc["col0"], desc["col0"] + self.d_local
        return np.stack([o.noise(desc["seed"], desc["offset"], k, i, c1)[c0:c1] for i in range(self.n)])

    def prep(self, desc, norms):
        X = desc["X"]
        desc["m"] = X.mean(axis=0)                       # centre (per column: local)
        norms[:] = __import__("torch").from_numpy(((X - desc["m"]) ** 2).sum(axis=1))
        desc["z"] = self._xi(desc, 0)                    # z <- xi_0 at t = 1

    def _coef(self, desc, k):
        from oracle import oracle as o
        t = 1.0 - k / desc["K"]
        return o.schedule(t, desc["eps"])

    def gram(self, desc, k, partial):
        import torch
        s = self._coef(desc, k)
        zc = desc["z"] - s["alpha"] * desc["m"]
        xc = desc["X"] - desc["m"]
        half = self.d_local // 2                         # two split-K ranges of this slice
        partial[0] = torch.from_numpy(zc[:, :half] @ xc[:, :half].T)
        partial[1] = torch.from_numpy(zc[:, half:] @ xc[:, half:].T)

    def update(self, desc, k, gathered, norms):
        s = self._coef(desc, k)
        a, b2 = s["alpha"], s["beta2"]
        G = np.zeros((self.n, self.n))
        for p in gathered.numpy():                       # rank order, then split order
            G += p
        logit = (2.0 * a * G - a * a * norms.numpy()[None, :]) / (2.0 * b2)   # Eq. 12, row constant dropped
        logit -= logit.max(axis=1, keepdims=True)
        w = np.exp(logit)
        w /= w.sum(axis=1, keepdims=True)                # Eq. 16
        self.weights[k] = w
        z, X = desc["z"], desc["X"]
        s_prior = -(z - a * (w @ X)) / b2                # Eq. 15
        if desc["obs_op"] == 1:
            g = (desc["y"] - np.arctan(z)) / (1.0 + z * z)
        else:
            g = desc["y"] - z
        g = g / desc["sigma"] ** 2
        if desc["mask"] is not None:
            g = g * desc["mask"]
        score = s_prior + s["h"] * g                     # Eq. 17
        dt = 1.0 / desc["K"]
        desc["z"] = z - dt * (s["b"] * z - s["sigma2"] * score) + np.sqrt(s["sigma2"] * dt) * self._xi(desc, k + 1)

    def output(self, desc):
        return desc["z"]


def _problem():
    sys.path.insert(0, ROOT)
    from paper_2407_12168_gb300 import inputs
    return inputs.small_case(seed=41, n=6, grid=8, layers=2, K=8, obs_op=1, obs_frac=0.5, sigma_obs=0.4)


def _worker(rank, world, port, store_port, q, leave_at):
    import datetime
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2407_12168_gb300 import sharded
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    store = dist.TCPStore("127.0.0.1", store_port, world, is_master=(rank == 0),
                          timeout=datetime.timedelta(seconds=30))
    p = _problem()
    (c0, dl), = [sharded.split_columns(p.d, world, multiple=32)[rank]]
    be = Fp64ShardBackend(p.n, dl, p.d)
    ex = sharded.TorchExchange(store=store, heartbeat_timeout_s=3.0)
    run = sharded.ShardedAnalysis(be, ex)

    def on_step(k):
        if leave_at is not None and rank == 1 and k == leave_at:
            q.put((rank, "left", k))
            os._exit(0)  # leaves between steps: nothing of its own is in flight

    mask = None if p.mask is None else p.mask[c0:c0 + dl]
    t0 = time.time()
    try:
        z = run.run(p.prior[:, c0:c0 + dl], p.y[c0:c0 + dl], mask, p.sigma_obs, p.K, p.eps, c0,
                    obs_op=p.obs_op, seed=p.seed, on_step=on_step)
        q.put((rank, "done", (c0, dl, z, be.weights[0])))
    except sharded.ShardLost as e:
        q.put((rank, "lost", (e.step, e.missing, time.time() - t0)))
    if leave_at is None:
        dist.destroy_process_group()


def _run(world, leave_at=None):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port, store_port = _free_port(), _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, store_port, q, leave_at)) for r in range(world)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(180)
        assert pr.exitcode == 0
    res = {}
    while not q.empty():
        r, kind, val = q.get()
        res.setdefault(r, []).append((kind, val))
    return res


def test_sharded_analysis_equals_unsharded_oracle_on_three_uneven_gloo_ranks():
    """Three ranks over 128 columns in 32-column blocks: slices of 32, 32 and 64."""
    from oracle import oracle as o
    p = _problem()
    res = _run(3)
    z = np.zeros((p.n, p.d))
    widths = []
    for r in range(3):
        (kind, (c0, dl, zr, _)), = res[r]
        assert kind == "done"
        z[:, c0:c0 + dl] = zr
        widths.append(dl)
    assert widths == [32, 32, 64]
    ref = o.analysis(p.prior, p.y, p.mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed)
    rel = np.linalg.norm(z - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() <= 1e-12, rel


def test_sharded_analysis_equals_unsharded_oracle_on_two_gloo_ranks():
    from oracle import oracle as o
    p = _problem()
    res = _run(2)
    z = np.zeros((p.n, p.d))
    for r in range(2):
        (kind, (c0, dl, zr, w0)), = res[r]
        assert kind == "done"
        z[:, c0:c0 + dl] = zr
        # the weights of the first step, formed on this rank from the gathered
        # partials, against the unsharded oracle's (particles at xi_0)
        s = o.schedule(1.0, p.eps)
        for i in range(p.n):
            ref, _ = o.weights(p.prior, o.noise(p.seed, 0, 0, i, p.d), s["alpha"], s["beta2"])
            np.testing.assert_allclose(w0[i], ref, rtol=0, atol=1e-13)
    # every rank formed the same weights
    assert np.array_equal(res[0][0][1][3], res[1][0][1][3])
    ref = o.analysis(p.prior, p.y, p.mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed)
    rel = np.linalg.norm(z - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() <= 1e-12, rel


def test_rank_that_leaves_between_steps_is_detected_on_the_host():
    res = _run(2, leave_at=3)
    assert res[1] == [("left", 3)]
    (kind, (step, missing, elapsed)), = res[0]
    assert kind == "lost" and step == 3 and missing == [1]
    assert elapsed < 60.0


def test_split_columns_covers_the_state_in_whole_blocks():
    sys.path.insert(0, ROOT)
    from paper_2407_12168_gb300 import sharded
    for d, world in [(524288, 8), (8192, 2), (32768, 4), (4160, 2)]:
        parts = sharded.split_columns(d, world)
        assert parts[0][0] == 0 and sum(dl for _, dl in parts) == d
        for (c0, dl), (c1, _) in zip(parts, parts[1:]):
            assert c0 + dl == c1 and dl % 64 == 0
    with pytest.raises(ValueError):
        sharded.split_columns(64, 2)
