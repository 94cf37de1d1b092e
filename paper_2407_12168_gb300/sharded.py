"""d-sharded EnSF analysis: one filter whose state is split along d across ranks.

The paper runs the EnSF of one large state on many GPUs (Sec. III-A.3, and
the weak-scaling study of Sec. IV-B).  Along the state dimension the method
splits with one exchange per Euler-Maruyama step: H is elementwise and R
diagonal, so the likelihood score, the weighted sum W X and the update
(Eq. 7, 15, 17) need only a rank's own columns, while the log-kernel of
Eq. 12 / 16 needs two sums over all of d -- the cross term z_i . x_j
(exchanged every step) and the squared norms |x_j - m|^2 (exchanged once per
analysis).  Each rank

    prep                 its columns' shares of the norms      -> all-reduce (sum)
    for k in 0 .. K-1:
        heartbeat(k)     every peer reached step k (host check, bounded)
        gram(k)          its columns' split-K partial Grams    -> all-gather (rank order)
        update(k)        the same weights on every rank from all partials,
                         then W X + score + update of its own columns

This module is the host side of that loop: the ranks' compute goes through
a backend (``CudaShardBackend``: the library's ensf_shard_* entry points on
this rank's GPU) and the exchange through ``TorchExchange``
(torch.distributed: NCCL between GPUs, gloo on CPU ranks).  Summing the
gathered partials in rank order keeps the weights bit-identical on every
rank.  Failure detection: before each step's launches every rank posts a
heartbeat to the store and waits, with a limit, for its peers'; a rank that
left between steps is reported as ``ShardLost`` on the others before they
enqueue more work.
"""
from __future__ import annotations

import datetime


class ShardLost(RuntimeError):
    """A peer rank did not reach a step of the sharded analysis in time."""

    def __init__(self, step: int, missing, detail: str = ""):
        self.step = step
        self.missing = sorted(missing)
        super().__init__(f"sharded analysis: rank(s) {self.missing} did not reach step {step}"
                         + (f" ({detail})" if detail else ""))


def split_columns(d: int, world: int, multiple: int = 64):
    """Column ranges [(col0, d_local)] of `world` ranks over a state of d
    entries: equal slices, each a multiple of `multiple` columns (a whole
    number of Gram k-blocks, so the slices line up with split-K ranges),
    the last taking the remainder."""
    if world < 1 or d < 1:
        raise ValueError("need world >= 1 and d >= 1")
    base = (d // world) // multiple * multiple
    if base == 0:
        raise ValueError(f"d = {d} too small for {world} slices of {multiple}-column blocks")
    out = []
    for r in range(world):
        col0 = r * base
        out.append((col0, base if r < world - 1 else d - col0))
    return out


class TorchExchange:
    """The two exchanges of the sharded analysis over a torch.distributed
    process group, plus a heartbeat on a key-value store (a
    torch.distributed Store: TCPStore, FileStore)."""

    def __init__(self, group=None, store=None, heartbeat_timeout_s: float = 30.0, tag: str = "ensf"):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.store = store
        self.timeout = datetime.timedelta(seconds=float(heartbeat_timeout_s))
        self.tag = tag
        self.analysis = 0

    def all_reduce_sum(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)

    def all_gather(self, gathered, local):
        """gathered [world * m ...] <- every rank's `local` [m ...] in rank order
        (`local` may be this rank's own slot of `gathered`: NCCL gathers in place)."""
        if self.dist.get_backend(self.group) == "nccl":
            self.dist.all_gather_into_tensor(gathered, local, group=self.group)
        else:
            chunks = list(gathered.chunk(self.world))
            self.dist.all_gather(chunks, local.clone(), group=self.group)

    def begin_analysis(self):
        self.analysis += 1

    def heartbeat(self, step: int):
        """Post this rank's arrival at `step` and wait (bounded) for the others'."""
        if self.store is None or self.world == 1:
            return
        key = f"{self.tag}/{self.analysis}/{step}/"
        try:
            self.store.set(key + str(self.rank), "1")
        except Exception as e:  # the store's host rank is gone
            raise ShardLost(step, [r for r in range(self.world) if r != self.rank], f"store: {e}") from e
        others = [key + str(r) for r in range(self.world) if r != self.rank]
        try:
            self.store.wait(others, self.timeout)
        except Exception as e:
            missing = []
            for r in range(self.world):
                if r == self.rank:
                    continue
                try:
                    if not self.store.check([key + str(r)]):
                        missing.append(r)
                except Exception:
                    missing.append(r)
            raise ShardLost(step, missing or [r for r in range(self.world) if r != self.rank], str(e)) from e


class CudaShardBackend:
    """This rank's slice computed by the library (ensf_shard_* on the GPU)."""

    def __init__(self, n: int, d_local: int, gram: str = "split", wx: str = "bf16", check_finite: bool = False,
                 inline_noise: bool = False):
        from . import ensf
        self.ensf = ensf
        self.f = ensf.Filter(n, d_local, gram=gram, wx=wx, check_finite=check_finite, inline_noise=inline_noise)
        self.n, self.d_local = int(n), int(d_local)

    def splits(self) -> int:
        return self.f.shard_splits(self.n, self.d_local)

    def zeros(self, shape, dtype):
        import torch
        return torch.zeros(shape, dtype=getattr(torch, dtype), device="cuda")

    def describe(self, prior, y, mask, sigma_obs, K, eps, col0, obs_op, seed, offset, noise, out):
        return self.f.shard(prior, y, mask, sigma_obs, K, eps, col0, obs_op=obs_op, seed=seed, offset=offset,
                            noise=noise, out=out)

    def prep(self, desc, norms):
        self.f.shard_prep(desc, norms)

    def gram(self, desc, k, partial):
        self.f.shard_gram(desc, k, partial)

    def update(self, desc, k, gathered, norms):
        self.f.shard_update(desc, k, gathered, norms)

    def output(self, desc):
        return desc.out_tensor


class ShardedAnalysis:
    """This rank's part of a d-sharded analysis: a compute backend for its
    columns and an exchange with the other ranks."""

    def __init__(self, backend, exchange):
        self.backend = backend
        self.exchange = exchange
        self.S = backend.splits()
        n = backend.n
        self.norms = backend.zeros((n,), "float64")
        self.gathered = backend.zeros((exchange.world * self.S, n, n), "float32")
        r = exchange.rank
        self.local = self.gathered[r * self.S:(r + 1) * self.S]

    def run(self, prior, y, mask, sigma_obs: float, K: int, eps: float, col0: int, obs_op: int = 0,
            seed: int = 0, offset: int = 0, noise=None, out=None, on_step=None):
        """Analysis of this rank's columns [col0, col0 + d_local); returns them
        (the slice of the analysis ensemble).  ``on_step(k)``, if given, runs
        on the host before step k's heartbeat (tests use it to stop a rank)."""
        be, ex = self.backend, self.exchange
        ex.begin_analysis()
        desc = be.describe(prior, y, mask, sigma_obs, K, eps, col0, obs_op, seed, offset, noise, out)
        be.prep(desc, self.norms)
        ex.all_reduce_sum(self.norms)
        for k in range(K):
            if on_step is not None:
                on_step(k)
            ex.heartbeat(k)
            be.gram(desc, k, self.local)
            ex.all_gather(self.gathered, self.local)
            be.update(desc, k, self.gathered, self.norms)
        return be.output(desc)
