"""Cycled data assimilation with the SQG forecast model and the EnSF analysis.

The paper's real-time workflow (Fig. 1, Sec. III): every cycle the forecast
model advances each analysis member over the observation interval (the
prediction step, Eq. 3), observations of the truth arrive (Eq. 2), and the
EnSF analysis (Sec. III-A.2) turns the forecast ensemble into the next
analysis ensemble, whose spread is relaxed to the forecast spread for
stability (Sec. IV-A).  Forecast models here: the project's SQG integrator,
the trained BF16 U-Net surrogate, or persistence (no forecast model).

Workload (the cycled configuration): SQG 2 x 128 x 128, N = 64 members,
100 cycles, a seeded 25 % of grid points observed through arctan with
sigma_obs = 0.1, K = 100 Euler-Maruyama steps per analysis.

Nondimensional model setup (the paper defers the SQG constants to an
external code; these are this project's choices): f = N = H = 1 (lengths in
deformation radii), domain side L = 20, shear Lambda = 1, dt = 0.02,
hyperdiffusion e-folding 0.1 at the cut-off, Newtonian relaxation time 5,
forecast interval Delta = 1 time unit (50 steps).

Everything numerical runs in the library (SQG integrator, U-Net kernels,
EnSF analysis, spread relaxation, ensemble statistics); this module only
sequences the calls and moves small host arrays (observations).
"""
from __future__ import annotations

import dataclasses
import json
import time
from typing import Callable, Dict, List

import numpy as np

from . import ensf, inputs


@dataclasses.dataclass
class CycledConfig:
    n: int = 128
    L: float = 20.0
    dt: float = 0.02
    tau_diss: float = 0.1
    tau_relax: float = 5.0
    delta: float = 1.0            # forecast interval (time units)
    members: int = 64
    cycles: int = 100
    obs_frac: float = 0.25
    sigma_obs: float = 0.1
    K: int = 100
    eps: float = 0.05
    spinup: float = 300.0         # time units of spin-up from small noise
    relax: float = 1.0            # relaxation factor
    relax_mode: str = "spread"    # "spread" (variances) or "perturbations"
    augment: float = 0.15         # std of the input noise added to the surrogate's training inputs
    seed: int = 11

    @property
    def steps_per_cycle(self) -> int:
        return int(round(self.delta / self.dt))


def _torch():
    import torch
    return torch


def sqg(cfg: CycledConfig, batch: int):
    return ensf.SQG(batch, n=cfg.n, L=cfg.L, dt=cfg.dt, tau_diss=cfg.tau_diss, tau_relax=cfg.tau_relax)


def climatology(cfg: CycledConfig, count: int, seed: int):
    """`count` independent model states after spin-up from small band-limited
    noise (states drawn from a long integration, as the paper's initial
    ensembles are)."""
    torch = _torch()
    g = np.random.default_rng(seed)
    n = cfg.n
    k = np.sqrt(np.fft.fftfreq(n)[:, None] ** 2 + np.fft.rfftfreq(n)[None, :] ** 2) * n
    filt = np.exp(-(k / 8.0) ** 2)
    x0 = np.empty((count, 2, n, n), np.float32)
    for b in range(count):
        for lev in range(2):
            f = np.fft.irfft2(np.fft.rfft2(g.standard_normal((n, n))) * filt, s=(n, n))
            x0[b, lev] = 0.1 * f / f.std()
    th = torch.from_numpy(x0).cuda()
    sim = sqg(cfg, count)
    sim.run(th, int(round(cfg.spinup / cfg.dt)))
    torch.cuda.synchronize()
    return th


def training_pairs(cfg: CycledConfig, count: int, trajectories: int, seed: int):
    """`count` (x_t, x_{t+Delta}) pairs from `trajectories` independent SQG runs."""
    torch = _torch()
    per = (count + trajectories - 1) // trajectories
    th = climatology(cfg, trajectories, seed)
    sim = sqg(cfg, trajectories)
    xs, ys = [], []
    for _ in range(per):
        x = th.clone()
        sim.run(th, cfg.steps_per_cycle)
        xs.append(x)
        ys.append(th.clone())
    X = torch.cat(xs)[:count].contiguous()
    Y = torch.cat(ys)[:count].contiguous()
    return X, Y


def train_surrogate(net, X, Y, scale: float, epochs: int, batch: int, lr: float, seed: int,
                    log: Callable[[str], None] = print, augment: float = 0.0) -> List[float]:
    """AdamW on the normalised pairs; the learning rate decays linearly.  With
    ``augment`` > 0 the inputs carry additive white noise of that standard
    deviation (in state units): analysis ensembles carry the small-scale noise
    of the reverse-time SDE, which the surrogate then learns to ignore."""
    torch = _torch()
    g = torch.Generator(device="cpu").manual_seed(seed)
    gdev = torch.Generator(device="cuda").manual_seed(seed + 1)
    Xn, Yn = (X / scale).contiguous(), (Y / scale).contiguous()
    n = Xn.shape[0]
    steps = epochs * (n // batch)
    losses, it = [], 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        acc = 0.0
        for b in range(n // batch):
            idx = perm[b * batch:(b + 1) * batch]
            xb, yb = Xn[idx].contiguous(), Yn[idx].contiguous()
            if augment > 0.0:
                xb = (xb + (augment / scale) * torch.randn(xb.shape, generator=gdev, device=xb.device)).contiguous()
            cur = lr * (1.0 - it / max(steps, 1))
            acc += float(net.train_step(xb, yb, lr=cur, weight_decay=1e-4).item())
            it += 1
        losses.append(acc / (n // batch))
        log(f"epoch {ep}: mean training loss {losses[-1]:.5f}")
    return losses


def observe(cfg: CycledConfig, truth_state, cycle: int):
    """Seeded 25 % mask, y = arctan(truth) + N(0, sigma_obs^2) on it."""
    torch = _torch()
    g = np.random.default_rng([cfg.seed, 7, cycle])
    d = 2 * cfg.n * cfg.n
    mask = np.zeros(d, np.uint8)
    mask[g.permutation(d)[: int(round(cfg.obs_frac * d))]] = 1
    truth = truth_state.reshape(-1).cpu().numpy().astype(np.float64)
    y = np.arctan(truth) + cfg.sigma_obs * g.standard_normal(d)
    y = np.where(mask.astype(bool), y, 0.0).astype(np.float32)
    return torch.from_numpy(y).cuda(), torch.from_numpy(mask).cuda()


def run_cycles(cfg: CycledConfig, forecast: Callable, truth0, ens0, gram: str = "split", wx: str = "bf16",
               log: Callable[[str], None] = print) -> Dict:
    """Cycle forecast -> observe -> EnSF analysis -> spread relaxation."""
    torch = _torch()
    d = 2 * cfg.n * cfg.n
    filt = ensf.Filter(cfg.members, d, gram=gram, wx=wx)
    truth = truth0.clone()
    truth_sim = sqg(cfg, 1)
    ens = ens0.clone()
    rmse_f, rmse_a, spread, t_fc, t_an = [], [], [], 0.0, 0.0
    for c in range(cfg.cycles):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ens = forecast(ens)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        truth_sim.run(truth, cfg.steps_per_cycle)
        y, mask = observe(cfg, truth, c)
        prior = ens.reshape(cfg.members, d).contiguous()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        post = filt.analysis(prior, y, mask, cfg.sigma_obs, cfg.K, cfg.eps, ensf.OBS_ARCTAN,
                             seed=cfg.seed * 7919 + c, offset=c)
        ensf.relax_spread(prior, post, cfg.relax, cfg.relax_mode)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        t_fc += t1 - t0
        t_an += t3 - t2
        tr = truth.reshape(-1)
        _, rf = ensf.ensemble_stats(prior, tr)
        _, ra = ensf.ensemble_stats(post, tr)
        rmse_f.append(float(rf.item()))
        rmse_a.append(float(ra.item()))
        spread.append(float(post.std(dim=0).mean().item()))
        ens = post.reshape(cfg.members, 2, cfg.n, cfg.n).contiguous()
        if c % 10 == 0 or c == cfg.cycles - 1:
            log(f"cycle {c}: forecast RMSE {rmse_f[-1]:.4f}  analysis RMSE {rmse_a[-1]:.4f}  spread {spread[-1]:.4f}")
    if filt.status_sync() != 0:
        raise RuntimeError("device error during cycling")
    return dict(rmse_forecast=rmse_f, rmse_analysis=rmse_a, spread=spread,
                forecast_seconds=t_fc, analysis_seconds=t_an,
                mean_analysis_rmse_second_half=float(np.mean(rmse_a[len(rmse_a) // 2:])))


def experiment(cfg: CycledConfig, pairs: int = 20000, trajectories: int = 64, epochs: int = 6, batch: int = 16,
               lr: float = 2e-3, widths=(32, 64, 128, 256), log: Callable[[str], None] = print) -> Dict:
    """The cycled comparison: surrogate vs integrator vs persistence forecasts."""
    torch = _torch()
    t0 = time.perf_counter()
    X, Y = training_pairs(cfg, pairs, trajectories, cfg.seed + 1)
    scale = float(X.std().item())
    t_data = time.perf_counter() - t0
    log(f"{pairs} training pairs in {t_data:.1f} s (state std {scale:.3f})")
    net = ensf.UNet(widths, cfg.n, cfg.n, max_batch=max(batch, cfg.members))
    net.set_params(torch.from_numpy(inputs.unet_init_params(widths, seed=cfg.seed + 2)).cuda())
    t0 = time.perf_counter()
    losses = train_surrogate(net, X, Y, scale, epochs, batch, lr, cfg.seed + 3, log, augment=cfg.augment)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del X, Y
    # held-out one-interval forecast skill
    Xv, Yv = training_pairs(cfg, 256, min(64, trajectories), cfg.seed + 4)
    pred = torch.cat([net.forward((Xv[i:i + batch] / scale).contiguous()) for i in range(0, 256, batch)]) * scale
    err_sur = float(((pred - Yv).norm() / (Yv - Yv.mean()).norm()).item())
    err_per = float(((Xv - Yv).norm() / (Yv - Yv.mean()).norm()).item())
    log(f"held-out forecast error over one interval: surrogate {err_sur:.4f}, persistence {err_per:.4f}")
    # the cycled runs share the truth and the initial ensemble
    truth0 = climatology(cfg, 1, cfg.seed + 5)
    ens0 = climatology(cfg, cfg.members, cfg.seed + 6)
    integ = sqg(cfg, cfg.members)
    forecasts = {
        "integrator": lambda e: integ.run(e, cfg.steps_per_cycle),
        "surrogate": lambda e: (net.forward((e / scale).contiguous()) * scale).contiguous(),
        "persistence": lambda e: e,
    }
    runs = {}
    for name, fc in forecasts.items():
        log(f"--- cycling with the {name} forecast")
        runs[name] = run_cycles(cfg, fc, truth0, ens0, log=log)
    return dict(config=dataclasses.asdict(cfg), pairs=pairs, epochs=epochs, batch=batch, widths=list(widths),
                unet_params=net.nparams, data_seconds=t_data, train_seconds=t_train, train_loss=losses,
                one_interval_error=dict(surrogate=err_sur, persistence=err_per),
                cycles={k: dict(mean_analysis_rmse_second_half=v["mean_analysis_rmse_second_half"],
                                final_analysis_rmse=v["rmse_analysis"][-1],
                                forecast_seconds=v["forecast_seconds"], analysis_seconds=v["analysis_seconds"],
                                rmse_analysis=v["rmse_analysis"], rmse_forecast=v["rmse_forecast"])
                        for k, v in runs.items()})


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--quick", action="store_true", help="64x64 grid, 16 members, 20 cycles, 2k pairs")
    ap.add_argument("--out", default=None, help="write the JSON report here")
    ap.add_argument("--relax-mode", default="spread", choices=["spread", "perturbations"])
    ap.add_argument("--relax", type=float, default=1.0)
    ap.add_argument("--augment", type=float, default=0.15)
    args = ap.parse_args(argv)
    if args.quick:
        cfg = CycledConfig(n=64, members=16, cycles=20, spinup=150.0, K=50, relax_mode=args.relax_mode,
                           relax=args.relax, augment=args.augment)
        rep = experiment(cfg, pairs=2000, trajectories=32, epochs=3, batch=16, widths=(16, 32, 64, 128))
    else:
        rep = experiment(CycledConfig(relax_mode=args.relax_mode, relax=args.relax, augment=args.augment))
    text = json.dumps(rep)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    print(json.dumps({k: v for k, v in rep.items() if k != "cycles"}))
    print(json.dumps({k: {kk: vv for kk, vv in v.items() if not isinstance(vv, list)} for k, v in rep["cycles"].items()}))


if __name__ == "__main__":
    main()
