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
import sys
import time
from typing import Callable, Dict, List, Optional

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
    obs_op: str = "arctan"        # "arctan" or "identity"
    model_error: bool = False     # imperfect model: random errors added to the truth every interval
    shear: float = 1.0            # Lambda of the truth and integrator
    surrogate_shear: float = 0.0  # Lambda of the model the surrogate learns offline (0: the same)
    online: bool = False          # also cycle a surrogate adapted online to the analyses
    seed: int = 11

    @property
    def steps_per_cycle(self) -> int:
        return int(round(self.delta / self.dt))


def _torch():
    import torch
    return torch


def sqg(cfg: CycledConfig, batch: int, shear: float = 0.0):
    return ensf.SQG(batch, n=cfg.n, L=cfg.L, dt=cfg.dt, tau_diss=cfg.tau_diss, tau_relax=cfg.tau_relax,
                    shear=shear or cfg.shear)


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


def training_pairs(cfg: CycledConfig, count: int, trajectories: int, seed: int, shear: float = 0.0):
    """`count` (x_t, x_{t+Delta}) pairs from `trajectories` independent SQG runs
    (of the model with mean shear `shear`, default the truth's)."""
    torch = _torch()
    per = (count + trajectories - 1) // trajectories
    th = climatology(cfg, trajectories, seed)
    sim = sqg(cfg, trajectories, shear)
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
                    log: Callable[[str], None] = print, augment: float = 0.0,
                    warmup_steps: int = 500) -> List[float]:
    """AdamW on the normalised pairs; the learning rate rises linearly over
    ``warmup_steps`` and then decays linearly to zero (without the warm-up,
    early Adam steps at the full rate can drive the SiLU pre-activations far
    negative, after which the network outputs nothing and stays there).  With
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
            cur = lr * min(1.0, (it + 1) / max(warmup_steps, 1)) * (1.0 - it / max(steps, 1))
            loss = float(net.train_step(xb, yb, lr=cur, weight_decay=1e-4).item())
            acc += loss
            it += 1
            if ep == 0 and it % 250 == 0:
                log(f"  step {it}: loss {loss:.5f}")
        losses.append(acc / (n // batch))
        log(f"epoch {ep}: mean training loss {losses[-1]:.5f}")
    return losses


# Imperfect-model errors of the twin experiment (Sec. IV-A): four processes,
# realised in a forecast interval with these probabilities, with these
# amplitudes relative to the model's average magnitude.
MODEL_ERROR_PROB = (0.20, 0.15, 0.10, 0.05)
MODEL_ERROR_AMP = (0.20, 0.30, 0.40, 0.50)


def model_error_coef(cfg: CycledConfig, cycle: int, magnitude: float) -> List[float]:
    """Per-process coefficients of one interval: realisation (a seeded
    Bernoulli draw per process) x amplitude x the model's average magnitude."""
    g = np.random.default_rng([cfg.seed, 13, cycle])
    real = g.random(len(MODEL_ERROR_PROB)) < np.array(MODEL_ERROR_PROB)
    return [float(r) * a * magnitude for r, a in zip(real, MODEL_ERROR_AMP)]


class OnlineAdapter:
    """Adapts the surrogate to the analyses while cycling (the framework's
    surrogate adapts in real time to the observations it assimilates, Sec. I):
    after each analysis the pair (previous analysis mean -> this analysis
    mean) joins a small replay buffer, and a few AdamW steps on random batches
    of it follow.  The surrogate is trained offline first; this only
    fine-tunes it.  With ``anchor`` (normalised offline pairs X, Y) half of
    every batch is drawn from them, so that a few noisy analysis pairs cannot
    pull the network away from the dynamics it learned offline."""

    def __init__(self, net, scale: float, capacity: int = 32, steps: int = 2, batch: int = 8, lr: float = 1e-4,
                 seed: int = 0, anchor=None):
        self.net, self.scale = net, scale
        self.capacity, self.steps, self.batch, self.lr = capacity, steps, batch, lr
        self.xs, self.ys = [], []
        self.g = np.random.default_rng(seed)
        self.anchor = anchor
        self.losses = []

    def __call__(self, prev_mean, mean, shape):
        self.xs.append((prev_mean.reshape(shape) / self.scale).contiguous())
        self.ys.append((mean.reshape(shape) / self.scale).contiguous())
        if len(self.xs) > self.capacity:
            self.xs.pop(0)
            self.ys.pop(0)
        torch = _torch()
        for _ in range(self.steps):
            own = self.batch // 2 if self.anchor is not None else self.batch
            idx = self.g.choice(len(self.xs), size=min(own, len(self.xs)), replace=False)
            xb = [self.xs[i] for i in idx]
            yb = [self.ys[i] for i in idx]
            if self.anchor is not None:
                ax, ay = self.anchor
                ai = torch.from_numpy(self.g.choice(ax.shape[0], size=self.batch - len(idx), replace=False))
                ai = ai.to(ax.device)
                xb = torch.cat([torch.stack(xb), ax[ai]])
                yb = torch.cat([torch.stack(yb), ay[ai]])
            else:
                xb, yb = torch.stack(xb), torch.stack(yb)
            self.losses.append(float(self.net.train_step(xb.contiguous(), yb.contiguous(), lr=self.lr,
                                                         weight_decay=0.0).item()))


def observe(cfg: CycledConfig, truth_state, cycle: int):
    """Seeded mask of obs_frac of the points, y = H(truth) + N(0, sigma_obs^2)
    on it (H = arctan or the identity)."""
    torch = _torch()
    g = np.random.default_rng([cfg.seed, 7, cycle])
    d = 2 * cfg.n * cfg.n
    mask = np.zeros(d, np.uint8)
    mask[g.permutation(d)[: int(round(cfg.obs_frac * d))]] = 1
    truth = truth_state.reshape(-1).cpu().numpy().astype(np.float64)
    y = (np.arctan(truth) if cfg.obs_op == "arctan" else truth) + cfg.sigma_obs * g.standard_normal(d)
    y = np.where(mask.astype(bool), y, 0.0).astype(np.float32)
    return torch.from_numpy(y).cuda(), torch.from_numpy(mask).cuda()


def run_cycles(cfg: CycledConfig, forecast: Callable, truth0, ens0, gram: str = "split", wx: str = "bf16",
               log: Callable[[str], None] = print, adapt: Optional[Callable] = None) -> Dict:
    """Cycle forecast -> observe -> EnSF analysis -> spread relaxation
    (-> online adaptation of the forecast model when `adapt` is given)."""
    torch = _torch()
    d = 2 * cfg.n * cfg.n
    filt = ensf.Filter(cfg.members, d, gram=gram, wx=wx)
    truth = truth0.clone()
    truth_sim = sqg(cfg, 1)
    ens = ens0.clone()
    rmse_f, rmse_a, spread, t_fc, t_an = [], [], [], 0.0, 0.0
    # the model's average magnitude (root mean square of the initial truth)
    _, mag = ensf.ensemble_stats(truth.reshape(1, d), torch.zeros(d, device=truth.device))
    magnitude = float(mag.item())
    obs_op = ensf.OBS_ARCTAN if cfg.obs_op == "arctan" else ensf.OBS_IDENTITY
    for c in range(cfg.cycles):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ens = forecast(ens)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        truth_sim.run(truth, cfg.steps_per_cycle)
        if cfg.model_error:
            ensf.model_error(truth.reshape(1, d), model_error_coef(cfg, c, magnitude), seed=cfg.seed * 31 + 3,
                             cycle=c)
        y, mask = observe(cfg, truth, c)
        prior = ens.reshape(cfg.members, d).contiguous()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        post = filt.analysis(prior, y, mask, cfg.sigma_obs, cfg.K, cfg.eps, obs_op,
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
        if adapt is not None:
            mean, _ = ensf.ensemble_stats(post)
            mean = mean.float()
            if c > 0:
                adapt(prev_mean, mean, (2, cfg.n, cfg.n))
            prev_mean = mean
        spread.append(float(post.std(dim=0).mean().item()))
        ens = post.reshape(cfg.members, 2, cfg.n, cfg.n).contiguous()
        if c % 10 == 0 or c == cfg.cycles - 1:
            log(f"cycle {c}: forecast RMSE {rmse_f[-1]:.4f}  analysis RMSE {rmse_a[-1]:.4f}  spread {spread[-1]:.4f}")
    if filt.status_sync() != 0:
        raise RuntimeError("device error during cycling")
    return dict(rmse_forecast=rmse_f, rmse_analysis=rmse_a, spread=spread,
                forecast_seconds=t_fc, analysis_seconds=t_an,
                mean_analysis_rmse_second_half=float(np.mean(rmse_a[len(rmse_a) // 2:])))


def relax_sweep(cfg: CycledConfig, settings, log: Callable[[str], None] = print) -> Dict:
    """Cycling with the integrator forecast for several (relax_mode, relax,
    delta) settings, all from the same truth and initial ensemble."""
    out = {}
    for mode, relax, delta in settings:
        c = dataclasses.replace(cfg, relax_mode=mode, relax=relax, delta=delta)
        truth0 = climatology(c, 1, c.seed + 5)
        ens0 = climatology(c, c.members, c.seed + 6)
        integ = sqg(c, c.members)
        log(f"--- integrator forecast, relax {mode} {relax}, interval {delta}")
        r = run_cycles(c, lambda e: integ.run(e, c.steps_per_cycle), truth0, ens0, log=log)
        out[f"{mode}:{relax}:{delta}"] = dict(mean_analysis_rmse_second_half=r["mean_analysis_rmse_second_half"],
                                              final_spread=r["spread"][-1], rmse_analysis=r["rmse_analysis"],
                                              spread=r["spread"])
    return out


def experiment(cfg: CycledConfig, pairs: int = 20000, trajectories: int = 64, epochs: int = 6, batch: int = 16,
               lr: float = 1e-3, widths=(32, 64, 128, 256), log: Callable[[str], None] = print) -> Dict:
    """The cycled comparison: surrogate vs integrator vs persistence forecasts."""
    torch = _torch()
    t0 = time.perf_counter()
    X, Y = training_pairs(cfg, pairs, trajectories, cfg.seed + 1, shear=cfg.surrogate_shear)
    scale = float(X.std().item())
    t_data = time.perf_counter() - t0
    log(f"{pairs} training pairs in {t_data:.1f} s (state std {scale:.3f})")
    net = ensf.UNet(widths, cfg.n, cfg.n, max_batch=max(batch, cfg.members))
    net.set_params(torch.from_numpy(inputs.unet_init_params(widths, seed=cfg.seed + 2)).cuda())
    t0 = time.perf_counter()
    losses = train_surrogate(net, X, Y, scale, epochs, batch, lr, cfg.seed + 3, log, augment=cfg.augment)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    # offline pairs kept for rehearsal by the online adapter (normalised)
    anchor = ((X[:2048] / scale).contiguous(), (Y[:2048] / scale).contiguous()) if cfg.online else None
    del X, Y
    # held-out one-interval forecast skill against the truth's model
    Xv, Yv = training_pairs(cfg, 256, min(64, trajectories), cfg.seed + 4)

    def one_interval_error(m):
        pred = torch.cat([m.forward((Xv[i:i + batch] / scale).contiguous()) for i in range(0, 256, batch)]) * scale
        return float(((pred - Yv).norm() / (Yv - Yv.mean()).norm()).item())
    err_sur = one_interval_error(net)
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
    adapters = {}
    if cfg.online:
        net_on = ensf.UNet(widths, cfg.n, cfg.n, max_batch=max(batch, cfg.members))
        net_on.set_params(net.get_params())
        forecasts["surrogate+online"] = lambda e: (net_on.forward((e / scale).contiguous()) * scale).contiguous()
        adapters["surrogate+online"] = OnlineAdapter(net_on, scale, seed=cfg.seed + 7, anchor=anchor)
    runs = {}
    for name, fc in forecasts.items():
        log(f"--- cycling with the {name} forecast")
        runs[name] = run_cycles(cfg, fc, truth0, ens0, log=log, adapt=adapters.get(name))
    errors = dict(surrogate=err_sur, persistence=err_per)
    if cfg.online:
        errors["surrogate+online (after cycling)"] = one_interval_error(net_on)
        log(f"held-out one-interval error of the adapted surrogate: {errors['surrogate+online (after cycling)']:.4f}")
    return dict(config=dataclasses.asdict(cfg), pairs=pairs, epochs=epochs, batch=batch, widths=list(widths),
                unet_params=net.nparams, data_seconds=t_data, train_seconds=t_train, train_loss=losses,
                one_interval_error=errors,
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
    ap.add_argument("--delta", type=float, default=None, help="forecast interval (time units)")
    ap.add_argument("--imperfect", action="store_true",
                    help="the paper's imperfect-model twin experiment: 64x64x2, 20 members, every point "
                         "observed with H = I and R = I, random model errors added to the truth")
    ap.add_argument("--online", action="store_true",
                    help="also cycle a surrogate adapted online to the analyses")
    ap.add_argument("--surrogate-shear", type=float, default=0.0,
                    help="mean shear of the model the surrogate learns offline (0: the truth's)")
    ap.add_argument("--sweep", action="store_true",
                    help="integrator-only cycling over relaxation modes, factors and intervals")
    args = ap.parse_args(argv)
    args.augment_set = any(a.startswith("--augment") for a in (argv if argv is not None else sys.argv[1:]))
    if args.sweep:
        cfg = CycledConfig()
        settings = [(m, r, dl) for dl in (1.0, 3.0) for m, r in (("spread", 1.0), ("perturbations", 1.0),
                                                                   ("perturbations", 0.5))]
        rep = relax_sweep(cfg, settings)
        if args.out:
            with open(args.out, "w") as f:
                f.write(json.dumps(rep))
        print(json.dumps({k: {kk: vv for kk, vv in v.items() if not isinstance(vv, list)} for k, v in rep.items()}))
        return
    extra = {} if args.delta is None else {"delta": args.delta}
    extra.update(online=args.online, surrogate_shear=args.surrogate_shear)
    if args.imperfect:
        # every point observed with R = I: the analyses carry white observation
        # noise of O(0.5), so the surrogate trains with inputs noised at that level
        augment = args.augment if args.augment_set else 0.5
        cfg = CycledConfig(n=64, members=20, obs_frac=1.0, obs_op="identity", sigma_obs=1.0, model_error=True,
                           spinup=150.0, relax_mode=args.relax_mode, relax=args.relax, augment=augment,
                           **extra)
        rep = experiment(cfg, pairs=20000, trajectories=64, epochs=6, batch=16, widths=(32, 64, 128, 256))
    elif args.quick:
        cfg = CycledConfig(n=64, members=16, cycles=20, spinup=150.0, K=50, relax_mode=args.relax_mode,
                           relax=args.relax, augment=args.augment, **extra)
        rep = experiment(cfg, pairs=2000, trajectories=32, epochs=3, batch=16, widths=(16, 32, 64, 128))
    else:
        rep = experiment(CycledConfig(relax_mode=args.relax_mode, relax=args.relax, augment=args.augment, **extra))
    text = json.dumps(rep)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    print(json.dumps({k: v for k, v in rep.items() if k != "cycles"}))
    print(json.dumps({k: {kk: vv for kk, vv in v.items() if not isinstance(vv, list)} for k, v in rep["cycles"].items()}))


if __name__ == "__main__":
    main()
