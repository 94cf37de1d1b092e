"""Cycled assimilation with the learned surrogate (reduced size): the trained
network forecasts better than persistence over one interval, and EnSF cycling
with it tracks the truth better than cycling without a forecast model."""
import pytest

pytestmark = pytest.mark.gpu


def test_surrogate_gains_over_no_forecast_model():
    from paper_2407_12168_gb300 import cycled
    cfg = cycled.CycledConfig(n=64, members=16, cycles=16, spinup=150.0, K=50, seed=5)
    rep = cycled.experiment(cfg, pairs=2000, trajectories=32, epochs=3, batch=16, widths=(16, 32, 64, 128),
                            log=lambda s: None)
    e = rep["one_interval_error"]
    assert e["surrogate"] < 0.7 * e["persistence"]
    c = rep["cycles"]
    assert c["surrogate"]["mean_analysis_rmse_second_half"] < c["persistence"]["mean_analysis_rmse_second_half"]
    assert c["integrator"]["mean_analysis_rmse_second_half"] < c["persistence"]["mean_analysis_rmse_second_half"]


def test_imperfect_model_cycling_with_online_adaptation():
    """The twin experiment's model errors reach the truth, and the online
    adapter fine-tunes the surrogate on consecutive analysis means while
    cycling (two AdamW steps per analysis after the first)."""
    import numpy as np
    import torch
    from paper_2407_12168_gb300 import cycled, ensf, inputs
    cfg = cycled.CycledConfig(n=32, members=8, cycles=6, spinup=40.0, K=20, obs_frac=1.0, obs_op="identity",
                              sigma_obs=1.0, model_error=True, seed=3)
    coefs = [cycled.model_error_coef(cfg, c, 1.0) for c in range(200)]
    realised = np.mean([[v != 0.0 for v in c] for c in coefs], axis=0)
    assert np.all(np.abs(realised - np.array(cycled.MODEL_ERROR_PROB)) < 0.1)
    truth0 = cycled.climatology(cfg, 1, 31)
    ens0 = cycled.climatology(cfg, cfg.members, 32)
    widths = (8, 16, 32, 64)
    net = ensf.UNet(widths, cfg.n, cfg.n, max_batch=cfg.members)
    net.set_params(torch.from_numpy(inputs.unet_init_params(widths, seed=5)).cuda())
    before = net.get_params().clone()
    adapter = cycled.OnlineAdapter(net, scale=1.0, steps=2, batch=4, lr=1e-3)
    r = cycled.run_cycles(cfg, lambda e: net.forward(e.contiguous()), truth0, ens0, log=lambda s: None,
                          adapt=adapter)
    assert np.all(np.isfinite(r["rmse_analysis"])) and np.all(np.isfinite(r["rmse_forecast"]))
    assert len(adapter.losses) == 2 * (cfg.cycles - 1) and np.all(np.isfinite(adapter.losses))
    assert not torch.equal(before, net.get_params())
