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
