"""The whole SLMC procedure (self-learning rounds, then production with cumulative updates)
through the library on a small lattice: it runs end to end, every reported number is finite
and in range, and the learned kinetic coupling is near Table S1's 1/(2 dtau^2)."""
import math

import pytest

from paper_1802_06177_gb300 import pipeline
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_pipeline_small_lattice():
    require_gpu()
    res = pipeline.run(Lx=4, L=40, n_s=10, chains=16, train=96, updates=10, sweeps=5, precision="fp32", rounds=2)
    assert res["training_configs"] == 96 and len(res["training_rounds"]) == 2
    assert 0.0 <= res["acceptance"] <= 1.0 and 0.0 < res["sweep_acceptance"] < 1.0
    assert math.isfinite(res["S_pipi_mean"]) and res["S_pipi_mean"] > 0.0
    assert all(math.isfinite(v) for v in res["J_final"])
    assert abs(res["J_final"][1] - 50.0) < 5.0  # J_k, Table S1
    assert res["evals_per_s"] > 0.0


def test_pipeline_trained_on_dqmc_configurations():
    require_gpu()
    res = pipeline.run(Lx=4, L=40, n_s=10, chains=16, train=64, updates=10, sweeps=5, precision="fp32", rounds=2,
                       train_source="dqmc", dqmc_therm=10, dqmc_gap=2)
    first, second = res["training_rounds"]
    assert first["round"] == "dqmc" and first["configs"] == 64 and 0.0 < first["dqmc_local_acceptance"] < 1.0
    assert second["round"] == 0  # one self-learning refinement after the DQMC fit
    assert abs(first["J"][1] - 50.0) < 5.0  # J_k, Table S1
    assert math.isfinite(res["S_pipi_mean"]) and 0.0 <= res["acceptance"] <= 1.0


def test_dqmc_only_run():
    require_gpu()
    res = pipeline.run_dqmc(4, 20, 10, chains=8, sweeps=25, nblock=1)
    assert res["method"] == "dqmc" and res["sweeps"] == 25
    assert 0.0 < res["local_acceptance"] < 1.0 and 0.0 <= res["block_acceptance"] <= 1.0
    assert math.isfinite(res["S_pipi_mean"]) and res["S_pipi_mean"] > 0.0
    assert res["chain_sweeps_per_s"] > 0.0


def test_autocorrelation_study_runs_both_methods():
    require_gpu()
    res = pipeline.autocorrelation_study([2, 4], beta=1.0, chains=8, steps=40, sweeps=4, train=32)
    assert [r["Lx"] for r in res["sizes"]] == [2, 4] and res["L"] == 10
    for r in res["sizes"]:
        assert r["dqmc_ms_per_step"] > 0.0 and r["slmc_ms_per_step"] > 0.0
        assert math.isfinite(r["dqmc_S"]) and math.isfinite(r["slmc_S"])
        assert 0.0 <= r["dqmc_block_acceptance"] <= 1.0 and 0.0 <= r["slmc_acceptance"] <= 1.0
    assert set(res["exponents"]) == {"dqmc_tau_steps", "slmc_tau_steps", "dqmc_ms_per_independent",
                                     "slmc_ms_per_independent"}


def test_fss_scan_runs():
    require_gpu()
    res = pipeline.fss_scan([2, 4], [0.8, 1.0, 1.2], chains=8, updates=6, sweeps=2, train=16, dqmc_therm=4)
    assert res["training_beta"] == 1.0 and len(res["points"]) == 6
    for pt in res["points"]:
        assert math.isfinite(pt["S_pipi"]) and pt["S_pipi"] > 0.0 and 0.0 <= pt["acceptance"] <= 1.0
        assert abs(pt["S_L_minus_7_4"] - pt["S_pipi"] * pt["Lx"] ** -1.75) < 1e-12
