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
