"""Host-side statistics of the SLMC pipeline: the integrated autocorrelation time estimator
against the closed form of an AR(1) process, tau_int = (1 + rho) / (2 (1 - rho)), and the
binned error of uncorrelated data against sigma / sqrt(T)."""
import math

import numpy as np

from paper_1802_06177_gb300.pipeline import binned_error, integrated_autocorrelation


def test_tau_int_of_ar1_process():
    rng = np.random.default_rng(0)
    for rho in (0.0, 0.5, 0.8):
        T, C = 20000, 8
        a = np.zeros((T, C))
        e = rng.normal(size=(T, C))
        for t in range(1, T):
            a[t] = rho * a[t - 1] + e[t]
        exact = (1 + rho) / (2 * (1 - rho))
        assert abs(integrated_autocorrelation(a) - exact) < 0.08 * exact + 0.03


def test_binned_error_of_white_noise():
    rng = np.random.default_rng(1)
    x = rng.normal(scale=2.0, size=40000)
    assert abs(binned_error(x, nbins=20) / (2.0 / math.sqrt(len(x))) - 1.0) < 0.5


def test_power_law_exponent():
    from paper_1802_06177_gb300.pipeline import power_law_exponent
    sizes = [4, 6, 8, 12]
    assert abs(power_law_exponent(sizes, [3.0 * s ** 2.5 for s in sizes]) - 2.5) < 1e-12
    assert math.isnan(power_law_exponent([4], [1.0]))


def test_crossings_of_scaled_curves():
    from paper_1802_06177_gb300.pipeline import crossings
    temps = [0.20, 0.25, 0.30]
    curves = {4: [1.0, 0.8, 0.6], 8: [1.2, 0.8, 0.4], 12: [1.3, 0.9, 0.5]}
    out = crossings([4, 8, 12], temps, curves)
    assert out[0]["sizes"] == [4, 8] and abs(out[0]["T"] - 0.25) < 1e-12  # exact touch at a scanned point
    assert all(c["sizes"] != [8, 12] for c in out)  # 12 stays above 8: no crossing
    out = crossings([4, 8], temps, {4: [1.0, 0.8, 0.6], 8: [1.1, 0.75, 0.5]})
    assert len(out) == 1 and 0.20 < out[0]["T"] < 0.25


def test_cdw_initial_fields_sit_at_the_double_well_minima():
    import numpy as np
    from paper_1802_06177_gb300.pipeline import initial_fields
    alpha, Lx, L = 4.0, 4, 10
    x = initial_fields("cdw", 3, Lx, L, alpha, seed=1).numpy()
    i = np.arange(Lx * Lx)
    stag = np.where(((i % Lx) + (i // Lx)) % 2 == 0, 1.0, -1.0)
    assert x.shape == (3, Lx * Lx, L)
    assert abs((x * stag[None, :, None]).mean() - alpha) < 0.05  # staggered pattern at +-alpha
    assert abs(x.std(axis=(0, 2)).mean() - 0.3) < 0.05           # noise 0.3 per site
    g = initial_fields("gaussian", 3, Lx, L, alpha, seed=1).numpy()
    assert abs(g.mean()) < 0.1 and abs(g.std() - 1.0) < 0.1


def test_warm_start_fields_are_copied_and_checked():
    import pytest
    import torch

    from paper_1802_06177_gb300.pipeline import initial_fields
    x = torch.randn(3, 16, 8, dtype=torch.float64)
    y = initial_fields(x, 3, 4, 8, 4.0, 0)
    assert torch.equal(y, x) and y.data_ptr() != x.data_ptr()
    with pytest.raises(ValueError):
        initial_fields(x, 2, 4, 8, 4.0, 0)
