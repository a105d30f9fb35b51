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


# ---- the drivers of the autocorrelation and finite-size-scaling studies against the oracle ----
# The studies sequence library calls (DQMC sweeps, fits, E_eff sweeps with Wolff updates,
# cumulative updates). In FP64 mode every one of those calls matches the oracle's trajectory,
# so replaying the same sequence with the oracle's functions on the same seeded fields and
# Philox streams must give the same per-step S(pi, pi) series and acceptance counts.

def _oracle_fields(init, chains, Lx, L, alpha, seed):
    from paper_1802_06177_gb300 import inputs
    if init == "cdw":
        return inputs.cdw_fields(chains, Lx, Lx, L, amp=alpha, noise=0.3, seed=seed)
    return inputs.gaussian_fields(chains, Lx, Lx, L, sigma=1.0, seed=seed)


def _oracle_run_dqmc(Lx, L, n_s, chains, sweeps, dtau, lam, omega0, seed, nblock, init, delta=0.5):
    import numpy as np

    from oracle import HolsteinParams
    from oracle.dqmc import dqmc_sweeps
    from oracle.fermion import fermion_logdet
    from oracle.lattice import exp_hopping
    from oracle.observables import s_cdw
    p = HolsteinParams(Lx, Lx, L, dtau=dtau, lam=lam, omega0=omega0, n_s=n_s)
    E = exp_hopping(Lx, Lx, 1.0, 0.0, dtau)
    x = _oracle_fields(init, chains, Lx, L, lam / omega0 ** 2, seed)
    S = np.zeros((sweeps, chains))
    nl, nb = [0] * chains, [0] * chains
    for k in range(sweeps):
        for c in range(chains):
            a, b = dqmc_sweeps(p, x[c], 1, k, c, seed, delta, nblock=nblock, E=E)
            nl[c] += a
            nb[c] += b
            S[k, c] = s_cdw(p, fermion_logdet(p, x[c], E=E)[2])
    return S, nl, nb


def _oracle_run(Lx, L, n_s, chains, train, updates, sweeps, dtau, lam, omega0, seed, rounds, wolff, train_source,
                dqmc_therm, init, J0=None, dqmc_gap=5, delta=0.3):
    """The SLMC run of pipeline.run replayed with the oracle: DQMC training (optional), self-learning
    rounds, then cumulative updates measuring S(pi, pi) after each. The library's Philox sweep
    counters are 32-bit, so the DQMC training offset 2^40 the driver passes is 0 here."""
    import math

    import numpy as np

    from oracle import HolsteinParams
    from oracle.chain import cumulative_update, eff_sweeps
    from oracle.dqmc import dqmc_sweeps
    from oracle.effective import fit_couplings
    from oracle.lattice import exp_hopping
    from oracle.observables import s_cdw
    from oracle.weight import log_weight
    p = HolsteinParams(Lx, Lx, L, dtau=dtau, lam=lam, omega0=omega0, n_s=n_s)
    E = exp_hopping(Lx, Lx, 1.0, 0.0, dtau)
    x = _oracle_fields(init, chains, Lx, L, lam / omega0 ** 2, seed)
    J = np.array([0.0, omega0 ** 2 / 4 + 1.0 / (2 * dtau ** 2), 0.1, 0.0, 0.0, omega0 ** 2 / 2] if J0 is None
                 else J0, dtype=np.float64)
    per_round = max(1, math.ceil(train / chains))
    sweep_ctr = 1 << 30
    xp = None
    Js = []

    def fit(X):
        Y = [log_weight(p, xi, E=E)[0] for xi in X]
        E0, Jv, _ = fit_couplings(p, X, Y)
        return np.concatenate(([E0], Jv))

    if train_source == "dqmc":
        xd = x.copy()
        for c in range(chains):
            dqmc_sweeps(p, xd[c], dqmc_therm, 0, c, seed, delta, E=E)
        ctr, snaps = dqmc_therm, []
        for _ in range(per_round):
            for c in range(chains):
                dqmc_sweeps(p, xd[c], dqmc_gap, ctr, c, seed, delta, E=E)
            ctr += dqmc_gap
            snaps.append(xd.copy())
        J = fit(np.concatenate(snaps))
        Js.append(J)
        x = xd
        xp = xd
        rounds = max(0, rounds - 1)
    for _ in range(rounds):
        xp = x.copy()
        xs = []
        for u in range(per_round):
            for c in range(chains):
                eff_sweeps(p, xp[c], J[1:], sweeps, sweep_ctr, u & 1, c, seed, delta, nwolff=wolff)
            sweep_ctr += sweeps
            xs.append(xp.copy())
        J = fit(np.concatenate(xs))
        Js.append(J)
    if train_source != "dqmc":
        x = xp if xp is not None else x
    lnw, S_cur = [], []
    for c in range(chains):
        lw, _, _, G = log_weight(p, x[c], E=E)
        lnw.append(lw)
        S_cur.append(s_cdw(p, G))
    S = np.zeros((updates, chains))
    n_acc = [0] * chains
    for u in range(updates):
        for c in range(chains):
            acc, lw, G, _ = cumulative_update(p, x[c], lnw[c], J[0], J[1:], sweeps, u, c, seed, delta, E=E,
                                              nwolff=wolff)
            if acc:
                lnw[c] = lw
                S_cur[c] = s_cdw(p, G)
                n_acc[c] += 1
            S[u, c] = S_cur[c]
    return S, n_acc, J


def test_autocorrelation_study_matches_oracle_chains():
    """autocorrelation_study on 2x2 and 4x4 lattices (beta = 0.8, the paper's g = 1, Omega = 0.5) in
    FP64: the DQMC chains (local sweeps + block updates) and the SLMC chains (DQMC training, one
    self-learning refinement, cumulative updates of E_eff sweeps with one Wolff update each) give the
    oracle's per-step S(pi, pi) series and acceptance counts."""
    import numpy as np
    require_gpu()
    beta, chains, steps, sweeps, train, therm, seed = 0.8, 4, 6, 2, 24, 2, 0x1802061774  # 24 >= 6 fit unknowns
    res = pipeline.autocorrelation_study([2, 4], beta=beta, n_s=10, chains=chains, steps=steps, sweeps=sweeps,
                                         train=train, seed=seed, nblock=2, wolff=1, init="cdw", dqmc_therm=therm,
                                         precision="fp64", want_series=True)
    L, dtau = res["L"], res["dtau"]
    assert L == 8
    for row in res["sizes"]:
        Lx = row["Lx"]
        S_d, nl, nb = _oracle_run_dqmc(Lx, L, min(10, L), chains, steps, dtau, 1.0, 0.5, seed, 2, "cdw")
        assert np.abs(np.array(row["dqmc_series"]) - S_d).max() <= 1e-8, Lx
        assert row["dqmc_accepted_local"] == nl and row["dqmc_accepted_block"] == nb
        S_s, na, J = _oracle_run(Lx, L, min(10, L), chains, train, max(4, steps // sweeps), sweeps, dtau, 1.0, 0.5,
                                 seed, 2, 1, "dqmc", therm, "cdw")
        np.testing.assert_allclose(row["slmc_J"], J, rtol=1e-6, atol=1e-6 * np.abs(J).max())
        assert np.abs(np.array(row["slmc_series"]) - S_s).max() <= 1e-8, Lx
        assert row["slmc_accepted"] == na


def test_fss_scan_matches_oracle_chains():
    """fss_scan on a 4x4 lattice at three temperatures in FP64: E_eff trained once (DQMC + one
    refinement) at the middle temperature, then cumulative updates at each temperature; every
    per-update S(pi, pi) series and acceptance count equals the oracle's replay."""
    import numpy as np
    require_gpu()
    chains, updates, sweeps, train, therm, seed = 4, 3, 2, 24, 2, 0x1802061774
    res = pipeline.fss_scan([4], [0.6, 0.8, 1.0], n_s=10, chains=chains, updates=updates, sweeps=sweeps, train=train,
                            dqmc_therm=therm, seed=seed, wolff=1, precision="fp64", want_series=True)
    mid = 8
    _, _, J = _oracle_run(4, mid, min(10, mid), chains, train, 4, sweeps, 0.1, 1.0, 0.5, seed, 2, 1, "dqmc", therm,
                          "cdw")
    assert len(res["points"]) == 3
    for pt in res["points"]:
        L = pt["L"]
        np.testing.assert_allclose(pt["J"], J, rtol=1e-6, atol=1e-6 * np.abs(J).max())
        S, na, _ = _oracle_run(4, L, min(10, L), chains, 0, updates, sweeps, 0.1, 1.0, 0.5, seed + 7919 * L, 0, 1,
                               "self", therm, "cdw", J0=J)
        assert np.abs(np.array(pt["series"]) - S).max() <= 1e-8, L
        assert pt["accepted"] == na
