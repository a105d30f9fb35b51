"""Self-learning Monte Carlo for the 2D Holstein model end to end on one GPU (every step runs
in libslmc's kernels; this module only sequences the calls and reduces the measurements).

Steps (Sec. "SLMC" and Suppl. Sec. "SLMC for the Holstein model"):
  1. start from the bare phonon action written in the E_eff basis (exact at lambda = 0:
     J_k = omega0^2/4 + 1/(2 dtau^2), J_nn' = omega0^2/2) plus a small double-well term;
  2. self-learning: propose configurations with effective-model sweeps under the current
     couplings (the proposals of the cumulative update), score each with the exact ln w and
     refit E_eff on them (Eq. (5)), and repeat; or (--train-source dqmc, as the paper does)
     train on configurations of conventional DQMC chains (Suppl. Eqs. (S3)-(S6)) after
     thermalisation, one per chain every --dqmc-gap sweeps, then refine with the remaining
     self-learning rounds;
  3. production: cumulative updates (Eq. (6)) with the learned couplings, measuring the CDW
     structure factor S(pi, pi) after every update and counting acceptances.
Error bars: the per-chain time series are averaged over chains, then binned in time.
--dqmc-only runs the conventional DQMC chains instead and measures S(pi, pi) after every sweep:
the baseline whose autocorrelation time and cost per sweep the self-learning method is
compared with (Sec. "Results").
Under torchrun every process runs its own chains on its own GPU (Philox key = seed + rank);
the regression is fitted over all processes' configurations (paper_1802_06177_gb300.dist)
and the measurements are summed over processes; rank 0 prints the result.

python -m paper_1802_06177_gb300.pipeline --Lx 24 --L 240 --n-s 8 --chains 32 --train 2000 \
    --updates 500 --sweeps 100 --precision fp32
"""
import argparse
import json
import math
import time

import numpy as np
import torch

from . import inputs
from .dist import fit_eff_distributed, sum_over_processes
from .slmc import UPDATE_CONTINUE, Context


def integrated_autocorrelation(series_per_chain, window=5.0):
    """Integrated autocorrelation time of a [T][chains] time series: the normalised
    autocorrelation is averaged over chains and summed up to the first lag M >= window * tau
    (Sokal's self-consistent window)."""
    a = np.asarray(series_per_chain, dtype=np.float64)
    a = a - a.mean(axis=0, keepdims=True)
    T = a.shape[0]
    var = (a * a).mean()
    if T < 4 or var == 0.0:
        return float("nan")
    tau = 0.5
    for m in range(1, T // 2):
        tau += float((a[:-m] * a[m:]).mean() / var)
        if m >= window * tau:
            break
    return tau


def binned_error(series, nbins=10):
    series = np.asarray(series, dtype=np.float64)
    nb = min(nbins, len(series))
    if nb < 2:
        return float("nan")
    means = np.array([b.mean() for b in np.array_split(series, nb)])
    return float(means.std(ddof=1) / math.sqrt(nb))


def initial_fields(init, chains, Lx, L, alpha, seed):
    """Starting fields: iid N(0, 1) ("gaussian"), or the checkerboard CDW state at the minima
    of the double well, alpha (-1)^(ix+iy) + N(0, 0.3^2) ("cdw": the ordered state the model
    develops below T_c, so that chains near the transition need not order first), or a given
    tensor [chains, N, L] (a warm start from another run's final fields, copied)."""
    if torch.is_tensor(init):
        if tuple(init.shape) != (chains, Lx * Lx, L):
            raise ValueError("initial fields of shape %s, expected %s" % (tuple(init.shape), (chains, Lx * Lx, L)))
        return init.detach().to(torch.float64).cpu().clone()
    if init == "cdw":
        return torch.from_numpy(inputs.cdw_fields(chains, Lx, Lx, L, amp=alpha, noise=0.3, seed=seed))
    return torch.from_numpy(inputs.gaussian_fields(chains, Lx, Lx, L, sigma=1.0, seed=seed))


def dqmc_configurations(ctx, x, therm, gap, count, sweep0=0):
    """Thermalise the DQMC chains x in place for `therm` sweeps, then take `count` snapshots
    of every chain, `gap` sweeps apart. Returns the stacked snapshots, the sweep counter
    reached and the local acceptance."""
    chains = x.shape[0]
    n_loc = torch.zeros(chains, dtype=torch.int64, device=x.device)
    ctx.dqmc_sweep(x, therm, sweep0=sweep0, n_acc_local=n_loc)
    snaps = []
    ctr = sweep0 + therm
    for _ in range(count):
        ctx.dqmc_sweep(x, gap, sweep0=ctr, n_acc_local=n_loc)
        ctr += gap
        snaps.append(x.clone())
    moves = chains * (therm + gap * count) * ctx.N * ctx.L
    return torch.cat(snaps), ctr, float(n_loc.sum().item()) / max(moves, 1)


def run_dqmc(Lx, L, n_s=8, chains=32, sweeps=500, precision="fp64", dtau=0.1, lam=1.0, omega0=1.0,
             sweep_delta=0.5, seed=0x1802061774, device="cuda", rank=0, world=1, nblock=0, init="gaussian",
             want_series=False, return_fields=False):
    """Conventional DQMC chains: S(pi, pi) from G after every sweep, its integrated
    autocorrelation time in sweeps and the time per sweep (want_series: also the per-sweep,
    per-chain S(pi, pi) and the acceptance counts of this process; return_fields: also the final
    fields as a device tensor under "x_final")."""
    dev = torch.device(device)
    seed = seed + rank
    ctx = Context(Lx, Lx, L, dtau=dtau, lam=lam, omega0=omega0, n_s=n_s, precision=precision,
                  sweep_delta=sweep_delta, seed=seed, max_fields=chains, device=dev)
    x = initial_fields(init, chains, Lx, L, lam / omega0 ** 2, seed).to(dev)
    n_loc = torch.zeros(chains, dtype=torch.int64, device=dev)
    n_blk = torch.zeros(chains, dtype=torch.int64, device=dev)
    G = torch.empty(chains, ctx.N, ctx.N, dtype=torch.float64, device=dev)
    obs = torch.empty(sweeps, chains, dtype=torch.float64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sweep_ms = 0.0
    for k in range(sweeps):
        e0.record()
        ctx.dqmc_sweep(x, 1, sweep0=k, nblock=nblock, n_acc_local=n_loc, n_acc_block=n_blk)
        e1.record()
        ctx.greens(x, G)
        obs[k] = ctx.measure_cdw(G)
        torch.cuda.synchronize()
        sweep_ms += e0.elapsed_time(e1)
    ctx.get_error()
    therm = sweeps // 5
    tau = integrated_autocorrelation(obs.cpu().numpy()[therm:])
    S_sum = sum_over_processes(obs.sum(dim=1))
    acc = sum_over_processes(torch.stack([n_loc.sum(), n_blk.sum()]))
    series = (S_sum / (chains * world)).cpu().numpy()[therm:]
    N = Lx * Lx
    res = {"method": "dqmc", "lattice": "%dx%d" % (Lx, Lx), "N": N, "L": L, "beta": L * dtau, "n_s": n_s,
           "lambda": lam, "omega0": omega0, "chains": chains * world, "sweeps": sweeps, "block_updates": nblock,
           "S_pipi_mean": float(series.mean()), "S_pipi_err": binned_error(series),
           "S_pipi_tau_int_sweeps": tau, "S_pipi_halves": [float(h.mean()) for h in np.array_split(series, 2)],
           "local_acceptance": float(acc[0].item()) / (chains * world * sweeps * N * L),
           "block_acceptance": float(acc[1].item()) / max(1, chains * world * sweeps * nblock),
           "ms_per_sweep": sweep_ms / sweeps, "chain_sweeps_per_s": chains * world * sweeps / (sweep_ms / 1e3),
           "ms_per_independent_sample": 2.0 * tau * sweep_ms / sweeps}
    if want_series:
        res["S_series"] = obs.cpu().numpy().tolist()
        res["accepted_local"] = n_loc.cpu().numpy().tolist()
        res["accepted_block"] = n_blk.cpu().numpy().tolist()
    if return_fields:
        res["x_final"] = x.clone()
    ctx.close()
    return res


def run(Lx, L, n_s=8, chains=32, train=2000, updates=500, sweeps=100, precision="fp32", dtau=0.1, lam=1.0,
        omega0=1.0, sweep_delta=0.3, seed=0x1802061774, rounds=2, device="cuda", rank=0, world=1, wolff=0,
        train_source="self", dqmc_therm=50, dqmc_gap=5, init="gaussian", J0=None, want_series=False,
        return_fields=False):
    """One SLMC run: self-learning (or DQMC) training of E_eff, then `updates` cumulative updates
    of every chain measuring S(pi, pi) after each (want_series: also the per-update, per-chain
    S(pi, pi), the acceptance counts and the couplings of every training round; return_fields:
    also the chains' final fields as a device tensor under "x_final", e.g. to warm-start DQMC)."""
    dev = torch.device(device)
    seed = seed + rank
    ctx = Context(Lx, Lx, L, dtau=dtau, lam=lam, omega0=omega0, n_s=n_s, precision=precision,
                  sweep_delta=sweep_delta, seed=seed, max_fields=chains, device=dev)
    ctx.set_wolff(wolff)  # Wolff cluster updates between the colours of every sweep
    N = Lx * Lx
    x = initial_fields(init, chains, Lx, L, lam / omega0 ** 2, seed).to(dev)
    J = torch.tensor([0.0, omega0 ** 2 / 4 + 1.0 / (2 * dtau ** 2), 0.1, 0.0, 0.0, omega0 ** 2 / 2] if J0 is None
                     else list(J0), dtype=torch.float64, device=dev)
    t0 = time.perf_counter()
    lnw, s = ctx.chain_init(x)
    ctx.set_update_counter(0)
    # ---- self-learning rounds: generate configurations with the current couplings, refit ----
    per_round = max(1, math.ceil(train / (chains * world)))
    history = []
    sweep_ctr = 1 << 30  # training proposals use Philox sweep counters far from the production ones
    xp = None
    if train_source == "dqmc":  # the paper's training data: equilibrated DQMC configurations
        xd = x.clone()
        X, _, dacc = dqmc_configurations(ctx, xd, dqmc_therm, dqmc_gap, per_round, sweep0=1 << 40)
        Y, _, _ = ctx.log_weight(X)
        J, resid = fit_eff_distributed(ctx, X.contiguous(), Y.contiguous())
        history.append({"round": "dqmc", "configs": int(X.shape[0]) * world, "dqmc_thermalisation": dqmc_therm,
                        "dqmc_gap": dqmc_gap, "dqmc_local_acceptance": dacc, "J": J.cpu().tolist(),
                        "rms_resid": float(resid.item())})
        x = xd  # the self-learning rounds and production start from the DQMC chains
        xp = xd
        del X, Y
        rounds = max(0, rounds - 1)
    for r in range(rounds):
        xs, ys = [], []
        xp = x.clone()
        n_sw = torch.zeros(chains, dtype=torch.int64, device=dev)
        for u in range(per_round):
            ctx.eff_sweep(xp, J, sweeps, sweep0=sweep_ctr, first_colour=u & 1, n_acc=n_sw)
            sweep_ctr += sweeps
            lw_p, _, _ = ctx.log_weight(xp)
            xs.append(xp.clone())
            ys.append(lw_p)
        X = torch.cat(xs)
        Y = torch.cat(ys)
        J, resid = fit_eff_distributed(ctx, X.contiguous(), Y.contiguous())
        sw = sum_over_processes(torch.stack([n_sw.sum(), torch.tensor(X.shape[0], device=dev)]))
        history.append({"round": r, "configs": int(sw[1].item()), "sweep_acceptance": float(sw[0].item()) /
                        (chains * world * per_round * sweeps * N * L), "J": J.cpu().tolist(),
                        "rms_resid": float(resid.item())})
        del xs, ys, X, Y
        if r < rounds - 1:
            del xp
    # production starts from the DQMC chains when they trained E_eff (configurations of the exact
    # weight w), else from the last self-generated configurations (inside the training
    # distribution; the initial Gaussian field is atypical for both weights). Near T_c, chains
    # started from E_eff-generated configurations keep a lower S(pi, pi) for thousands of steps.
    if train_source != "dqmc":
        x = xp if xp is not None else x
    x = x.contiguous()
    lnw, s = ctx.chain_init(x)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    # ---- production ----
    ctx.wolff_sites(reset=True)
    n_acc = torch.zeros(chains, dtype=torch.int64, device=dev)
    n_sw = torch.zeros(chains, dtype=torch.int64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    obs = ctx.cumulative_update(x, J, sweeps, updates, UPDATE_CONTINUE, lnw, s, n_acc, n_sw, want_obs=True)
    e1.record()
    torch.cuda.synchronize()
    ctx.get_error()
    ms = e0.elapsed_time(e1)
    tau = integrated_autocorrelation(obs.cpu().numpy()[updates // 5:])  # this process's chains
    wsites = ctx.wolff_sites()
    S_sum = sum_over_processes(obs.sum(dim=1))  # [updates], summed over every process's chains
    acc = sum_over_processes(torch.stack([n_acc.sum(), n_sw.sum()]))
    therm = updates // 5
    series = (S_sum / (chains * world)).cpu().numpy()[therm:]
    res = {
        "lattice": "%dx%d" % (Lx, Lx), "N": N, "L": L, "beta": L * dtau, "n_s": n_s, "precision": precision,
        "chains": chains * world, "processes": world,
        "training_configs": history[-1]["configs"] if history else 0,
        "training_rounds": history,
        "updates": updates, "sweeps_per_update": sweeps,
        "S_pipi_mean": float(series.mean()), "S_pipi_err": binned_error(series),
        "S_pipi_tau_int_updates": tau, "wolff_per_sweep": wolff,
        "S_pipi_halves": [float(h.mean()) for h in np.array_split(series, 2)],  # drift check
        "wolff_mean_cluster": (wsites / (chains * updates * sweeps * wolff)) if wolff else None,
        "acceptance": float(acc[0].item()) / (chains * world * updates),
        "sweep_acceptance": float(acc[1].item()) / (chains * world * updates * sweeps * N * L),
        "production_seconds": ms / 1e3, "training_seconds": t_train,
        "evals_per_s": chains * world * updates / (ms / 1e3), "J_final": J.cpu().tolist(),
    }
    if want_series:
        res["S_series"] = obs.cpu().numpy().tolist()
        res["accepted"] = n_acc.cpu().numpy().tolist()
    if return_fields:
        res["x_final"] = x.clone()
    ctx.close()
    return res


def power_law_exponent(sizes, values):
    """Least-squares slope of ln(value) against ln(size)."""
    lx, ly = np.log(np.asarray(sizes, dtype=np.float64)), np.log(np.asarray(values, dtype=np.float64))
    if len(lx) < 2 or not np.all(np.isfinite(ly)):
        return float("nan")
    return float(np.polyfit(lx, ly, 1)[0])


def autocorrelation_study(sizes, beta=4.1, dtau=0.1, lam=1.0, omega0=0.5, n_s=10, chains=64, steps=2000,
                          sweeps=10, train=1024, seed=0x1802061774, device="cuda", rank=0, world=1, nblock=4,
                          wolff=1, init="cdw", dqmc_therm=200, precision="fp32", want_series=False):
    """Autocorrelation time tau_L of S(pi, pi) against the linear size for DQMC and SLMC with the
    paper's Monte Carlo steps (Sec. "Results"): a DQMC step is a sweep of local updates plus
    `nblock` block updates; an SLMC step is a sweep of local updates of E_eff plus `wolff` Wolff
    cluster updates, so tau in SLMC steps is tau in cumulative updates times `sweeps`. Also the
    GPU time per statistically independent configuration, 2 tau_L times the time per step, and
    the power-law exponents of both against the size. Defaults: the paper's critical point
    (lambda = 0.5 from g = 1, Omega = 0.5; beta = 1 / T_c = 4.1). precision: the slice products of
    the SLMC runs (the DQMC chains are FP64); want_series: the per-step S(pi, pi) of every run."""
    L = 2 * max(1, int(round(beta / (2.0 * dtau))))  # the checkerboard sweeps of E_eff need an even L
    dtau = beta / L
    rows = []
    for Lx in sizes:
        d = run_dqmc(Lx, L, min(n_s, L), chains, steps, "fp64", dtau=dtau, lam=lam, omega0=omega0, seed=seed,
                     device=device, rank=rank, world=world, nblock=nblock, init=init, want_series=want_series)
        m = run(Lx, L, min(n_s, L), chains, train, max(4, steps // sweeps), sweeps, precision, dtau=dtau, lam=lam,
                omega0=omega0, seed=seed, rounds=2, device=device, rank=rank, world=world, wolff=wolff,
                train_source="dqmc", dqmc_therm=dqmc_therm, init=init, want_series=want_series)
        s_ms = 1e3 * m["production_seconds"] / m["updates"] / sweeps  # per SLMC step
        rows.append({"Lx": Lx, "dqmc_tau_steps": d["S_pipi_tau_int_sweeps"], "dqmc_ms_per_step": d["ms_per_sweep"],
                     "dqmc_ms_per_independent": d["ms_per_independent_sample"], "dqmc_S": d["S_pipi_mean"],
                     "dqmc_S_err": d["S_pipi_err"], "dqmc_S_halves": d["S_pipi_halves"],
                     "dqmc_block_acceptance": d["block_acceptance"],
                     "slmc_tau_steps": m["S_pipi_tau_int_updates"] * sweeps, "slmc_ms_per_step": s_ms,
                     "slmc_ms_per_independent": 2.0 * m["S_pipi_tau_int_updates"] * sweeps * s_ms,
                     "slmc_S": m["S_pipi_mean"], "slmc_S_err": m["S_pipi_err"], "slmc_S_halves": m["S_pipi_halves"],
                     "slmc_acceptance": m["acceptance"], "slmc_mean_cluster": m["wolff_mean_cluster"]})
        if want_series:
            rows[-1].update({"dqmc_series": d["S_series"], "dqmc_accepted_local": d["accepted_local"],
                             "dqmc_accepted_block": d["accepted_block"], "slmc_series": m["S_series"],
                             "slmc_accepted": m["accepted"], "slmc_J": m["J_final"]})
    fit = {k: power_law_exponent([r["Lx"] for r in rows], [r[k] for r in rows])
           for k in ("dqmc_tau_steps", "slmc_tau_steps", "dqmc_ms_per_independent", "slmc_ms_per_independent")}
    return {"study": "autocorrelation", "beta": beta, "L": L, "dtau": dtau, "g": lam, "omega0": omega0,
            "lambda_dimensionless": lam ** 2 / (8.0 * omega0 ** 2), "chains": chains * world, "steps": steps,
            "sweeps_per_update": sweeps, "dqmc_block_updates_per_step": nblock, "wolff_per_sweep": wolff,
            "init": init, "slmc_training_dqmc_thermalisation": dqmc_therm,
            "sizes": rows, "exponents": fit}


def crossings(sizes, temps, curves):
    """Temperatures where the curves of consecutive sizes cross (linear interpolation between the
    scanned temperatures where their difference changes sign)."""
    out = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        d = [curves[b][k] - curves[a][k] for k in range(len(temps))]
        for k in range(len(temps) - 1):
            if d[k] == 0.0 or d[k] * d[k + 1] < 0.0:
                f = d[k] / (d[k] - d[k + 1]) if d[k] != d[k + 1] else 0.0
                out.append({"sizes": [a, b], "T": temps[k] + f * (temps[k + 1] - temps[k])})
    return out


def fss_scan(sizes, betas, dtau=0.1, lam=1.0, omega0=0.5, n_s=10, chains=64, updates=300, sweeps=10, train=1024,
             dqmc_therm=300, seed=0x1802061774, device="cuda", rank=0, world=1, wolff=1, precision="fp32",
             want_series=False):
    """Finite-size scaling of the CDW structure factor (Sec. "Results", Fig. 3(a)): S(pi, pi) L^{-7/4}
    against T for each linear size L, whose crossings estimate T_c (2D Ising: 2 beta/nu = 1/4). Per
    size, E_eff is learned once from DQMC configurations at the middle inverse temperature (the
    paper's training data); the cumulative updates at the other temperatures stay exact with those
    couplings and only accept less often. Inverse temperatures are multiples of 2 dtau (the E_eff
    checkerboard needs an even number of slices); every run starts from the CDW state. precision:
    the slice products of the SLMC runs; want_series: the per-update S(pi, pi) of every run."""
    betas = sorted(betas)
    Ls = [2 * max(1, int(round(b / (2.0 * dtau)))) for b in betas]
    mid = Ls[len(Ls) // 2]
    rows, curves, training = [], {}, {}
    temps = [1.0 / (l * dtau) for l in Ls]
    for Lx in sizes:
        # DQMC fit, then one self-learning refinement (as in the autocorrelation study)
        tr = run(Lx, mid, min(n_s, mid), chains, train, 4, sweeps, precision, dtau=dtau, lam=lam, omega0=omega0,
                 seed=seed, rounds=2, device=device, rank=rank, world=world, wolff=wolff, train_source="dqmc",
                 dqmc_therm=dqmc_therm, init="cdw")
        training[Lx] = {"rms_resid": [h["rms_resid"] for h in tr["training_rounds"]], "J": tr["J_final"],
                        "acceptance_at_training_beta": tr["acceptance"]}
        curves[Lx] = []
        for L, T in zip(Ls, temps):
            m = run(Lx, L, min(n_s, L), chains, 0, updates, sweeps, precision, dtau=dtau, lam=lam, omega0=omega0,
                    seed=seed + 7919 * L, rounds=0, device=device, rank=rank, world=world, wolff=wolff,
                    init="cdw", J0=tr["J_final"], want_series=want_series)
            y = m["S_pipi_mean"] * Lx ** (-1.75)
            curves[Lx].append(y)
            rows.append({"Lx": Lx, "L": L, "beta": L * dtau, "T": T, "S_pipi": m["S_pipi_mean"],
                         "S_pipi_err": m["S_pipi_err"], "S_L_minus_7_4": y, "S_L_minus_7_4_err":
                         m["S_pipi_err"] * Lx ** (-1.75), "S_halves": m["S_pipi_halves"],
                         "tau_int_updates": m["S_pipi_tau_int_updates"], "acceptance": m["acceptance"],
                         "production_seconds": m["production_seconds"]})
            if want_series:
                rows[-1].update({"series": m["S_series"], "accepted": m["accepted"], "J": tr["J_final"]})
    return {"study": "fss", "g": lam, "omega0": omega0, "lambda_dimensionless": lam ** 2 / (8.0 * omega0 ** 2),
            "dtau": dtau, "chains": chains * world, "updates": updates, "sweeps_per_update": sweeps,
            "wolff_per_sweep": wolff, "training_beta": mid * dtau, "training": training, "temperatures": temps,
            "points": rows,
            "crossings": crossings(list(sizes), temps, curves)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--Lx", type=int, default=24)
    ap.add_argument("--L", type=int, default=240)
    ap.add_argument("--n-s", type=int, default=8)
    ap.add_argument("--chains", type=int, default=32)
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--updates", type=int, default=500)
    ap.add_argument("--sweeps", type=int, default=100)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--rounds", type=int, default=2)
    ap.add_argument("--wolff", type=int, default=0, help="Wolff cluster updates per sweep")
    ap.add_argument("--lam", type=float, default=1.0, help="electron-phonon coupling g")
    ap.add_argument("--omega0", type=float, default=1.0, help="phonon frequency")
    ap.add_argument("--seed", type=int, default=0x1802061774)
    ap.add_argument("--train-source", default="self", choices=["self", "dqmc"],
                    help="training configurations: self-generated proposals, or DQMC chains (the paper's way)")
    ap.add_argument("--dqmc-therm", type=int, default=50, help="DQMC thermalisation sweeps before the training set")
    ap.add_argument("--dqmc-gap", type=int, default=5, help="DQMC sweeps between training configurations")
    ap.add_argument("--dqmc-only", action="store_true", help="run DQMC chains and measure S(pi,pi) every sweep")
    ap.add_argument("--dqmc-block", type=int, default=0, help="DQMC block updates per sweep (--dqmc-only)")
    ap.add_argument("--autocorr", default=None,
                    help="comma-separated linear sizes: tau_L of S(pi,pi) for DQMC and SLMC (paper's MC steps)")
    ap.add_argument("--beta", type=float, default=4.1, help="--autocorr: inverse temperature")
    ap.add_argument("--fss", default=None, help="comma-separated linear sizes: S(pi,pi) L^-7/4 against T")
    ap.add_argument("--betas", default="3.6,3.8,4.0,4.2,4.4,4.6", help="--fss: inverse temperatures")
    ap.add_argument("--steps", type=int, default=2000, help="--autocorr: MC steps per method and size")
    ap.add_argument("--init", default=None, choices=["gaussian", "cdw"],
                    help="starting fields (default gaussian; cdw for --autocorr)")
    ap.add_argument("--sweep-delta", type=float, default=None,
                    help="proposal width (default 0.3 for E_eff sweeps, 0.5 for DQMC sweeps)")
    a = ap.parse_args()
    import os
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if a.fss:
        res = fss_scan([int(v) for v in a.fss.split(",")], [float(v) for v in a.betas.split(",")], lam=a.lam,
                       omega0=a.omega0, n_s=a.n_s, chains=a.chains, updates=a.updates, sweeps=a.sweeps,
                       train=a.train, dqmc_therm=a.dqmc_therm, seed=a.seed, device="cuda:%d" % local, rank=rank,
                       world=world, wolff=a.wolff if a.wolff else 1)
    elif a.autocorr:
        res = autocorrelation_study([int(v) for v in a.autocorr.split(",")], beta=a.beta, lam=a.lam,
                                    omega0=a.omega0, n_s=a.n_s, chains=a.chains, steps=a.steps, sweeps=a.sweeps,
                                    train=a.train, seed=a.seed, device="cuda:%d" % local, rank=rank, world=world,
                                    nblock=a.dqmc_block if a.dqmc_block else 4, wolff=a.wolff if a.wolff else 1,
                                    init=a.init or "cdw", dqmc_therm=a.dqmc_therm)
    elif a.dqmc_only:
        res = run_dqmc(a.Lx, a.L, a.n_s, a.chains, a.updates, "fp64", lam=a.lam, omega0=a.omega0,
                       sweep_delta=0.5 if a.sweep_delta is None else a.sweep_delta, seed=a.seed,
                       device="cuda:%d" % local, rank=rank, world=world, nblock=a.dqmc_block,
                       init=a.init or "gaussian")
    else:
        res = run(a.Lx, a.L, a.n_s, a.chains, a.train, a.updates, a.sweeps, a.precision, rounds=a.rounds,
                  device="cuda:%d" % local, rank=rank, world=world, wolff=a.wolff, lam=a.lam, omega0=a.omega0,
                  seed=a.seed, sweep_delta=0.3 if a.sweep_delta is None else a.sweep_delta,
                  train_source=a.train_source, dqmc_therm=a.dqmc_therm, dqmc_gap=a.dqmc_gap,
                  init=a.init or "gaussian")
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
