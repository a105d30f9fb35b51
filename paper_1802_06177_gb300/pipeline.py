"""Self-learning Monte Carlo for the 2D Holstein model end to end on one GPU (every step runs
in libslmc's kernels; this module only sequences the calls and reduces the measurements).

Steps (Sec. "SLMC" and Suppl. Sec. "SLMC for the Holstein model"):
  1. start from the bare phonon action written in the E_eff basis (exact at lambda = 0:
     J_k = omega0^2/4 + 1/(2 dtau^2), J_nn' = omega0^2/2) plus a small double-well term;
  2. self-learning: propose configurations with effective-model sweeps under the current
     couplings (the proposals of the cumulative update), score each with the exact ln w and
     refit E_eff on them (Eq. (5)) -- the training data is generated by the method itself,
     since the DQMC configurations of the paper are not available -- and repeat;
  3. production: cumulative updates (Eq. (6)) with the learned couplings, measuring the CDW
     structure factor S(pi, pi) after every update and counting acceptances.
Error bars: the per-chain time series are averaged over chains, then binned in time.
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


def run(Lx, L, n_s=8, chains=32, train=2000, updates=500, sweeps=100, precision="fp32", dtau=0.1, lam=1.0,
        omega0=1.0, sweep_delta=0.3, seed=0x1802061774, rounds=2, device="cuda", rank=0, world=1, wolff=0):
    dev = torch.device(device)
    seed = seed + rank
    ctx = Context(Lx, Lx, L, dtau=dtau, lam=lam, omega0=omega0, n_s=n_s, precision=precision,
                  sweep_delta=sweep_delta, seed=seed, max_fields=chains, device=dev)
    ctx.set_wolff(wolff)  # Wolff cluster updates between the colours of every sweep
    N = Lx * Lx
    x = torch.from_numpy(inputs.gaussian_fields(chains, Lx, Lx, L, sigma=1.0, seed=seed)).to(dev)
    J = torch.tensor([0.0, omega0 ** 2 / 4 + 1.0 / (2 * dtau ** 2), 0.1, 0.0, 0.0, omega0 ** 2 / 2],
                     dtype=torch.float64, device=dev)
    t0 = time.perf_counter()
    lnw, s = ctx.chain_init(x)
    ctx.set_update_counter(0)
    # ---- self-learning rounds: generate configurations with the current couplings, refit ----
    per_round = max(1, math.ceil(train / (chains * world)))
    history = []
    sweep_ctr = 1 << 30  # training proposals use Philox sweep counters far from the production ones
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
    # production starts from the last self-generated configurations (inside the training
    # distribution); the initial Gaussian field is atypical for both weights
    x = xp.contiguous()
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
        "chains": chains * world, "processes": world, "training_configs": history[-1]["configs"],
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
    ctx.close()
    return res


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
    a = ap.parse_args()
    import os
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    res = run(a.Lx, a.L, a.n_s, a.chains, a.train, a.updates, a.sweeps, a.precision, rounds=a.rounds,
              device="cuda:%d" % local, rank=rank, world=world, wolff=a.wolff, lam=a.lam, omega0=a.omega0,
              seed=a.seed)
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
