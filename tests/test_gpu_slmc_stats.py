"""SLMC observables of the GPU chain in mixed precision (FP32 slices) agree with those of the
FP64 oracle chain: the CDW structure factor S(pi, pi) and the cumulative-update acceptance rate
on the 4x4, beta = 4 (L = 40) lattice.

Paired design: GPU chain c and oracle chain c start from the same field and draw the same
Philox streams, so their S(pi, pi) series can be compared update by update; mixed precision
changes ln w by ~1e-5, which can flip an acceptance only very rarely. Error bars of the
ensemble means are taken from the chain-to-chain spread (chains are independent; updates
within a chain are autocorrelated)."""
import math

import numpy as np
import pytest
import torch

from oracle import HolsteinParams
from oracle.chain import cumulative_update
from oracle.lattice import exp_hopping
from oracle.observables import s_cdw
from oracle.weight import log_weight
from paper_1802_06177_gb300 import inputs
from tests.gpu_util import cuda, make_ctx, require_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

J = np.array([0.0, 50.25, 0.3, 0.0, 0.02, 0.45])
SEED, DELTA, NSW = 0x1802061770, 0.35, 10


def test_observables_match_oracle_chain():
    require_gpu()
    Lx, L, n_s = 4, 40, 10
    nch, nup = 6, 120
    x0 = inputs.gaussian_fields(nch, Lx, Lx, L, sigma=0.5, seed=1)
    ctx = make_ctx(Lx, L, n_s, precision="fp32", max_fields=nch, seed=SEED, sweep_delta=DELTA)
    x = cuda(x0.copy())
    lnw, s = ctx.chain_init(x)
    n_acc = torch.zeros(nch, dtype=torch.int64, device="cuda")
    obs = ctx.cumulative_update(x, cuda(J), NSW, nup, 0, lnw, s, n_acc, want_obs=True)
    torch.cuda.synchronize()
    g = obs.cpu().numpy()  # [update][chain]
    p = HolsteinParams(Lx, Lx, L, n_s=n_s)
    E = exp_hopping(Lx, Lx, 1.0, 0.0, 0.1)
    o = np.zeros((nup, nch))
    o_acc = np.zeros(nch)
    for c in range(nch):
        xo = x0[c].copy()
        lw, _, _, G = log_weight(p, xo, E)
        S = s_cdw(p, G)
        for u in range(nup):
            acc, lw, Gn, _ = cumulative_update(p, xo, lw, J[0], J[1:], NSW, u, c, SEED, DELTA, E=E)
            o_acc[c] += acc
            if acc:
                S = s_cdw(p, Gn)
            o[u, c] = S
    # per-chain time averages after thermalisation: ensemble means with chain-to-chain errors
    gm, om = g[20:].mean(axis=0), o[20:].mean(axis=0)
    err = math.sqrt(gm.var(ddof=1) / nch + om.var(ddof=1) / nch)
    assert abs(gm.mean() - om.mean()) <= 3.0 * err + 1e-9, (gm.mean(), om.mean(), err)
    # paired: identical except after a (rare) flipped acceptance
    same = np.mean(np.abs(g - o) < 1e-6)
    assert same > 0.8, same
    g_acc = n_acc.cpu().numpy() / nup
    assert np.abs(g_acc - o_acc / nup).max() <= 0.05
    assert 0.05 < g_acc.mean() < 0.999
