"""Parity of the GPU modified Wolff cluster update (Sec. "Wolff update of the effective
Hamiltonian", Eq. (S9)) with the oracle through the C ABI: with the same Philox streams the
effective-model trajectories with Wolff updates between the colours of every sweep, the
reflected-column totals, and whole cumulative-update chains (Eq. (6)) are identical."""
import numpy as np
import pytest
import torch

from oracle import HolsteinParams
from oracle.chain import cumulative_update, eff_sweeps
from oracle.lattice import exp_hopping
from oracle.observables import s_cdw
from oracle.weight import log_weight
from paper_1802_06177_gb300 import inputs
from tests.gpu_util import cuda, make_ctx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("Lx,Ly,L,nwolff,Jnn", [(4, 4, 40, 1, 0.35), (6, 4, 10, 2, -0.5), (2, 2, 6, 3, 0.8),
                                                 (12, 12, 20, 1, 0.2)])
def test_sweeps_with_wolff_reproduce_oracle(Lx, Ly, L, nwolff, Jnn):
    nf, seed, delta, nsweeps, sweep0, first = 3, 0x5EED1234, 0.4, 4, 77, 1
    J = np.array([0.0, 45.0, 0.3, 0.01, Jnn, 0.3])
    # CDW-like fields, so that J_nn F_nn has bonds to activate for either sign of J_nn
    x = inputs.mixed_fields(nf, Lx, Ly, L, seed=Lx * 7 + L)
    ctx = make_ctx(Lx, L, 10, Ly=Ly, seed=seed, sweep_delta=delta)
    ctx.set_wolff(nwolff)
    ctx.wolff_sites(reset=True)
    xg = cuda(x.copy())
    n_acc = torch.zeros(nf, dtype=torch.int64, device="cuda")
    ctx.eff_sweep(xg, cuda(J), nsweeps, sweep0=sweep0, first_colour=first, n_acc=n_acc)
    total = ctx.wolff_sites()
    p = HolsteinParams(Lx, Ly, L)
    sizes = []
    for f in range(nf):
        xo = x[f].copy()
        na = eff_sweeps(p, xo, J[1:], nsweeps, sweep0, first, f, seed, delta, nwolff=nwolff, wolff_sizes=sizes)
        assert np.array_equal(xg[f].cpu().numpy(), xo)
        assert n_acc[f].item() == na
    assert total == sum(sizes) and len(sizes) == nf * nsweeps * nwolff
    assert max(sizes) > 1  # clusters grow beyond the seed


def test_cumulative_update_with_wolff_matches_oracle_chain():
    Lx, L, n_s, nsweeps, nup, nchains, nwolff = 4, 40, 10, 4, 10, 3, 1
    seed, delta = 0x1802061770, 0.5
    J = np.array([0.0, 45.0, 0.6, 0.0, 0.3, 0.2])
    x0 = inputs.mixed_fields(nchains, Lx, Lx, L, seed=5)
    ctx = make_ctx(Lx, L, n_s, seed=seed, sweep_delta=delta, max_fields=2)  # 2 internal batches
    ctx.set_wolff(nwolff)
    xg = cuda(x0.copy())
    lnw, s = ctx.chain_init(xg)
    n_acc = torch.zeros(nchains, dtype=torch.int64, device="cuda")
    n_sw = torch.zeros(nchains, dtype=torch.int64, device="cuda")
    obs = ctx.cumulative_update(xg, cuda(J), nsweeps, nup, 0, lnw, s, n_acc, n_sw, want_obs=True)
    torch.cuda.synchronize()
    ctx.get_error()
    p = HolsteinParams(Lx, Lx, L, n_s=n_s)
    E = exp_hopping(Lx, Lx, 1.0, 0.0, 0.1)
    for c in range(nchains):
        x = x0[c].copy()
        lw, _, _, G = log_weight(p, x, E)
        S = s_cdw(p, G)
        acc_count = 0
        for u in range(nup):
            acc, lw, Gn, _ = cumulative_update(p, x, lw, J[0], J[1:], nsweeps, u, c, seed, delta, E=E, nwolff=nwolff)
            acc_count += acc
            if acc:
                S = s_cdw(p, Gn)
            assert abs(obs[u, c].item() - S) < 1e-9
        assert np.array_equal(xg[c].cpu().numpy(), x)
        assert abs(lnw[c].item() - lw) < 1e-7
        assert n_acc[c].item() == acc_count
