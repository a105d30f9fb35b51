"""Parity of the GPU conventional DQMC updates (Supplemental Material, Eqs. (S3)-(S6), and the
block update described after them) with the oracle through the C ABI: with the same Philox
streams the fields after local sweeps (fast ratio, Sherman-Morrison update, wrapping,
recomputation every n_s slices) and after column-reflection block updates are identical, and so
are the acceptance counts."""
import numpy as np
import pytest
import torch

from oracle import HolsteinParams
from oracle.dqmc import dqmc_sweeps
from oracle.lattice import exp_hopping
from paper_1802_06177_gb300 import inputs
from paper_1802_06177_gb300.slmc import SlmcError
from tests.gpu_util import cuda, make_ctx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("Lx,Ly,L,n_s,nsweeps,nblock,max_fields", [
    (4, 4, 12, 4, 2, 0, 64),
    (3, 2, 7, 3, 2, 3, 64),    # ragged last group of slices
    (2, 2, 2, 1, 3, 2, 64),    # recomputation at every slice
    (6, 6, 20, 10, 1, 4, 2),   # two internal batches of chains
    (8, 6, 16, 5, 1, 2, 64),
    (13, 13, 6, 3, 1, 1, 64),  # N = 169: G no longer fits in shared memory (kept in global memory)
    (16, 16, 4, 2, 1, 1, 64),  # N = 256, the benchmark lattice
])
def test_dqmc_sweeps_reproduce_oracle(Lx, Ly, L, n_s, nsweeps, nblock, max_fields):
    nf, seed, delta, sweep0 = 3, 0xD0C5EED, 0.7, 11
    x = inputs.mixed_fields(nf, Lx, Ly, L, seed=Lx * 31 + L)
    ctx = make_ctx(Lx, L, n_s, Ly=Ly, seed=seed, sweep_delta=delta, max_fields=max_fields)
    xg = cuda(x.copy())
    nl = torch.zeros(nf, dtype=torch.int64, device="cuda")
    nb = torch.zeros(nf, dtype=torch.int64, device="cuda")
    ctx.dqmc_sweep(xg, nsweeps, sweep0=sweep0, nblock=nblock, n_acc_local=nl, n_acc_block=nb)
    torch.cuda.synchronize()
    p = HolsteinParams(Lx, Ly, L, n_s=n_s)
    E = exp_hopping(Lx, Ly, 1.0, 0.0, p.dtau)
    for f in range(nf):
        xo = x[f].copy()
        a_l, a_b = dqmc_sweeps(p, xo, nsweeps, sweep0, f, seed, delta, nblock=nblock, E=E)
        assert np.array_equal(xg[f].cpu().numpy(), xo)
        assert nl[f].item() == a_l and nb[f].item() == a_b
    assert 0 < nl.sum().item() < nf * nsweeps * p.N * L  # moves accepted and rejected


def test_dqmc_counts_accumulate_and_need_two_slices():
    ctx = make_ctx(2, 4, 2, seed=3, sweep_delta=0.5)
    x = cuda(inputs.mixed_fields(2, 2, 2, 4, seed=1))
    nl = torch.full((2,), 5, dtype=torch.int64, device="cuda")
    ctx.dqmc_sweep(x, 1, n_acc_local=nl)
    assert (nl >= 5).all()
    ctx1 = make_ctx(2, 1, 1, seed=3)
    with pytest.raises(SlmcError):
        ctx1.dqmc_sweep(cuda(inputs.mixed_fields(1, 2, 2, 1, seed=1)), 1)


def test_dqmc_local_updates_are_fp64_in_every_precision_mode():
    # the local updates and the recomputation of G run in FP64 whatever the context's precision
    Lx, L, n_s, nf = 6, 20, 5, 3
    x = inputs.mixed_fields(nf, Lx, Lx, L, seed=9)
    out = []
    for prec in ("fp64", "fp32"):
        ctx = make_ctx(Lx, L, n_s, precision=prec, seed=4, sweep_delta=0.6, max_fields=nf)
        xg = cuda(x.copy())
        nl = torch.zeros(nf, dtype=torch.int64, device="cuda")
        ctx.dqmc_sweep(xg, 2, sweep0=5, n_acc_local=nl)
        torch.cuda.synchronize()
        out.append((xg.cpu().numpy(), nl.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
