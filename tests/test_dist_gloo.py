"""The multi-process exchange of a multi-GPU run, on CPU ranks (gloo, world size 2):
partial regression states are all-gathered in rank order, every rank merges the same
stacked states, and accumulators are summed. The per-rank libslmc context is replaced by a
stand-in with the same two methods whose state is the normal-equation sums of its rows, so
the test checks the protocol: a fit over both ranks' data, identical on both ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


class _NormalEquationsCtx:
    """State = [Phi^T Phi (36), Phi^T y (6), count, padding] of the rows [1, F(x)]."""

    def fit_eff_state(self, xs, lnw):
        phi = torch.cat([torch.ones(xs.shape[0], 1, dtype=torch.float64), xs], dim=1)
        st = torch.zeros(64, dtype=torch.float64)
        st[:36] = (phi.T @ phi).reshape(-1)
        st[36:42] = phi.T @ lnw
        st[42] = xs.shape[0]
        return st

    def fit_eff_merge(self, states):
        tot = states.sum(dim=0)
        A = tot[:36].reshape(6, 6)
        b = tot[36:42]
        return torch.linalg.solve(A, b), states.clone()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    from paper_1802_06177_gb300.dist import fit_eff_distributed, gather_states, sum_over_processes
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(100 + rank)
        n = 7 + 5 * rank  # uneven shares
        xs = torch.from_numpy(rng.standard_normal((n, 5)))
        coef = torch.tensor([0.5, -1.0, 2.0, 0.25, 3.0, -0.75], dtype=torch.float64)
        y = coef[0] + xs @ coef[1:]
        J, states = fit_eff_distributed(_NormalEquationsCtx(), xs, y)
        g = gather_states(torch.full((64,), float(rank + 1), dtype=torch.float64))
        acc = sum_over_processes(torch.tensor([n, 10 * rank], dtype=torch.int64))
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), J=J.numpy(), states=states.numpy(), g=g.numpy(),
                 acc=acc.numpy(), coef=coef.numpy())
    finally:
        dist.destroy_process_group()


def test_fit_exchange_two_gloo_ranks(tmp_path):
    if not dist.is_available():
        pytest.skip("torch.distributed unavailable")
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / ("rank%d.npz" % k)) for k in range(world)]
    # both ranks hold identical couplings, which fit the data of both ranks
    assert np.array_equal(r[0]["J"], r[1]["J"])
    assert np.allclose(r[0]["J"], r[0]["coef"], rtol=1e-10, atol=1e-10)
    # states arrive in rank order, the same on every rank
    assert np.array_equal(r[0]["states"], r[1]["states"])
    assert r[0]["states"][0, 42] == 7 and r[0]["states"][1, 42] == 12
    for k in range(world):
        assert np.array_equal(r[k]["g"], np.stack([np.full(64, 1.0), np.full(64, 2.0)]))
        assert list(r[k]["acc"]) == [19, 10]


def test_single_process_exchange_is_identity():
    from paper_1802_06177_gb300.dist import gather_states, sum_over_processes
    st = torch.arange(64, dtype=torch.float64)
    g = gather_states(st)
    assert g.shape == (1, 64) and torch.equal(g[0], st)
    t = torch.tensor([3, 4])
    assert torch.equal(sum_over_processes(t), torch.tensor([3, 4]))
