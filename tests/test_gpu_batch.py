"""Batched chains of uneven lattice size in one captured CUDA graph, the device-side update
counter (checkpoint / resume) and the autotuner, through the C ABI."""
import numpy as np
import pytest
import torch

from paper_1802_06177_gb300 import inputs
from tests.gpu_util import cuda, make_ctx, require_gpu

pytestmark = pytest.mark.gpu

CLASSES = [dict(Lx=4, L=20, n_s=5, nchains=3), dict(Lx=6, L=12, n_s=4, nchains=2), dict(Lx=8, L=16, n_s=8, nchains=2)]
J = [0.0, 45.0, 0.6, 0.0, 0.1, 0.0]
SEED, DELTA, NSW = 0xC0FFEE, 0.5, 3


def chains(cl, seed):
    return cuda(inputs.gaussian_fields(cl["nchains"], cl["Lx"], cl["Lx"], cl["L"], sigma=0.5, seed=seed))


WOLFF = [1, 0, 2]  # Wolff updates per sweep of each class (uneven: queue phases a class skips)


@pytest.mark.parametrize("queue,wolff", [(True, False), (True, True), (False, True)])
def test_graph_rounds_equal_direct_calls(queue, wolff):
    """Rounds of the captured graph -- with the E_eff sweeps of all classes in the persistent
    queue launch, or as per-class kernel sequences -- reproduce successive direct calls bit for bit
    (fields, ln w, S, acceptance counts of the cumulative and of the sweep moves, Wolff sites)."""
    require_gpu()
    from paper_1802_06177_gb300.slmc import UPDATE_CONTINUE, Batch
    rounds = 4
    Jt = torch.tensor(J, dtype=torch.float64, device="cuda")
    # direct calls on standalone contexts
    direct = []
    for q, cl in enumerate(CLASSES):
        ctx = make_ctx(cl["Lx"], cl["L"], cl["n_s"], max_fields=cl["nchains"], seed=SEED, sweep_delta=DELTA)
        if wolff:
            ctx.set_wolff(WOLFF[q])
        x = chains(cl, 10 + q)
        lnw, s = ctx.chain_init(x)
        n_acc = torch.zeros(cl["nchains"], dtype=torch.int64, device="cuda")
        n_sw = torch.zeros(cl["nchains"], dtype=torch.int64, device="cuda")
        ctx.set_update_counter(0)
        for r in range(rounds):
            ctx.cumulative_update(x, Jt, NSW, 1, UPDATE_CONTINUE, lnw, s, n_acc, n_sw)
        torch.cuda.synchronize()
        direct.append((x.cpu().numpy(), lnw.cpu().numpy(), s.cpu().numpy(), n_acc.cpu().numpy(),
                       n_sw.cpu().numpy(), ctx.get_update_counter(), ctx.wolff_sites()))
    # the same through one graph
    b = Batch([dict(cl, seed=SEED, sweep_delta=DELTA, precision="fp64") for cl in CLASSES])
    b.set_sweep_queue(queue)
    state = []
    for q, cl in enumerate(CLASSES):
        ctx = b.context(q)
        if wolff:
            ctx.set_wolff(WOLFF[q])
        x = chains(cl, 10 + q)
        with torch.cuda.stream(b.stream):
            lnw, s = ctx.chain_init(x)
            ctx.set_update_counter(0)
        n_acc = torch.zeros(cl["nchains"], dtype=torch.int64, device="cuda")
        n_sw = torch.zeros(cl["nchains"], dtype=torch.int64, device="cuda")
        b.bind(q, x, Jt, lnw, s, n_acc, n_sw)
        state.append((x, lnw, s, n_acc, n_sw, ctx))
    torch.cuda.synchronize()
    b.capture(NSW, 1)
    b.launch(rounds)
    b.stream.synchronize()
    for q, (x, lnw, s, n_acc, n_sw, ctx) in enumerate(state):
        dx, dl, ds, dn, dsw, dc, dw = direct[q]
        assert np.array_equal(x.cpu().numpy(), dx)
        assert np.array_equal(lnw.cpu().numpy(), dl)
        assert np.array_equal(s.cpu().numpy(), ds)
        assert np.array_equal(n_acc.cpu().numpy(), dn)
        assert np.array_equal(n_sw.cpu().numpy(), dsw) and dsw.min() > 0
        with torch.cuda.stream(b.stream):
            ctx.get_error()
            assert ctx.get_update_counter() == dc == rounds
            assert ctx.wolff_sites() == dw
            assert (dw > 0) == (wolff and WOLFF[q] > 0)
    b.close()


def test_queue_rounds_with_several_updates_per_round():
    """nupdates > 1 per captured round: the queue launch of update u of the round continues the
    sweep counter as the u-th of successive direct updates."""
    require_gpu()
    from paper_1802_06177_gb300.slmc import UPDATE_CONTINUE, Batch
    Jt = torch.tensor(J, dtype=torch.float64, device="cuda")
    cls = CLASSES[:2]
    ref = []
    for q, cl in enumerate(cls):
        ctx = make_ctx(cl["Lx"], cl["L"], cl["n_s"], max_fields=cl["nchains"], seed=SEED, sweep_delta=DELTA)
        x = chains(cl, 40 + q)
        lnw, s = ctx.chain_init(x)
        ctx.set_update_counter(0)
        ctx.cumulative_update(x, Jt, NSW, 6, UPDATE_CONTINUE, lnw, s)
        torch.cuda.synchronize()
        ref.append((x.cpu().numpy(), lnw.cpu().numpy()))
    b = Batch([dict(cl, seed=SEED, sweep_delta=DELTA, precision="fp64") for cl in cls])
    state = []
    for q, cl in enumerate(cls):
        ctx = b.context(q)
        x = chains(cl, 40 + q)
        with torch.cuda.stream(b.stream):
            lnw, s = ctx.chain_init(x)
            ctx.set_update_counter(0)
        b.bind(q, x, Jt, lnw, s)
        state.append((x, lnw))
    torch.cuda.synchronize()
    b.capture(NSW, 3)
    b.launch(2)
    b.stream.synchronize()
    for (x, lnw), (rx, rl) in zip(state, ref):
        assert np.array_equal(x.cpu().numpy(), rx)
        assert np.array_equal(lnw.cpu().numpy(), rl)
    b.close()


def test_queue_wait_runs_out_and_reports_timeout():
    """A queue item made to wait for a completion count that nothing reaches gives up after the
    injected limit (about 1 ms), flags SLMC_ERR_TIMEOUT in every class's context and stops the
    queue; the device stays usable and a re-captured normal round runs clean."""
    require_gpu()
    from paper_1802_06177_gb300.slmc import Batch, SlmcError
    Jt = torch.tensor(J, dtype=torch.float64, device="cuda")
    b = Batch([dict(cl, seed=SEED, sweep_delta=DELTA, precision="fp64") for cl in CLASSES])
    state = []
    for q, cl in enumerate(CLASSES):
        ctx = b.context(q)
        x = chains(cl, 20 + q)
        with torch.cuda.stream(b.stream):
            lnw, s = ctx.chain_init(x)
        b.bind(q, x, Jt, lnw, s)
        state.append(ctx)
    torch.cuda.synchronize()
    b.inject_stall(2_000_000)
    b.capture(NSW, 1)
    b.launch(1)
    b.stream.synchronize()
    for ctx in state:
        with torch.cuda.stream(b.stream):
            with pytest.raises(SlmcError) as e:
                ctx.get_error()
        assert e.value.status == 4  # SLMC_ERR_TIMEOUT
    b.inject_stall(0)
    b.capture(NSW, 1)
    b.launch(2)
    b.stream.synchronize()
    for ctx in state:
        with torch.cuda.stream(b.stream):
            ctx.get_error()
    b.close()


def test_checkpoint_resume_reproduces_trajectory():
    require_gpu()
    from paper_1802_06177_gb300.slmc import UPDATE_CONTINUE
    cl = CLASSES[0]
    Jt = torch.tensor(J, dtype=torch.float64, device="cuda")
    ctx = make_ctx(cl["Lx"], cl["L"], cl["n_s"], max_fields=cl["nchains"], seed=SEED, sweep_delta=DELTA)
    x = chains(cl, 3)
    lnw, s = ctx.chain_init(x)
    ctx.cumulative_update(x, Jt, NSW, 3, 0, lnw, s)
    saved = (x.clone(), lnw.clone(), s.clone(), ctx.get_update_counter())
    ctx.cumulative_update(x, Jt, NSW, 2, UPDATE_CONTINUE, lnw, s)
    ref = (x.cpu().numpy(), lnw.cpu().numpy(), s.cpu().numpy())
    # resume from the checkpoint in a fresh context
    ctx2 = make_ctx(cl["Lx"], cl["L"], cl["n_s"], max_fields=cl["nchains"], seed=SEED, sweep_delta=DELTA)
    x2, lnw2, s2, ctr = saved
    ctx2.set_update_counter(ctr)
    ctx2.cumulative_update(x2, Jt, NSW, 2, UPDATE_CONTINUE, lnw2, s2)
    torch.cuda.synchronize()
    assert ctr == 3 and ctx2.get_update_counter() == 5
    assert np.array_equal(x2.cpu().numpy(), ref[0])
    assert np.array_equal(lnw2.cpu().numpy(), ref[1]) and np.array_equal(s2.cpu().numpy(), ref[2])


@pytest.mark.parametrize("precision,Lx,L", [("fp32", 8, 80), ("fp64", 6, 24)])
def test_autotune_returns_fastest_within_tolerance(precision, Lx, L):
    require_gpu()
    from paper_1802_06177_gb300.slmc import autotune
    r = autotune(Lx, Lx, L, precision=precision, ntune=8, tol=5e-5)
    assert r["n_s"] in (4, 6, 8, 10, 12, 16, 20, 24, 32) and r["n_s"] <= L
    assert r["max_abs_dlndet"] <= 5e-5 and r["sec_per_eval"] > 0 and r["candidates"] >= 5
    # the tuned configuration reproduces the FP64 oracle
    from oracle import HolsteinParams
    from oracle.fermion import fermion_logdet
    x = inputs.gaussian_fields(3, Lx, Lx, L, seed=1)
    ctx = make_ctx(Lx, L, r["n_s"], precision=precision, max_fields=3)
    ctx.set_tuning(r["qr_panel"], r["slice_cols"])
    lndet, _ = ctx.logdet(cuda(x))
    p = HolsteinParams(Lx, Lx, L, n_s=8)
    ref = np.array([fermion_logdet(p, xf, want_G=False)[0] for xf in x])
    assert np.abs(lndet.cpu().numpy() - ref).max() <= 5e-5
