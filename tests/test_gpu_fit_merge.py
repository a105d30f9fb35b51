"""The regression of Eq. (5) split into partial states (one per process) and merged, through
the C ABI: the merged couplings equal the fit of all configurations at once and the oracle's
least-squares fit, whatever the split (uneven parts, an empty part, any order)."""
import numpy as np
import pytest
import torch

from oracle import HolsteinParams
from oracle.effective import fit_couplings, log_weight_eff
from oracle.lattice import exp_hopping
from oracle.weight import log_weight
from paper_1802_06177_gb300.dist import fit_eff_distributed
from paper_1802_06177_gb300.slmc import SlmcError
from tests.gpu_util import cuda, make_ctx

pytestmark = pytest.mark.gpu

J_TEST = np.array([1.5, 50.0, 0.35, -0.02, 0.06, 0.4])


def _configs(Lx, L, n, seed):
    rng = np.random.default_rng(seed)
    # parts drawn around different means, so the partial states have far-apart references
    return np.stack([rng.standard_normal((Lx * Lx, L)) * rng.uniform(0.3, 1.5) + rng.uniform(-0.8, 0.8)
                     for _ in range(n)])


def _merge(ctx, xs, y, cuts):
    states = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        states.append(ctx.fit_eff_state(cuda(np.ascontiguousarray(xs[a:b])), cuda(np.ascontiguousarray(y[a:b]))))
    return ctx.fit_eff_merge(torch.stack(states))


def test_merge_recovers_known_couplings():
    Lx, L = 4, 12
    p = HolsteinParams(Lx, Lx, L)
    xs = _configs(Lx, L, 150, 3)
    y = np.array([log_weight_eff(p, x, J_TEST[0], J_TEST[1:]) for x in xs])
    ctx = make_ctx(Lx, L, 6, max_fields=32)  # parts larger than the workspace batch
    J, resid = _merge(ctx, xs, y, [0, 7, 7, 90, 150])  # includes an empty part
    assert np.allclose(J.cpu().numpy(), J_TEST, rtol=1e-7, atol=1e-9)
    assert resid.item() < 1e-7


def test_merge_equals_single_fit_and_oracle():
    Lx, L = 4, 40
    p = HolsteinParams(Lx, Lx, L, n_s=10)
    E = exp_hopping(Lx, Lx, 1.0, 0.0, 0.1)
    xs = _configs(Lx, L, 90, 11)
    y = np.array([log_weight(p, x, E)[0] for x in xs])
    ctx = make_ctx(Lx, L, 10)
    J1, r1 = ctx.fit_eff(cuda(xs), cuda(y))
    J1, r1 = J1.cpu().numpy(), r1.item()
    E0r, Jr, rr = fit_couplings(p, xs, y)
    ref = np.concatenate(([E0r], Jr))
    for cuts in ([0, 90], [0, 1, 90], [0, 30, 31, 60, 90], [0, 45, 45, 90]):
        J, r = _merge(ctx, xs, y, cuts)
        J, r = J.cpu().numpy(), r.item()
        assert np.allclose(J, J1, rtol=1e-8, atol=1e-8 * np.abs(J1).max()), (cuts, J, J1)
        assert abs(r - r1) <= 1e-8 * max(r1, 1.0)
        assert np.allclose(J, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max()), (cuts, J, ref)
        assert abs(r - rr) < 1e-6 * max(rr, 1.0)
    # the order of the parts does not matter beyond rounding
    sa = ctx.fit_eff_state(cuda(xs[:40].copy()), cuda(y[:40].copy()))
    sb = ctx.fit_eff_state(cuda(xs[40:].copy()), cuda(y[40:].copy()))
    Jab = ctx.fit_eff_merge(torch.stack([sa, sb]))[0].cpu().numpy()
    Jba = ctx.fit_eff_merge(torch.stack([sb, sa]))[0].cpu().numpy()
    assert np.allclose(Jab, Jba, rtol=1e-8, atol=1e-8 * np.abs(Jab).max())


def test_state_layout_and_empty_merge():
    Lx, L = 4, 12
    ctx = make_ctx(Lx, L, 6)
    xs = _configs(Lx, L, 9, 5)
    y = np.linspace(-3.0, 4.0, 9)
    st = ctx.fit_eff_state(cuda(xs), cuda(y)).cpu().numpy()
    assert st[55] == 1.0 and st[56] == 9.0 and st[54] == y[0]
    R = st[:49].reshape(7, 7)
    assert np.all(np.tril(R, -1) == 0.0)
    assert np.all(st[57:] == 0.0)
    empty = ctx.fit_eff_state(torch.empty((0, 16, L), dtype=torch.float64, device="cuda"),
                              torch.empty(0, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.all(empty == 0.0)
    # a merge of empty states has no data: SINGULAR is flagged, not a fault
    ctx.fit_eff_merge(torch.zeros((2, 64), dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    with pytest.raises(SlmcError) as e:
        ctx.get_error()
    assert e.value.status == 7  # SLMC_ERR_SINGULAR


def test_fit_eff_distributed_single_process():
    Lx, L = 4, 12
    p = HolsteinParams(Lx, Lx, L)
    xs = _configs(Lx, L, 40, 8)
    y = np.array([log_weight_eff(p, x, J_TEST[0], J_TEST[1:]) for x in xs])
    ctx = make_ctx(Lx, L, 6)
    J, _ = fit_eff_distributed(ctx, cuda(xs), cuda(y))
    assert np.allclose(J.cpu().numpy(), J_TEST, rtol=1e-7, atol=1e-9)
