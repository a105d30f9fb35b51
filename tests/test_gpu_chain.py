"""Parity of the CUDA effective-model path with the oracle through the C ABI: features
and ln w_eff, checkerboard sweeps (identical Philox streams, so identical trajectories),
the cumulative update of Eq. (6), the regression of Eq. (5) and S(pi, pi)."""
import numpy as np
import pytest
import torch

from oracle import HolsteinParams
from oracle.chain import cumulative_update, eff_sweeps
from oracle.effective import features, fit_couplings, log_weight_eff
from oracle.fermion import fermion_logdet
from oracle.lattice import exp_hopping
from oracle.observables import s_cdw
from oracle.weight import log_weight
from paper_1802_06177_gb300 import inputs
from tests.gpu_util import cuda, make_ctx

pytestmark = pytest.mark.gpu

J_TEST = np.array([1.5, 50.0, 0.35, -0.02, 0.06, 0.4])  # E0, J_k, J_p, J_p', J_nn, J_nn'


@pytest.mark.parametrize("Lx,Ly,L", [(4, 4, 40), (6, 4, 10), (2, 2, 2), (24, 24, 240)])
def test_features_and_eff_log_weight(Lx, Ly, L):
    nf = 3
    x = inputs.gaussian_fields(nf, Lx, Ly, L, seed=Lx * L)
    ctx = make_ctx(Lx, L, 10, Ly=Ly, lam=1.2, omega0=0.9)
    F = ctx.eff_features(cuda(x)).cpu().numpy()
    lw = ctx.eff_log_weight(cuda(x), cuda(J_TEST)).cpu().numpy()
    p = HolsteinParams(Lx, Ly, L, lam=1.2, omega0=0.9)
    for f in range(nf):
        Fr = features(p, x[f])
        assert np.allclose(F[f], Fr, rtol=1e-12, atol=1e-9 * Lx * Ly * L)
        ref = log_weight_eff(p, x[f], J_TEST[0], J_TEST[1:])
        assert abs(lw[f] - ref) <= 1e-11 * max(1.0, abs(ref))


@pytest.mark.parametrize("Lx,L,nsweeps,first", [(4, 40, 5, 0), (6, 12, 3, 1), (2, 2, 4, 0), (12, 120, 2, 1)])
def test_sweeps_reproduce_oracle_trajectory(Lx, L, nsweeps, first):
    nf, seed, delta = 3, 0xABCDEF12345, 0.45
    x = inputs.gaussian_fields(nf, Lx, Lx, L, seed=77)
    ctx = make_ctx(Lx, L, 10, seed=seed, sweep_delta=delta)
    xg = cuda(x.copy())
    n_acc = torch.zeros(nf, dtype=torch.int64, device="cuda")
    ctx.eff_sweep(xg, cuda(J_TEST), nsweeps, sweep0=123, first_colour=first, n_acc=n_acc)
    p = HolsteinParams(Lx, Lx, L)
    for f in range(nf):
        xo = x[f].copy()
        na = eff_sweeps(p, xo, J_TEST[1:], nsweeps, 123, first, f, seed, delta)
        assert np.array_equal(xg[f].cpu().numpy(), xo)
        assert n_acc[f].item() == na
        assert 0 < na < nsweeps * Lx * Lx * L


def test_sweep_rejects_odd_lattice():
    from paper_1802_06177_gb300.slmc import SlmcError
    ctx = make_ctx(3, 4, 2, Ly=4)
    x = torch.zeros((1, 12, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(SlmcError) as e:
        ctx.eff_sweep(x, cuda(J_TEST), 1)
    assert e.value.status == 5


def test_cumulative_update_matches_oracle_chain():
    # small workload shape: 4x4, L=40, n_s=10; a few chains and updates
    Lx, L, n_s, nsweeps, nup, nchains = 4, 40, 10, 5, 12, 3
    seed, delta = 0x1802061770, 0.5
    J = np.array([0.0, 45.0, 0.6, 0.0, 0.1, 0.0])  # deliberately imperfect: about half rejected
    x0 = inputs.gaussian_fields(nchains, Lx, Lx, L, sigma=0.5, seed=3)
    ctx = make_ctx(Lx, L, n_s, seed=seed, sweep_delta=delta, max_fields=2)  # 2 internal batches
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
        acc_count, sw_count = 0, 0
        for u in range(nup):
            acc, lw, Gn, nsw = cumulative_update(p, x, lw, J[0], J[1:], nsweeps, u, c, seed, delta, E=E)
            acc_count += acc
            sw_count += nsw
            if acc:
                S = s_cdw(p, Gn)
            assert abs(obs[u, c].item() - S) < 1e-9
        assert np.array_equal(xg[c].cpu().numpy(), x)
        assert abs(lnw[c].item() - lw) < 1e-7
        assert n_acc[c].item() == acc_count and n_sw[c].item() == sw_count
    assert 0 < n_acc.sum().item() < nchains * nup


def test_fit_recovers_known_couplings():
    Lx, L = 4, 12
    p = HolsteinParams(Lx, Lx, L)
    rng = np.random.default_rng(2)
    xs = np.stack([rng.standard_normal((16, L)) * rng.uniform(0.5, 1.5) + rng.uniform(-0.3, 0.3)
                   for _ in range(150)])
    y = np.array([log_weight_eff(p, x, J_TEST[0], J_TEST[1:]) for x in xs])
    ctx = make_ctx(Lx, L, 6, max_fields=64)  # 3 batches through the accumulator
    J, resid = ctx.fit_eff(cuda(xs), cuda(y))
    J = J.cpu().numpy()
    assert np.allclose(J, J_TEST, rtol=1e-7, atol=1e-9), J
    assert resid.item() < 1e-7


def test_fit_matches_oracle_lstsq_on_exact_weights():
    Lx, L = 4, 40
    p = HolsteinParams(Lx, Lx, L, n_s=10)
    E = exp_hopping(Lx, Lx, 1.0, 0.0, 0.1)
    rng = np.random.default_rng(5)
    xs = np.stack([rng.standard_normal((16, L)) * rng.uniform(0.3, 1.5) for _ in range(120)])
    y = np.array([log_weight(p, x, E)[0] for x in xs])
    E0r, Jr, rr = fit_couplings(p, xs, y)
    ctx = make_ctx(Lx, L, 10)
    J, resid = ctx.fit_eff(cuda(xs), cuda(y))
    J = J.cpu().numpy()
    ref = np.concatenate(([E0r], Jr))
    # both are backward-stable least-squares solvers; agreement limited by conditioning
    assert np.allclose(J, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max()), (J, ref)
    assert abs(resid.item() - rr) < 1e-6 * max(rr, 1.0)
    assert abs(J[1] - 50.0) < 0.5  # Table S1's J_k


def test_cdw_structure_factor():
    x = inputs.mixed_fields(4, 6, 6, 24, seed=4)
    ctx = make_ctx(6, 24, 6)
    G, _, _ = ctx.greens(cuda(x))
    S = ctx.measure_cdw(G).cpu().numpy()
    p = HolsteinParams(6, 6, 24, n_s=6)
    for f in range(4):
        _, _, Gr = fermion_logdet(p, x[f])
        assert abs(S[f] - s_cdw(p, Gr)) < 1e-9
