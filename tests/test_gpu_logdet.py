"""Parity of the CUDA determinant path (slmc_logdet / slmc_greens / slmc_log_weight,
called through the C ABI) with the FP64 oracle, element by element on the same seeded
fields. Bar: |d ln det| <= 1e-8 and |d G| <= 1e-9 in FP64 mode."""
import numpy as np
import pytest
import torch

from oracle import HolsteinParams
from oracle.fermion import fermion_logdet
from oracle.lattice import dispersion, exp_hopping, staggered_sign
from oracle.weight import log_weight
from paper_1802_06177_gb300 import inputs
from tests.gpu_util import cuda, make_ctx

pytestmark = pytest.mark.gpu

TOL_LNDET_FP64 = 1e-8
TOL_G_FP64 = 1e-9


def oracle_many(p, x, want_G=True):
    E = exp_hopping(p.Lx, p.Ly, p.t, p.mu, p.dtau)
    out = [fermion_logdet(p, xf, E=E, want_G=want_G) for xf in x]
    return (np.array([o[0] for o in out]), np.array([o[1] for o in out]),
            np.array([o[2] for o in out]) if want_G else None)


@pytest.mark.parametrize("Lx,Ly,L,n_s,nf,kind", [
    (4, 4, 40, 10, 64, "gaussian"),       # small workload, all 64 fields
    (6, 4, 37, 8, 12, "gaussian"),        # Lx != Ly, ragged last group
    (10, 10, 30, 7, 6, "mixed"),          # N = 100: ragged rows per lane
    (12, 12, 120, 10, 6, "mixed"),        # 12x12 workload shape, sampled fields
    (2, 2, 5, 10, 3, "gaussian"),         # L < n_s: one short group
    (4, 4, 16, 1, 4, "gaussian"),         # QR after every slice
])
def test_logdet_and_greens_fp64(Lx, Ly, L, n_s, nf, kind):
    seed = 1000 + Lx * 100 + L
    x = (inputs.gaussian_fields(nf, Lx, Ly, L, seed=seed) if kind == "gaussian"
         else inputs.mixed_fields(nf, Lx, Ly, L, seed=seed))
    ctx = make_ctx(Lx, L, n_s, Ly=Ly, max_fields=64)
    G, lndet, sign = ctx.greens(cuda(x))
    lndet2, sign2 = ctx.logdet(cuda(x))
    torch.cuda.synchronize()
    ctx.get_error()
    p = HolsteinParams(Lx, Ly, L, n_s=n_s)
    l_ref, s_ref, G_ref = oracle_many(p, x)
    assert np.abs(lndet.cpu().numpy() - l_ref).max() <= TOL_LNDET_FP64
    assert np.array_equal(sign.cpu().numpy(), s_ref)
    assert np.abs(G.cpu().numpy() - G_ref).max() <= TOL_G_FP64
    assert np.array_equal(lndet.cpu().numpy(), lndet2.cpu().numpy())
    assert np.array_equal(sign2.cpu().numpy(), s_ref)


def test_batches_larger_than_workspace():
    x = inputs.gaussian_fields(11, 4, 4, 20, seed=5)
    ctx = make_ctx(4, 20, 5, max_fields=4)  # 3 internal batches, last one ragged
    lndet, sign = ctx.logdet(cuda(x))
    l_ref, s_ref, _ = oracle_many(HolsteinParams(4, 4, 20, n_s=5), x, want_G=False)
    assert np.abs(lndet.cpu().numpy() - l_ref).max() <= TOL_LNDET_FP64
    assert np.array_equal(sign.cpu().numpy(), s_ref)


def test_empty_batch_is_noop():
    ctx = make_ctx(4, 10, 5)
    lndet, sign = ctx.logdet(torch.empty((0, 16, 10), dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert lndet.numel() == 0


def test_negative_determinants_match_sign():
    # large dtau and strong fields give negative single-species determinants
    from oracle.fermion import block_matrix
    rng = np.random.default_rng(11)
    x = 3.0 * rng.standard_normal((64, 4, 6))
    ctx = make_ctx(2, 6, 1, dtau=1.0)
    lndet, sign = ctx.logdet(cuda(x))
    p = HolsteinParams(2, 2, 6, dtau=1.0, n_s=1)
    E = exp_hopping(2, 2, 1.0, 0.0, 1.0)
    ref = [np.linalg.slogdet(block_matrix(E, xf, 1.0, 1.0)) for xf in x]
    s_ref = np.array([int(r[0]) for r in ref])
    assert (s_ref < 0).any()
    assert np.array_equal(sign.cpu().numpy(), s_ref)
    assert np.abs(lndet.cpu().numpy() - np.array([r[1] for r in ref])).max() < 1e-7


def test_closed_forms_on_gpu():
    # lambda = 0 and the static staggered field at the 16x16, L=160 shape
    Lx, L = 16, 160
    eps, _, _ = dispersion(Lx, Lx, 1.0, 0.0)
    ctx0 = make_ctx(Lx, L, 8, lam=0.0, max_fields=2)
    l0, s0 = ctx0.logdet(torch.zeros((1, Lx * Lx, L), dtype=torch.float64, device="cuda"))
    ref0 = np.sum(np.log1p(np.exp(-16.0 * eps)))
    assert abs(l0.item() - ref0) <= TOL_LNDET_FP64 and s0.item() == 1
    m = 0.8
    xs = np.repeat((m * staggered_sign(Lx, Lx))[:, None], L, axis=1)[None]
    ctx = make_ctx(Lx, L, 8, max_fields=2)
    ls, ss = ctx.logdet(cuda(xs))
    theta = np.arccosh(np.cosh(0.1 * m) * np.cosh(0.1 * eps))
    refs = np.sum(np.log(2 * np.cosh(L * theta / 2)))
    assert abs(ls.item() - refs) <= TOL_LNDET_FP64 and ss.item() == 1


def test_atomic_limit_on_gpu():
    x = inputs.gaussian_fields(3, 4, 4, 30, seed=3)
    ctx = make_ctx(4, 30, 7, t=0.0)
    G, lndet, _ = ctx.greens(cuda(x))
    ref = np.sum(np.log1p(np.exp(-0.1 * x.sum(axis=2))), axis=1)
    assert np.abs(lndet.cpu().numpy() - ref).max() <= TOL_LNDET_FP64
    Gd = 1.0 / (1.0 + np.exp(-0.1 * x.sum(axis=2)))
    assert np.abs(G.cpu().numpy() - np.stack([np.diag(g) for g in Gd])).max() <= TOL_G_FP64


def test_log_weight_fp64():
    x = inputs.mixed_fields(6, 6, 6, 24, seed=9)
    ctx = make_ctx(6, 24, 6, lam=1.0, omega0=1.0)
    lnw, lndet, sign = ctx.log_weight(cuda(x))
    p = HolsteinParams(6, 6, 24, n_s=6)
    ref = np.array([log_weight(p, xf)[0] for xf in x])
    assert np.abs(lnw.cpu().numpy() - ref).max() <= 2 * TOL_LNDET_FP64 + 1e-10 * np.abs(ref).max()
    # even in x (particle-hole symmetry of the full weight)
    lnw_m, _, _ = ctx.log_weight(cuda(-x))
    assert np.abs(lnw.cpu().numpy() - lnw_m.cpu().numpy()).max() < 1e-8


def test_full_size_16x16_L160_sampled():
    # The 16x16, beta=16 workload in the launch configuration the benchmark uses (many
    # fields per batch); the oracle checks a sample of them one by one.
    nf = 64
    x = inputs.mixed_fields(nf, 16, 16, 160, seed=0x1802061772)
    ctx = make_ctx(16, 160, 8, max_fields=nf)
    lndet, sign = ctx.logdet(cuda(x))
    torch.cuda.synchronize()
    ctx.get_error()
    p = HolsteinParams(16, 16, 160, n_s=8)
    E = exp_hopping(16, 16, 1.0, 0.0, 0.1)
    for f in (0, 17, nf // 2, nf - 1):
        l_ref, s_ref, _ = fermion_logdet(p, x[f], E=E, want_G=False)
        assert abs(lndet[f].item() - l_ref) <= TOL_LNDET_FP64
        assert sign[f].item() == s_ref


TOL_LNDET_MIXED = 5e-5  # |d ln w| = 2 |d ln det| <= 1e-4


@pytest.mark.parametrize("Lx,L,n_s,nf", [(12, 120, 10, 8), (16, 160, 8, 32), (24, 48, 8, 1), (4, 40, 10, 8),
                                         (24, 240, 8, 2)])
def test_fp32_slices_meet_mixed_bar(Lx, L, n_s, nf):
    # FP32 slice products as D_l (Y + F Y), F = E - I split into two FP32 terms, block-compensated
    # accumulation (FP64 QR / LU): |d ln w| <= 1e-4.
    x = inputs.mixed_fields(max(nf, 2), Lx, Lx, L, seed=21)[:nf]
    ctx = make_ctx(Lx, L, n_s, precision="fp32", max_fields=nf)
    G, lndet, sign = ctx.greens(cuda(x))
    l_ref, s_ref, G_ref = oracle_many(HolsteinParams(Lx, Lx, L, n_s=n_s), x)
    err = np.abs(lndet.cpu().numpy() - l_ref).max()
    assert err <= TOL_LNDET_MIXED, err
    assert np.array_equal(sign.cpu().numpy(), s_ref)
    assert np.abs(G.cpu().numpy() - G_ref).max() <= 1e-6


def test_nonfinite_field_is_reported():
    from paper_1802_06177_gb300.slmc import SlmcError
    x = inputs.gaussian_fields(2, 4, 4, 10, seed=1)
    x[1, 3, 4] = np.nan
    ctx = make_ctx(4, 10, 5)
    lndet, sign = ctx.logdet(cuda(x))
    with pytest.raises(SlmcError) as e:
        ctx.get_error()
    assert e.value.status == 2
    assert np.isnan(lndet[1].item()) and sign[1].item() == 0
    assert np.isfinite(lndet[0].item()) and sign[0].item() == 1
    ctx.get_error()  # cleared


@pytest.mark.parametrize("qr_mode", ["prepivot", "pivoted"])
@pytest.mark.parametrize("Lx,Ly,L,n_s,nf", [(4, 4, 40, 10, 8), (6, 4, 37, 8, 4), (10, 10, 30, 7, 3),
                                            (18, 18, 36, 9, 2), (24, 24, 48, 8, 1)])
def test_both_qr_modes(qr_mode, Lx, Ly, L, n_s, nf):
    # N = 324 and 576 use 16-column panels in the blocked QR; N <= 256 uses 32
    x = inputs.mixed_fields(nf, Lx, Ly, L, seed=77 + L)
    ctx = make_ctx(Lx, L, n_s, Ly=Ly, max_fields=nf, qr_mode=qr_mode)
    G, lndet, sign = ctx.greens(cuda(x))
    torch.cuda.synchronize()
    ctx.get_error()
    l_ref, s_ref, G_ref = oracle_many(HolsteinParams(Lx, Ly, L, n_s=n_s), x)
    assert np.abs(lndet.cpu().numpy() - l_ref).max() <= TOL_LNDET_FP64
    assert np.array_equal(sign.cpu().numpy(), s_ref)
    assert np.abs(G.cpu().numpy() - G_ref).max() <= TOL_G_FP64


@pytest.mark.parametrize("qr_mode", ["prepivot", "pivoted"])
def test_mixed_both_qr_modes(qr_mode):
    x = inputs.mixed_fields(4, 12, 12, 120, seed=5)
    ctx = make_ctx(12, 120, 10, precision="fp32", max_fields=4, qr_mode=qr_mode)
    lndet, sign = ctx.logdet(cuda(x))
    l_ref, s_ref, _ = oracle_many(HolsteinParams(12, 12, 120, n_s=10), x, want_G=False)
    assert np.abs(lndet.cpu().numpy() - l_ref).max() <= TOL_LNDET_MIXED
    assert np.array_equal(sign.cpu().numpy(), s_ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16x9"])
def test_sub_batch_split_is_bit_identical_and_profiled(precision):
    """Splitting a batch over 1-4 forked streams changes only which stream runs a field:
    ln det, sign and G are bit-identical; the profiler counts every field once per launch
    class and the busy time of a class (union of its launch intervals) never exceeds the
    summed launch time."""
    Lx, L, n_s, nf = 6, 24, 6, 130
    x = inputs.mixed_fields(nf, Lx, Lx, L, seed=77)
    ctx = make_ctx(Lx, L, n_s, precision=precision, max_fields=nf)
    out = []
    for nsub in (1, 2, 3, 4):
        ctx.set_sub_batches(nsub)
        ctx.profile(True)
        G, ld, sg = ctx.greens(cuda(x))
        prof = ctx.profile_read_detail()
        ctx.profile(False)
        out.append((G.cpu().numpy(), ld.cpu().numpy(), sg.cpu().numpy()))
        groups = -(-L // n_s)
        # the QR runs as one call per panel of 32 columns (factorisation, "qr") and one per panel
        # but the last (tensor-core trailing update, "qrtc")
        npan = -(-(Lx * Lx) // 32)
        ms, calls, busy, units = prof["qr"]
        assert units == nf * groups * npan and calls == groups * nsub * npan
        assert 0.0 < busy <= ms * (1 + 1e-6) + 1e-3
        ms, calls, busy, units = prof["qrtc"]
        assert units == nf * groups * (npan - 1) and calls == groups * nsub * (npan - 1)
        assert 0.0 < busy <= ms * (1 + 1e-6) + 1e-3
        assert prof["greens"][3] == nf
    ctx.set_sub_batches(3)
    ctx.set_sub_batch_priorities(1)
    G, ld, sg = ctx.greens(cuda(x))
    out.append((G.cpu().numpy(), ld.cpu().numpy(), sg.cpu().numpy()))
    for G, ld, sg in out[1:]:
        assert np.array_equal(G, out[0][0]) and np.array_equal(ld, out[0][1]) and np.array_equal(sg, out[0][2])
    p = HolsteinParams(Lx, Lx, L, n_s=n_s)
    E = exp_hopping(Lx, Lx, 1.0, 0.0, 0.1)
    tol = 1e-8 if precision == "fp64" else 5e-5
    for f in (0, 64, 129):
        ref = fermion_logdet(p, x[f], E=E, want_G=False)[0]
        assert abs(out[0][1][f] - ref) <= tol


def test_slice_column_groups_bit_identical():
    """The thread layouts of the FP32 slice kernel (one or two column groups of 256 row threads,
    four groups of 64 row threads) run the same arithmetic per output element: bit-identical
    results."""
    Lx, L, n_s, nf = 12, 40, 10, 20
    x = inputs.mixed_fields(nf, Lx, Lx, L, seed=91)
    ctx = make_ctx(Lx, L, n_s, precision="fp32", max_fields=nf)
    G2, ld2, _ = ctx.greens(cuda(x))
    for groups in (2, 4):
        ctx.set_slice_groups(groups)
        G1, ld1, _ = ctx.greens(cuda(x))
        assert torch.equal(G1, G2) and torch.equal(ld1, ld2), groups


@pytest.mark.parametrize("Lx,Ly,L,n_s,nf,precision", [(16, 16, 40, 8, 6, "fp64"), (10, 10, 30, 10, 5, "fp32"),
                                                      (6, 6, 12, 6, 3, "fp64"), (24, 24, 24, 8, 2, "fp32")])
def test_qr_cluster_bit_identical(Lx, Ly, L, n_s, nf, precision):
    """The QR on a cluster of 2 or 4 CTAs per field (panels round-robin, reflectors shared
    through distributed shared memory) and the column-split formation of Q do the same
    arithmetic per column as one CTA: bit-identical ln det, sign and G; and they match the
    oracle."""
    x = inputs.mixed_fields(nf, Lx, Ly, L, seed=Lx * 31 + L)
    ctx = make_ctx(Lx, L, n_s, Ly=Ly, precision=precision, max_fields=nf)
    res = []
    for ctas in (1, 2, 4):
        ctx.set_qr_cluster(ctas)
        G, ld, sg = ctx.greens(cuda(x))
        ctx.get_error()
        res.append((G.cpu().numpy(), ld.cpu().numpy(), sg.cpu().numpy()))
    for G, ld, sg in res[1:]:
        assert np.array_equal(G, res[0][0]) and np.array_equal(ld, res[0][1]) and np.array_equal(sg, res[0][2])
    p = HolsteinParams(Lx, Ly, L, n_s=n_s)
    E = exp_hopping(Lx, Ly, 1.0, 0.0, 0.1)
    tol = 1e-8 if precision == "fp64" else 5e-5
    for f in range(nf):
        ref = fermion_logdet(p, x[f], E=E, want_G=False)[0]
        assert abs(res[0][1][f] - ref) <= tol, (f, res[0][1][f], ref)


@pytest.mark.parametrize("Lx,Ly,L,n_s", [(16, 16, 40, 8), (6, 4, 30, 7), (2, 5, 12, 5)])
def test_fp64_separable_and_dense_slices_agree(Lx, Ly, L, n_s):
    # FP64 slices through exp(-dtau K) = e^{dtau mu} E_x kron E_y against the dense products
    # (mu != 0 exercises the scalar factor), both against the oracle.
    x = inputs.mixed_fields(4, Lx, Ly, L, seed=Lx + 7 * L)
    out = {}
    for dense in (0, 1):
        ctx = make_ctx(Lx, L, n_s, Ly=Ly, max_fields=4, mu=0.3)
        ctx.set_dense_slices(dense)
        G, lndet, sign = ctx.greens(cuda(x))
        out[dense] = (G.cpu().numpy(), lndet.cpu().numpy(), sign.cpu().numpy())
    assert np.abs(out[0][1] - out[1][1]).max() <= 1e-10
    assert np.abs(out[0][0] - out[1][0]).max() <= 1e-11
    p = HolsteinParams(Lx, Ly, L, n_s=n_s, mu=0.3)
    E = exp_hopping(Lx, Ly, 1.0, 0.3, 0.1)
    for f in range(4):
        l_ref, s_ref, G_ref = fermion_logdet(p, x[f], E=E)
        assert abs(out[0][1][f] - l_ref) <= TOL_LNDET_FP64 and out[0][2][f] == s_ref
        assert np.abs(out[0][0][f] - G_ref).max() <= 1e-9


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("Lx,Ly,L,n_s,nf", [(4, 4, 40, 10, 6), (6, 4, 37, 8, 3), (10, 10, 30, 7, 3),
                                            (12, 12, 120, 10, 3), (16, 16, 160, 8, 3), (18, 18, 36, 9, 2),
                                            (24, 24, 48, 8, 2)])
def test_tupdate_paths(precision, Lx, Ly, L, n_s, nf):
    """T <- (D^-1 R) P^T T on the tensor cores (exact 7-bit slices, path 0), with FP64 FMAs
    (path 1) and through the tensor kernel's per-tile FP64 fallback (path 2): each within the
    bars of the oracle, and the three within the FP64 bars (1e-8 ln det, 1e-9 G) of one another."""
    x = inputs.mixed_fields(nf, Lx, Ly, L, seed=400 + L)
    ctx = make_ctx(Lx, L, n_s, Ly=Ly, precision=precision, max_fields=nf)
    out = []
    for path in (0, 1, 2):
        ctx.set_tupdate_path(path)
        G, ld, sg = ctx.greens(cuda(x))
        ctx.get_error()
        out.append((G.cpu().numpy(), ld.cpu().numpy(), sg.cpu().numpy()))
    l_ref, s_ref, G_ref = oracle_many(HolsteinParams(Lx, Ly, L, n_s=n_s), x)
    tl, tg = (TOL_LNDET_FP64, TOL_G_FP64) if precision == "fp64" else (TOL_LNDET_MIXED, 1e-6)
    for G, ld, sg in out:
        assert np.abs(ld - l_ref).max() <= tl
        assert np.array_equal(sg, s_ref)
        assert np.abs(G - G_ref).max() <= tg
    for G, ld, sg in out[1:]:
        assert np.abs(ld - out[0][1]).max() <= TOL_LNDET_FP64
        assert np.abs(G - out[0][0]).max() <= TOL_G_FP64


@pytest.mark.parametrize("precision", ["fp64", "bf16x9"])
@pytest.mark.parametrize("Lx,Ly,L,n_s,nf", [(4, 4, 40, 10, 6), (6, 4, 37, 8, 3), (10, 10, 30, 7, 3),
                                            (12, 12, 120, 10, 3), (16, 16, 160, 8, 3), (18, 18, 36, 9, 2),
                                            (24, 24, 48, 8, 2)])
def test_qr_paths(precision, Lx, Ly, L, n_s, nf):
    """The pre-pivoted blocked QR with its trailing updates on the tensor cores (exact 7-bit
    slices of C, V and W', path 0) and with FP64 FMAs (path 1): each within the bars of the
    oracle, and in FP64 mode the two within the FP64 bars (1e-8 ln det, 1e-9 G) of each other. The shapes span
    one to five panels of 32 (16 above N = 256) columns, ragged last panels and row tiles, and two
    accumulator segments of W = V^T C (N = 576 > 448 rows)."""
    x = inputs.mixed_fields(nf, Lx, Ly, L, seed=500 + L)
    ctx = make_ctx(Lx, L, n_s, Ly=Ly, precision=precision, max_fields=nf)
    out = []
    for path in (0, 1):
        ctx.set_qr_path(path)
        G, ld, sg = ctx.greens(cuda(x))
        ctx.get_error()
        out.append((G.cpu().numpy(), ld.cpu().numpy(), sg.cpu().numpy()))
    l_ref, s_ref, G_ref = oracle_many(HolsteinParams(Lx, Ly, L, n_s=n_s), x)
    tl, tg = (TOL_LNDET_FP64, TOL_G_FP64) if precision == "fp64" else (TOL_LNDET_MIXED, 1e-6)
    for G, ld, sg in out:
        assert np.abs(ld - l_ref).max() <= tl
        assert np.array_equal(sg, s_ref)
        assert np.abs(G - G_ref).max() <= tg
    # FP64 mode: the two paths agree to the FP64 bars. Mixed modes cut Q into reduced-precision
    # slices, where a rounding-level change of Q moves the result by up to a few 1e-7.
    xl, xg = (TOL_LNDET_FP64, TOL_G_FP64) if precision == "fp64" else (TOL_LNDET_MIXED / 10, 1e-7)
    assert np.abs(out[0][1] - out[1][1]).max() <= xl
    assert np.abs(out[0][0] - out[1][0]).max() <= xg
