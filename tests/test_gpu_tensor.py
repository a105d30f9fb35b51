"""Parity of the tensor-core (tcgen05) slice products with the FP64 oracle through the C ABI.
The QR, D scales, LU and log-det stay FP64.

BF16x9 (exact sliced mode): F and Y are cut into fixed-point BF16 slices and the nine slice
products are summed by level, so that every partial sum on the tensor cores is an integer the
FP32 accumulator holds exactly. It meets the mixed-precision bar |d ln w| <= 1e-4, i.e.
|d ln det| <= 5e-5, on every shape below; and its accumulation is checked to be exact against a
numpy model of the same fixed-point arithmetic.

TF32x3 (the literature's split-TF32 scheme: two TF32 pieces per operand, three products) runs on
the tensor cores' truncating FP32 accumulation, whose one-sided error adds up over the slices of
a chain: it does not meet the bar. Its test is marked as an expected failure against the bar
(strict, so an unexpected pass is reported), and a separate check covers what the mode does
guarantee: the sign, G to 1e-4 and a finite, bounded ln det."""
import numpy as np
import pytest
import scipy.linalg
import torch

from oracle import HolsteinParams
from oracle.fermion import fermion_logdet, logdet_greens_from_udt
from oracle.lattice import exp_hopping
from paper_1802_06177_gb300 import inputs
from tests.gpu_util import cuda, make_ctx

pytestmark = pytest.mark.gpu

TOL_LNDET_MIXED = 5e-5  # |d ln w| = 2 |d ln det| <= 1e-4
TOL_G_MIXED = 1e-6


def _oracle(p, x, want_G=True):
    E = exp_hopping(p.Lx, p.Ly, p.t, p.mu, p.dtau)
    out = [fermion_logdet(p, xf, E=E, want_G=want_G) for xf in x]
    return (np.array([o[0] for o in out]), np.array([o[1] for o in out]),
            np.array([o[2] for o in out]) if want_G else None)


@pytest.mark.parametrize("Lx,Ly,L,n_s,nf", [
    (4, 4, 40, 10, 8),      # small workload shape
    (10, 10, 30, 7, 3),     # N = 100: one 128-row tile, ragged K chunk, ragged last group
    (12, 12, 120, 10, 8),   # 12x12 workload shape
    (16, 16, 160, 8, 32),   # benchmark shape, 32 fields (half Gaussian, half CDW + noise)
    (6, 4, 37, 8, 4),       # Lx != Ly, N = 24
    (18, 18, 36, 9, 2),     # N = 324: three row tiles
    (24, 24, 240, 8, 2),    # large shape: N = 576, beta = 24 (five row tiles)
])
def test_bf16x9_meets_mixed_bar(Lx, Ly, L, n_s, nf):
    x = inputs.mixed_fields(max(nf, 2), Lx, Ly, L, seed=300 + L)[:nf]
    ctx = make_ctx(Lx, L, n_s, Ly=Ly, precision="bf16x9", max_fields=nf)
    G, lndet, sign = ctx.greens(cuda(x))
    torch.cuda.synchronize()
    ctx.get_error()
    l_ref, s_ref, G_ref = _oracle(HolsteinParams(Lx, Ly, L, n_s=n_s), x)
    err = np.abs(lndet.cpu().numpy() - l_ref)
    assert err.max() <= TOL_LNDET_MIXED, err.max()
    assert np.array_equal(sign.cpu().numpy(), s_ref)
    assert np.abs(G.cpu().numpy() - G_ref).max() <= TOL_G_MIXED


def _frexp_floor(m):
    g, e = np.frexp(m)
    return np.where(m > 0, e - 1, 0).astype(np.float64)


def _fixed_slices(v, e, n):
    """Round-to-nearest 7-bit slices of v scaled by 2^(6 - e): v = 2^(e-6) sum_s q_s 2^(-7 s)."""
    r = v * np.exp2(6.0 - e)
    out = []
    for _ in range(n):
        q = np.rint(r)
        out.append(q)
        r = (r - q) * 128.0
    return out


def _sliced_group_model(E, x, dtau, lam):
    """One stabilisation group started from U = I with the fixed-point arithmetic of the BF16x9
    mode: F in four slices per row, Y in three per column, the products f_a y_b (a + b <= 3)
    summed exactly per level a + b (float64 holds these integers exactly), the levels combined
    smallest first in FP32, then Y' = fp32(fp32(Y + F Y) * s_l)."""
    f32 = np.float32
    N, L = x.shape
    F = E - np.eye(N)
    eF = _frexp_floor(np.abs(F).max(axis=1))[:, None]
    Fs = _fixed_slices(F, eF, 4)
    sc = np.exp(-dtau * lam * x).astype(f32)
    Y = np.eye(N, dtype=f32)
    for l in range(L):
        eY = _frexp_floor(np.abs(Y).max(axis=0).astype(np.float64))[None, :]
        Ys = _fixed_slices(Y.astype(np.float64), eY, 3)
        t = np.zeros(Y.shape, f32)
        for lev, w in ((3, 2.0 ** -21), (2, 2.0 ** -14), (1, 2.0 ** -7), (0, 1.0)):
            acc = sum(Fs[a] @ Ys[lev - a] for a in range(4) if 0 <= lev - a < 3)
            t = (t + (acc * w).astype(f32)).astype(f32)
        fy = (t.astype(np.float64) * np.exp2(eF + eY - 12.0)).astype(f32)
        Y = ((Y + fy).astype(f32) * sc[:, l][:, None]).astype(f32)
    return Y.astype(np.float64)


@pytest.mark.parametrize("Lx,L", [(12, 24), (16, 40)])
def test_bf16x9_accumulation_is_exact(Lx, L):
    """With one stabilisation group (n_s = L, started from U = I) the GPU's slice product is the
    fixed-point model's bit for bit if, and only if, the tensor cores added every level exactly:
    the two ln det then agree to FP64 rounding of the final QR and LU (1e-9), while both differ
    from the exact product by far more (a long unstabilised group loses FP32 accuracy), so any
    rounding in the accumulation would show."""
    p = HolsteinParams(Lx, Lx, L, n_s=L)
    E = exp_hopping(Lx, Lx, 1.0, 0.0, 0.1)
    x = inputs.mixed_fields(2, Lx, Lx, L, seed=5)
    ctx = make_ctx(Lx, L, L, precision="bf16x9", max_fields=2)
    # the QR and LU of the model are scipy's FP64 ones: compare with the FP64 QR path (the
    # tensor-core trailing updates err normwise, which this unstabilised group of L slices,
    # far worse conditioned than any stabilisation interval, turns into ~1e-8 of ln det)
    ctx.set_qr_path(1)
    lndet, sign = ctx.logdet(cuda(x))
    torch.cuda.synchronize()
    ctx.get_error()
    for f in range(2):
        Y = _sliced_group_model(E, x[f], p.dtau, p.lam)
        Q, R, P = scipy.linalg.qr(Y, pivoting=True)
        D = np.abs(np.diag(R))
        l_model = logdet_greens_from_udt(Q, D, (R / D[:, None])[:, np.argsort(P)])[0]
        l_exact = fermion_logdet(p, x[f], E=E, want_G=False)[0]
        assert abs(l_model - l_exact) > 1e-6  # the comparison below is sensitive
        assert abs(lndet[f].item() - l_model) <= 1e-9, (f, lndet[f].item() - l_model)


def test_bf16x9_batches_subbatches_and_chain():
    # more fields than the workspace (internal batches), sub-batch streams bit-identical, and a
    # cumulative update in this mode
    x = inputs.gaussian_fields(70, 4, 4, 20, seed=9)
    ctx = make_ctx(4, 20, 5, precision="bf16x9", max_fields=66)
    lndet, sign = ctx.logdet(cuda(x))
    p = HolsteinParams(4, 4, 20, n_s=5)
    ref, s_ref, _ = _oracle(p, x, want_G=False)
    assert np.abs(lndet.cpu().numpy() - ref).max() <= TOL_LNDET_MIXED
    assert np.array_equal(sign.cpu().numpy(), s_ref)
    ctx.set_sub_batches(1)
    ld1, _ = ctx.logdet(cuda(x))
    assert torch.equal(ld1, lndet)
    J = torch.tensor([0.0, 50.25, 0.05, 0.0, 0.02, 0.45], dtype=torch.float64, device="cuda")
    xc = cuda(x[:2].copy())
    lnw, s = ctx.chain_init(xc)
    ctx.cumulative_update(xc, J, 3, 4, 0, lnw, s)
    torch.cuda.synchronize()
    ctx.get_error()
    assert torch.isfinite(lnw).all()


TF32_CASES = [(4, 4, 40, 10, 6), (12, 12, 120, 10, 3), (16, 16, 160, 8, 3)]


@pytest.mark.xfail(strict=True, reason="split TF32 on truncating FP32 accumulation misses |d ln w| <= 1e-4")
@pytest.mark.parametrize("Lx,Ly,L,n_s,nf", TF32_CASES[2:])
def test_tf32x3_against_mixed_bar(Lx, Ly, L, n_s, nf):
    x = inputs.mixed_fields(max(nf, 2), Lx, Ly, L, seed=300 + L)[:nf]
    ctx = make_ctx(Lx, L, n_s, Ly=Ly, precision="tf32x3", max_fields=nf)
    lndet, sign = ctx.logdet(cuda(x))
    l_ref, _, _ = _oracle(HolsteinParams(Lx, Ly, L, n_s=n_s), x, want_G=False)
    assert np.abs(lndet.cpu().numpy() - l_ref).max() <= TOL_LNDET_MIXED


@pytest.mark.parametrize("Lx,Ly,L,n_s,nf", TF32_CASES)
def test_tf32x3_sign_greens_and_bounded_error(Lx, Ly, L, n_s, nf):
    x = inputs.mixed_fields(max(nf, 2), Lx, Ly, L, seed=300 + L)[:nf]
    ctx = make_ctx(Lx, L, n_s, Ly=Ly, precision="tf32x3", max_fields=nf)
    G, lndet, sign = ctx.greens(cuda(x))
    torch.cuda.synchronize()
    ctx.get_error()
    l_ref, s_ref, G_ref = _oracle(HolsteinParams(Lx, Ly, L, n_s=n_s), x)
    assert np.array_equal(sign.cpu().numpy(), s_ref)
    assert np.abs(G.cpu().numpy() - G_ref).max() <= 1e-4
    assert np.abs(lndet.cpu().numpy() - l_ref).max() <= 1e-2
