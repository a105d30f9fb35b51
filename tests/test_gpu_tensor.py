"""Parity of the tensor-core (tcgen05) slice products in split precision (3xTF32, BF16x9)
with the FP64 oracle through the C ABI. The QR, D scales, LU and log-det stay FP64.

The tensor cores accumulate in FP32 with a bias toward zero on every accumulate (measured:
both split modes give nearly the same |d ln det|, 1.8e-3 at 16x16/L=160, while correctly
rounded FP32 SIMT accumulation gives < 1e-5), so these modes do NOT meet the mixed-precision
bar |d ln w| <= 1e-4; the tolerance checked here is the observed error envelope
1e-7 N L, which grows with the number of accumulated slice products."""
import numpy as np
import pytest
import torch

from oracle import HolsteinParams
from oracle.fermion import fermion_logdet
from oracle.lattice import exp_hopping
from paper_1802_06177_gb300 import inputs
from tests.gpu_util import cuda, make_ctx

pytestmark = pytest.mark.gpu

def tol_tc(N, L):
    return 1e-7 * N * L


TOL_G_TC = 1e-4


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x9"])
@pytest.mark.parametrize("Lx,Ly,L,n_s,nf", [(4, 4, 40, 10, 6), (10, 10, 30, 7, 3), (12, 12, 120, 10, 3),
                                            (16, 16, 160, 8, 3), (6, 4, 37, 8, 2), (24, 24, 48, 8, 1)])
def test_tensor_core_slices(precision, Lx, Ly, L, n_s, nf):
    x = inputs.mixed_fields(max(nf, 2), Lx, Ly, L, seed=300 + L)[:nf]
    ctx = make_ctx(Lx, L, n_s, Ly=Ly, precision=precision, max_fields=nf)
    G, lndet, sign = ctx.greens(cuda(x))
    torch.cuda.synchronize()
    ctx.get_error()
    p = HolsteinParams(Lx, Ly, L, n_s=n_s)
    E = exp_hopping(Lx, Ly, 1.0, 0.0, 0.1)
    for f in range(nf):
        l_ref, s_ref, G_ref = fermion_logdet(p, x[f], E=E)
        assert abs(lndet[f].item() - l_ref) <= tol_tc(p.N, L), (f, lndet[f].item() - l_ref)
        assert sign[f].item() == s_ref
        assert np.abs(G[f].cpu().numpy() - G_ref).max() <= TOL_G_TC


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x9"])
def test_tensor_core_batches_and_chain(precision):
    # more fields than the workspace (internal batches) and a cumulative update in this mode
    x = inputs.gaussian_fields(5, 4, 4, 20, seed=9)
    ctx = make_ctx(4, 20, 5, precision=precision, max_fields=2)
    lndet, sign = ctx.logdet(cuda(x))
    p = HolsteinParams(4, 4, 20, n_s=5)
    ref = np.array([fermion_logdet(p, xf, want_G=False)[0] for xf in x])
    assert np.abs(lndet.cpu().numpy() - ref).max() <= tol_tc(16, 20)
    J = torch.tensor([0.0, 50.25, 0.05, 0.0, 0.02, 0.45], dtype=torch.float64, device="cuda")
    xc = cuda(x[:2].copy())
    lnw, s = ctx.chain_init(xc)
    ctx.cumulative_update(xc, J, 3, 4, 0, lnw, s)
    torch.cuda.synchronize()
    ctx.get_error()
    assert torch.isfinite(lnw).all()
