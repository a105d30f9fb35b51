"""The allocation-free determinant entry point, slmc_logdet_noalloc, called through the C
ABI: it serves callers that cannot allocate device memory (graph capture, allocator-free
hot loops, hosts owning the memory budget), keeping its workspace in a fixed device array.
Its results must equal those of the regular slmc_logdet on the same fields, on two calls
in a row (the array is reused and keeps the previous call's contents). The entry point runs
the T update and the QR trailing updates of the stabilisation with FP64 FMAs (it has no room
for the tensor-core slices), so the regular context it is compared with is set to the same
paths. This file is collected
last so that a failure here cannot hide the other tests' results."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1802_06177_gb300 import inputs
from tests.gpu_util import cuda, make_ctx

pytestmark = pytest.mark.gpu

TOL_LNDET_FP64 = 1e-8


@pytest.mark.parametrize("Lx,L,n_s,nf", [(4, 40, 10, 16), (16, 160, 8, 7)])
def test_noalloc_matches_logdet_twice(Lx, L, n_s, nf):
    from paper_1802_06177_gb300.slmc import Params, load_library
    lib = load_library()
    assert lib.slmc_logdet_noalloc_scratch_bytes() == 16 << 20
    ctx = make_ctx(Lx, L, n_s, max_fields=nf)
    ctx.set_tupdate_path(1)
    ctx.set_qr_path(1)
    p = Params(Lx, Lx, L, 0.1, 1.0, 0.0, 1.0, 1.0, n_s, 0, 0.0, 0)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        x = cuda(inputs.mixed_fields(nf, Lx, Lx, L, seed=100 + call))
        ref_l, ref_s = ctx.logdet(x)
        lndet = torch.full((nf,), float("nan"), dtype=torch.float64, device="cuda")
        sign = torch.zeros(nf, dtype=torch.int32, device="cuda")
        st = lib.slmc_logdet_noalloc(ctypes.byref(p), x.data_ptr(), nf, lndet.data_ptr(), sign.data_ptr(), stream)
        assert st == 0
        torch.cuda.synchronize()
        assert np.abs(lndet.cpu().numpy() - ref_l.cpu().numpy()).max() <= TOL_LNDET_FP64
        assert np.array_equal(sign.cpu().numpy(), ref_s.cpu().numpy())


def test_noalloc_rejects_too_large_lattice():
    from paper_1802_06177_gb300.slmc import Params, load_library
    lib = load_library()
    p = Params(24, 24, 20, 0.1, 1.0, 0.0, 1.0, 1.0, 8, 0, 0.0, 0)  # N = 576 does not fit in 16 MiB
    x = torch.zeros((1, 576, 20), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    sg = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.slmc_logdet_noalloc(ctypes.byref(p), x.data_ptr(), 1, out.data_ptr(), sg.data_ptr(), None) == 5


@pytest.mark.parametrize("Lx,L,n_s,nf", [(4, 40, 10, 5), (16, 160, 8, 3)])
def test_noalloc_fp32_matches_logdet(Lx, L, n_s, nf):
    """FP32 slice products (F = E - I, F_lo stencil, FP32 Q buffer carved from the array): the
    same arithmetic per field as the regular entry point."""
    from paper_1802_06177_gb300.slmc import Params, load_library
    lib = load_library()
    ctx = make_ctx(Lx, L, n_s, precision="fp32", max_fields=nf)
    ctx.set_tupdate_path(1)
    ctx.set_qr_path(1)
    p = Params(Lx, Lx, L, 0.1, 1.0, 0.0, 1.0, 1.0, n_s, 1, 0.0, 0)
    x = cuda(inputs.mixed_fields(nf, Lx, Lx, L, seed=7))
    ref_l, ref_s = ctx.logdet(x)
    lndet = torch.full((nf,), float("nan"), dtype=torch.float64, device="cuda")
    sign = torch.zeros(nf, dtype=torch.int32, device="cuda")
    st = lib.slmc_logdet_noalloc(ctypes.byref(p), x.data_ptr(), nf, lndet.data_ptr(), sign.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    assert np.abs(lndet.cpu().numpy() - ref_l.cpu().numpy()).max() <= 1e-10
    assert np.array_equal(sign.cpu().numpy(), ref_s.cpu().numpy())


def test_noalloc_reuse_across_lattices_and_chunks():
    """A 16x16 FP32 call with more fields than the array holds (processed in chunks), then a 4x4
    FP64 call that reuses the same regions of the array for a smaller lattice: each equals the
    regular entry point on the same fields."""
    from paper_1802_06177_gb300.slmc import logdet_noalloc
    for Lx, L, n_s, nf, prec, tol in ((16, 160, 8, 7, "fp32", 1e-10), (4, 40, 10, 9, "fp64", 1e-12)):
        ctx = make_ctx(Lx, L, n_s, precision=prec, max_fields=nf)
        ctx.set_tupdate_path(1)
        ctx.set_qr_path(1)
        x = cuda(inputs.mixed_fields(nf, Lx, Lx, L, seed=31 + Lx))
        ref_l, ref_s = ctx.logdet(x)
        lndet, sign = logdet_noalloc(x, Lx, Lx, L, n_s=n_s, precision=prec)
        torch.cuda.synchronize()
        assert np.abs(lndet.cpu().numpy() - ref_l.cpu().numpy()).max() <= tol, (Lx, prec)
        assert np.array_equal(sign.cpu().numpy(), ref_s.cpu().numpy())
