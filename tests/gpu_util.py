"""Shared helpers of the GPU tests (not collected: no test_ prefix)."""
import pytest
import torch


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def cuda(a):
    return torch.from_numpy(a).to("cuda")


def make_ctx(Lx, L, n_s, Ly=None, precision="fp64", max_fields=64, **kw):
    from paper_1802_06177_gb300.slmc import Context
    require_gpu()
    return Context(Lx, Ly or Lx, L, n_s=n_s, precision=precision, max_fields=max_fields, **kw)
