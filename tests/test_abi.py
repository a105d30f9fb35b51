"""The C-ABI library builds, loads without a GPU and exports every entry point that
include/slmc.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "slmc.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SLMC_API\s+(?:const\s+char\s*\*|long\s+long|size_t|slmc_ctx\s*\*|int)\s+(slmc_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1802_06177_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return build.LIB


def test_header_declares_entry_points():
    syms = declared_symbols()
    for name in ("slmc_init", "slmc_logdet", "slmc_greens", "slmc_eff_sweep", "slmc_cumulative_update",
                 "slmc_fit_eff"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_declares_every_export():
    from paper_1802_06177_gb300 import slmc
    assert sorted(slmc.EXPORTS) == declared_symbols()


def test_status_strings_without_gpu(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.slmc_status_string.restype = ctypes.c_char_p
    assert lib.slmc_status_string(0) == b"ok"
    assert lib.slmc_status_string(5) == b"unsupported shape or mode"


def test_init_rejects_bad_params_on_host(lib_path):
    # argument validation happens before any CUDA call, so it runs without a GPU
    from paper_1802_06177_gb300.slmc import Params
    lib = ctypes.CDLL(lib_path)
    out = ctypes.c_void_p()
    bad = Params(1, 4, 10, 0.1, 1.0, 0.0, 1.0, 1.0, 10, 0, 0.5, 0)
    assert lib.slmc_init(ctypes.byref(bad), 4, ctypes.byref(out)) == 1
    big = Params(40, 40, 10, 0.1, 1.0, 0.0, 1.0, 1.0, 10, 0, 0.5, 0)
    assert lib.slmc_init(ctypes.byref(big), 4, ctypes.byref(out)) == 5
    neg = Params(4, 4, 10, -0.1, 1.0, 0.0, 1.0, 1.0, 10, 0, 0.5, 0)
    assert lib.slmc_init(ctypes.byref(neg), 4, ctypes.byref(out)) == 1
    assert lib.slmc_init(None, 4, ctypes.byref(out)) == 1
    assert not out.value


def test_params_struct_layout_matches_header():
    from paper_1802_06177_gb300.slmc import Params
    # int Lx, Ly, L; pad; 5 doubles; int n_s, precision; double sweep_delta; uint64 seed; int qr_mode; pad
    assert ctypes.sizeof(Params) == 12 + 4 + 5 * 8 + 8 + 8 + 8 + 8
    assert Params.dtau.offset == 16 and Params.n_s.offset == 56 and Params.seed.offset == 72
    assert Params.qr_mode.offset == 80
