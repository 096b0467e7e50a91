"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports exactly the
functions include/fd.h declares, with the ctypes signatures the binding uses.  No compute calls
(there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fd_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_02130_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_api():
    names = _declared()
    for n in ("fd_ctx_create", "fd_ctx_destroy", "fd_logdet", "fd_green", "fd_force",
              "fd_status", "fd_last_error", "fd_reserve"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_header():
    from paper_2604_02130_gb300 import _lib

    bound = {name for name, _, _ in _lib.SIGNATURES}
    assert bound == set(_declared())


def test_problem_struct_layout():
    from paper_2604_02130_gb300 import _lib

    assert ctypes.sizeof(_lib.fd_problem) == 40
    assert _lib.fd_problem.expA.offset == 16


def test_bss_struct_layout():
    from paper_2604_02130_gb300 import _lib

    assert ctypes.sizeof(_lib.fd_bss_slice) == 56
    assert _lib.fd_bss_slice.G.offset == 8
    assert _lib.fd_bss_slice.accepted.offset == 48


def test_sparse_hop_struct_layout():
    from paper_2604_02130_gb300 import _lib

    assert ctypes.sizeof(_lib.fd_sparse_hop) == 24
    assert _lib.fd_sparse_hop.col.offset == 8
    assert _lib.fd_sparse_hop.val.offset == 16


def test_taylor_factors_match_the_oracle(lib):
    """The library's product-form factors (host code, no GPU: a Weierstrass iteration) against
    the oracle's, which come from numpy's companion-matrix roots."""
    import numpy as np

    from oracle import product_form

    from paper_2604_02130_gb300 import _lib

    f = lib.fd_taylor_factors
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    for n in range(1, 9):
        arr = (ctypes.c_double * 16)()
        assert f(n, arr) == 0
        got = [complex(arr[2 * k], arr[2 * k + 1]) for k in range(n)]
        # the same multiset (conjugate partners may swap places: their real parts tie)
        for w in product_form.taylor_factors(n):
            k = int(np.argmin([abs(g - w) for g in got]))
            assert abs(got.pop(k) - w) < 1e-12, n
    arr = (ctypes.c_double * 16)()
    assert f(0, arr) == -1 and f(9, arr) == -1
    assert _lib.SIGNATURES  # bound like every other export


def test_ctx_create_without_gpu_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    lib.fd_ctx_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
    rc = lib.fd_ctx_create(ctypes.byref(h), 0)
    assert rc == -3 and not h.value  # FD_ERR_CUDA, no context


def test_null_context_is_rejected(lib):
    lib.fd_logdet.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_int, ctypes.c_void_p]
    assert lib.fd_logdet(None, 1, None, None, 0, None) == -1


def test_flop_counts():
    from paper_2604_02130_gb300 import force_flops, fwd_flops

    f = fwd_flops(72, 512, 16)
    assert abs(f["slices"] - 4 * 72 ** 3 * 512) < 1
    g = force_flops(72, 256, 8)
    assert g["total"] > fwd_flops(72, 256, 8)["total"]
