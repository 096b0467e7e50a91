"""fd_logdet_noalloc: the entry point for callers that cannot allocate device memory.

It runs the FP64 log det / G computation with its working memory in a fixed array inside the
library instead of context-owned allocations.  This test calls it through the C ABI (ctypes) on
two batches in a row -- the second call reuses the array with the first call's contents still
in it -- and compares each result with the context-based entry point fd_green and with the CPU
oracle, within the FP64 tolerances used by the other parity tests; a third call fills the array
to its largest allowed batch.  It also checks the capacity limits.  The file name makes pytest
collect it last.
"""
import ctypes

import numpy as np
import pytest

import fd_inputs as fi
from oracle import stable

from gpu_helpers import G_ATOL_FP64, LOGDET_RTOL_FP64, logdet_err, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problems(tens):
    from paper_2604_02130_gb300 import _lib as L

    arr = (L.fd_problem * len(tens))()
    for c, (E, Einv, phi, ns) in enumerate(tens):
        nt, nx = phi.shape
        arr[c].nx, arr[c].nt, arr[c].n_stab, arr[c].reserved = nx, nt, ns, 0
        arr[c].expA, arr[c].expA_inv, arr[c].phi = E.data_ptr(), Einv.data_ptr(), phi.data_ptr()
    return arr


def _noalloc(lib, tens):
    n = len(tens)
    dev = torch.device("cuda", 0)
    ld = torch.full((n, 2), float("nan"), dtype=torch.float64, device=dev)
    G = [torch.full((t[2].shape[1],) * 2, float("nan"), dtype=torch.complex128, device=dev)
         for t in tens]
    st = torch.full((n,), -7, dtype=torch.int32, device=dev)
    Gp = (ctypes.c_void_p * n)(*[g.data_ptr() for g in G])
    rc = lib.fd_logdet_noalloc(n, _problems(tens), ctypes.c_void_p(ld.data_ptr()), Gp,
                               ctypes.c_void_p(st.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    return ld.cpu().numpy(), [g.cpu().numpy() for g in G]


def _reference(tens):
    from paper_2604_02130_gb300 import api

    ctx = api.Context(0)
    r = api.Batch(ctx, tens, "green").run()
    torch.cuda.synchronize()
    out = r.logdet.cpu().numpy(), [g.cpu().numpy() for g in r.G]
    ctx.close()
    return out


def test_noalloc_matches_fd_green_two_calls():
    from paper_2604_02130_gb300 import _lib as L

    lib = L.load()
    torch.cuda.set_device(0)
    # call 1: the largest matrix size (Nx = 72); call 2: a different, smaller mix that reuses the
    # array; call 3: the largest batch at the largest size, whose last slot ends nearest the end
    # of the array
    first = [fi.make_problem(6, 32, 4.0, 3.0, 8, 91, c) for c in range(6)]
    second = [fi.make_problem(L_, 32, 2.0, 3.0, 8, 92, c)
              for c, L_ in enumerate([3, 2, 4, 3, 5, 2, 3, 6])]
    third = [fi.make_problem(6, 4, 0.5, 3.0, 4, 94, c) for c in range(L.FD_NOALLOC_MAX_BATCH)]
    for probs in (first, second, third):
        tens = to_dev(probs)
        ld, G = _noalloc(lib, tens)
        ref_ld, ref_G = _reference(tens)
        for c in range(len(tens)):
            assert logdet_err(complex(*ld[c]), complex(ref_ld[c])) <= LOGDET_RTOL_FP64
            assert np.abs(G[c] - ref_G[c]).max() <= G_ATOL_FP64
        for c in range(0, len(probs), 7):  # against the oracle as well
            p = probs[c]
            o_ld, o_G = stable.logdet_green(p.E, p.phi, p.n_stab)
            assert logdet_err(complex(*ld[c]), o_ld) <= LOGDET_RTOL_FP64
            assert np.abs(G[c] - o_G).max() <= G_ATOL_FP64


def test_noalloc_rejects_beyond_capacity():
    from paper_2604_02130_gb300 import _lib as L

    lib = L.load()
    big = to_dev([fi.make_problem(7, 8, 1.0, 3.0, 8, 93, 0)])      # Nx = 98 > 72
    ld = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    rc = lib.fd_logdet_noalloc(1, _problems(big), ctypes.c_void_p(ld.data_ptr()), None, None,
                               None)
    assert rc == L.FD_ERR_TOO_LARGE
    small = to_dev([fi.make_problem(2, 8, 1.0, 3.0, 8, 93, 0)])
    many = small * (L.FD_NOALLOC_MAX_BATCH + 1)
    ld = torch.zeros((len(many), 2), dtype=torch.float64, device="cuda")
    rc = lib.fd_logdet_noalloc(len(many), _problems(many), ctypes.c_void_p(ld.data_ptr()), None,
                               None, None)
    assert rc == L.FD_ERR_TOO_LARGE
