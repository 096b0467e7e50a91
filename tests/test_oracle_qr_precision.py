"""How much precision the QR re-orthogonalisation of the stabilised method needs (Section 7).

The oracle's chain is run with every QR result (Q, R and the updated T) perturbed by relative
noise of size u, emulating a QR carried out with unit roundoff u, and compared with the FP64
chain at beta = 64 and at the batch18 shape.  With u = 2^-46 (double-float pairs on FP32 units)
log det and G stay within 1e-12 of the FP64 result, far inside the FP64 path's 1e-8 target;
with u = 2^-24 (plain FP32) the errors are of the order of the mixed 3xTF32 path's bounds.
A property of the method, not of an implementation: it bounds the arithmetic a faster QR may use.
"""
import numpy as np
import pytest
import scipy.linalg

import fd_inputs as fi
from oracle import stable
from oracle.plain import slice_matrix


def _chain(E, phi, n_stab, u, rng):
    def noisy(a):
        z = rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape)
        return a * (1 + u * z / np.sqrt(2))

    nt, nx = phi.shape
    X = np.eye(nx, dtype=complex)
    D = np.ones(nx)
    T = np.eye(nx, dtype=complex)
    for t in range(0, nt, n_stab):
        for s in range(t, t + n_stab):
            X = slice_matrix(E, phi[s]) @ X
        Q, R, perm = scipy.linalg.qr(X * D[None, :], pivoting=True)
        Q, R = noisy(Q), noisy(R)
        d = np.abs(np.diag(R))
        T = noisy((R / d[:, None]) @ T[perm, :])
        X, D = Q, d
    return stable.assemble(X, D, T)


@pytest.mark.parametrize("L,nt,beta,U,n_stab", [(3, 512, 64.0, 3.5, 16), (3, 64, 8.0, 3.0, 8)])
def test_qr_precision_needed(L, nt, beta, U, n_stab):
    p = fi.make_problem(L, nt, beta, U, n_stab, 1002, 0)
    ld0, G0 = stable.logdet_green(p.E, p.phi, n_stab)
    scale = max(1.0, float(np.abs(G0).max())) ** 2
    errs = {}
    for u in (2.0 ** -46, 2.0 ** -24):
        ld, G = _chain(p.E, p.phi, n_stab, u, np.random.default_rng(0))
        errs[u] = (abs(ld.real - ld0.real) / abs(ld0), float(np.abs(G - G0).max()) / scale)
    assert errs[2.0 ** -46][0] < 1e-12 and errs[2.0 ** -46][1] < 1e-10
    assert errs[2.0 ** -24][0] < 1e-6 and errs[2.0 ** -24][1] < 1e-4
    # the errors follow the precision (a test that perturbed nothing would pass the bounds too)
    assert errs[2.0 ** -24][1] > 1e3 * errs[2.0 ** -46][1]
