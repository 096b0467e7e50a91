"""The plain definition (Section 2) evaluated in mpmath at 250 significant digits.

At beta = 64 the singular values of B_Nt...B_1 span e^{+-192} ~ 10^{+-83}; with 250 digits the
plain product keeps every direction, so log det(1 + P) and (1 + P)^{-1} come out exact to far
beyond FP64 for the FP64 inputs (E and phi are converted exactly from their float64 values).
Nx = 8 only: pure-Python matrix products.  Not imported by ``oracle/__init__`` (mpmath is an
optional dependency).
"""
from __future__ import annotations

import numpy as np


def logdet_green(E: np.ndarray, phi: np.ndarray, dps: int = 250):
    import mpmath as mp

    mp.mp.dps = dps
    nt, nx = phi.shape
    Em = [[mp.mpf(float(E[i, j])) for j in range(nx)] for i in range(nx)]
    P = [[mp.mpc(1 if i == j else 0) for j in range(nx)] for i in range(nx)]
    for t in range(nt):
        ph = [mp.expj(mp.mpf(float(phi[t, k]))) for k in range(nx)]
        Y = [[ph[k] * P[k][j] for j in range(nx)] for k in range(nx)]
        P = [[mp.fsum(Em[i][k] * Y[k][j] for k in range(nx)) for j in range(nx)]
             for i in range(nx)]
    Mh = mp.matrix(nx, nx)
    for i in range(nx):
        for j in range(nx):
            Mh[i, j] = P[i][j] + (1 if i == j else 0)
    det = mp.det(Mh)
    logdet = mp.log(det)
    Ginv = mp.inverse(Mh)
    G = np.array([[complex(Ginv[i, j]) for j in range(nx)] for i in range(nx)])
    im = float(mp.im(logdet))
    im = float(np.angle(np.exp(1j * im)))
    return complex(float(mp.re(logdet)), im), G


def green_tau(E: np.ndarray, phi: np.ndarray, taus, dps: int = 250) -> dict:
    """{tau: (L_tau^{-1} + R_tau)^{-1}} from the plain products in mpmath (Section 4.2)."""
    import mpmath as mp

    mp.mp.dps = dps
    nt, nx = phi.shape
    Em = mp.matrix([[mp.mpf(float(E[i, j])) for j in range(nx)] for i in range(nx)])

    def slice_m(t):
        ph = [mp.expj(mp.mpf(float(phi[t, k]))) for k in range(nx)]
        B = mp.matrix(nx, nx)
        for i in range(nx):
            for k in range(nx):
                B[i, k] = Em[i, k] * ph[k]
        return B

    slices = [slice_m(t) for t in range(nt)]
    out = {}
    for tau in taus:
        L = mp.eye(nx)
        for t in range(tau):
            L = slices[t] * L
        R = mp.eye(nx)
        for t in range(tau, nt):
            R = slices[t] * R
        Gt = mp.inverse(mp.inverse(L) + R)
        out[int(tau)] = np.array([[complex(Gt[i, j]) for j in range(nx)] for i in range(nx)])
    return out
