"""The naive small-volume, high-temperature algorithm of Section 6.

Steps (Section 6): form every slice matrix, multiply the product and diagonalise it,
P = S D' S^{-1} (not Hermitian in general); then det(1+P) = prod(1 + D') and
(1+P)^{-1} = S (1 + D')^{-1} S^{-1}.  With the factored slices B_t = E diag(e^{i phi_t}) the
slice matrices are formed directly instead of via an eigen-decomposition of K_t.  Unstable at
large beta (the paper says so); used only as a cross-check at beta <= 4.
"""
from __future__ import annotations

import numpy as np

from .plain import slice_matrix


def logdet_green(E: np.ndarray, phi: np.ndarray):
    nt, nx = phi.shape
    P = np.eye(nx, dtype=complex)
    for t in range(nt):
        P = slice_matrix(E, phi[t]) @ P
    dprime, S = np.linalg.eig(P)
    dhat = 1.0 + dprime
    logdet = np.sum(np.log(dhat))
    G = (S / dhat[None, :]) @ np.linalg.inv(S)
    im = float(np.angle(np.exp(1j * logdet.imag)))
    return complex(logdet.real, im), G
