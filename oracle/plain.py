"""The plain definitions (Section 2), no stabilisation.  Valid only while B_Nt...B_1 fits FP64
without swamping its small singular values (beta*kappa*3 up to ~8 for honeycomb fields).

Product order: the block fermion matrix of Section 2 has +M_{Nt-1} in its top-right block and
-M_t below the diagonal, so det M = det(1 + M_{Nt-1} ... M_0).  With M_{t-1} = B_t this is
det(1 + B_Nt ... B_1), and the Green's function is G = (1 + B_Nt ... B_1)^{-1}.
"""
from __future__ import annotations

import numpy as np


def slice_matrix(E: np.ndarray, phi_t: np.ndarray) -> np.ndarray:
    """B_t = E diag(exp(i phi_t))."""
    return E * np.exp(1j * phi_t)[None, :]


def product(E: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """P = B_Nt ... B_1; row t-1 of phi belongs to slice t (slice 1 acts first)."""
    nt, nx = phi.shape
    P = np.eye(nx, dtype=complex)
    for t in range(nt):
        P = slice_matrix(E, phi[t]) @ P
    return P


def logdet_green(E: np.ndarray, phi: np.ndarray):
    """(log det(1+P), (1+P)^{-1}) straight from the definition."""
    P = product(E, phi)
    Mhat = np.eye(P.shape[0]) + P
    sign, logabs = np.linalg.slogdet(Mhat)
    return logabs + 1j * np.angle(sign), np.linalg.inv(Mhat)
