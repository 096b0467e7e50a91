"""Brute force on the full fermion matrix of Section 2 (tiny sizes only: (Nt*Nx)^2 dense).

Block layout (0-based block rows/columns tau = 0..Nt-1, each Nx x Nx):
    M[tau, tau]    = 1
    M[tau, tau-1]  = -B_tau          (tau = 1..Nt-1)
    M[0, Nt-1]     = +B_Nt           (anti-periodic boundary)
This is the paper's block matrix with M_{t-1} = B_t.  Then det M = det(1 + B_Nt ... B_1) and the
diagonal blocks of M^{-1} are the equal-time Green's functions
    (M^{-1})[tau, tau] = (1 + B_tau ... B_1 B_Nt ... B_{tau+1})^{-1} = G_tau,
so (M^{-1})[0, 0] = G.  (Solve M psi = e_0: psi_tau = B_tau ... B_1 psi_0, and block row 0 gives
psi_0 + B_Nt psi_{Nt-1} = 1.)
"""
from __future__ import annotations

import numpy as np

from .plain import slice_matrix


def full_matrix(E: np.ndarray, phi: np.ndarray) -> np.ndarray:
    nt, nx = phi.shape
    M = np.eye(nt * nx, dtype=complex)
    for tau in range(1, nt):
        M[tau * nx:(tau + 1) * nx, (tau - 1) * nx:tau * nx] = -slice_matrix(E, phi[tau - 1])
    M[0:nx, (nt - 1) * nx:nt * nx] += slice_matrix(E, phi[nt - 1])
    return M


def logdet(E: np.ndarray, phi: np.ndarray) -> complex:
    sign, logabs = np.linalg.slogdet(full_matrix(E, phi))
    return logabs + 1j * np.angle(sign)


def green_blocks(E: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """All diagonal blocks G_tau = (M^{-1})[tau, tau], shape (Nt, Nx, Nx)."""
    nt, nx = phi.shape
    Minv = np.linalg.inv(full_matrix(E, phi))
    return np.stack([Minv[t * nx:(t + 1) * nx, t * nx:(t + 1) * nx] for t in range(nt)])


def inverse_column(E: np.ndarray, phi: np.ndarray, t0: int = 0) -> np.ndarray:
    """Blocks (M^{-1})[tau, t0] for tau = 0..Nt-1, shape (Nt, Nx, Nx): the unequal-time Green's
    function G(tau, t0) (Section 4.2)."""
    nt, nx = phi.shape
    Minv = np.linalg.inv(full_matrix(E, phi))
    return np.stack([Minv[t * nx:(t + 1) * nx, t0 * nx:(t0 + 1) * nx] for t in range(nt)])
