"""Closed form at zero field.

With phi = 0 every slice is E = exp(delta*kappa*A), so B_Nt...B_1 = exp(beta*kappa*A) and, with
A = U diag(lambda) U^T,
    log det(1 + P) = sum_k log(1 + exp(beta*kappa*lambda_k)),
    G = U diag(1 / (1 + exp(beta*kappa*lambda_k))) U^T.
This is the free-fermion partition function det(1 + e^{-beta K}) with K = -kappa A.
"""
from __future__ import annotations

import numpy as np


def logdet_green(A: np.ndarray, beta: float, kappa: float = 1.0):
    lam, U = np.linalg.eigh(A)
    x = beta * kappa * lam
    logdet = np.sum(np.logaddexp(0.0, x))
    fermi = 0.5 * (1.0 - np.tanh(0.5 * x))  # 1/(1+e^x), overflow-free
    G = (U * fermi[None, :]) @ U.T
    return complex(logdet, 0.0), G.astype(complex)


def logdet_from_spectrum(lam: np.ndarray, beta: float, kappa: float = 1.0) -> float:
    """Same log det from a given single-particle spectrum (e.g. the momentum-space bands)."""
    return float(np.sum(np.logaddexp(0.0, beta * kappa * np.asarray(lam))))
