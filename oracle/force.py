"""HMC force F[t, x] = d log det(1 + B_Nt...B_1) / d phi[t, x] (Section 4, Eq. response_result).

Jacobi's formula with dB_t/dphi_{t,x} = B_t (i e_x e_x^T) and the cyclic rewriting of
Eq. response_result give, for slice t (1-based),
    F[t, x] = i [R (1 + L B_t R)^{-1} L B_t]_{xx} = i (1 - [G_{t-1}]_{xx}),
    L = B_Nt ... B_{t+1},  R = B_{t-1} ... B_1,
    G_{t-1} = (1 + B_{t-1} ... B_1 B_Nt ... B_t)^{-1}.
G_{t-1} is the Green's function of the same field with its slices rotated so that slice t acts
first, so each row of F costs one independent stabilised evaluation (O(Nt^2) in total: slow and
simple, on purpose).  Row t-1 of the returned array is slice t, matching phi.
"""
from __future__ import annotations

from typing import Iterable, Sequence, Tuple

import numpy as np

from . import stable


def green_at(E: np.ndarray, phi: np.ndarray, n_stab: int, tau: int) -> np.ndarray:
    """Equal-time G_tau = (1 + B_tau...B_1 B_Nt...B_{tau+1})^{-1}, tau = 0..Nt-1."""
    rolled = np.roll(phi, -tau, axis=0)  # row 0 is slice tau+1
    return stable.logdet_green(E, rolled, n_stab)[1]


def force(E: np.ndarray, phi: np.ndarray, n_stab: int) -> np.ndarray:
    nt, nx = phi.shape
    F = np.empty((nt, nx), dtype=complex)
    for t in range(1, nt + 1):
        F[t - 1] = 1j * (1.0 - np.diag(green_at(E, phi, n_stab, t - 1)))
    return F


def force_rows(E: np.ndarray, phi: np.ndarray, n_stab: int, rows: Iterable[int]) -> dict:
    """{row: F[row, :]} for selected rows (row = t-1) -- for sampled checks at full size."""
    return {int(r): 1j * (1.0 - np.diag(green_at(E, phi, n_stab, int(r)))) for r in rows}


def finite_difference(E: np.ndarray, phi: np.ndarray, n_stab: int,
                      entries: Sequence[Tuple[int, int]], h: float = 1e-6) -> np.ndarray:
    """Central differences (logdet(phi + h e) - logdet(phi - h e)) / 2h at (row, x) entries.

    The imaginary part of log det is only defined mod 2 pi, so the difference of imaginary parts
    is taken on the principal branch."""
    out = []
    for (r, x) in entries:
        p = phi.copy()
        p[r, x] += h
        lp, _ = stable.logdet_green(E, p, n_stab)
        p[r, x] -= 2 * h
        lm, _ = stable.logdet_green(E, p, n_stab)
        dre = (lp.real - lm.real) / (2 * h)
        dim = np.angle(np.exp(1j * (lp.imag - lm.imag))) / (2 * h)
        out.append(dre + 1j * dim)
    return np.asarray(out)
