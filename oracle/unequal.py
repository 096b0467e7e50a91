"""Unequal-time Green's function G(tau, 0) = (M^{-1})_{tau, 0}, tau = 0..Nt-1 (Section 4.2).

Eq. sausage_all_in_denominator with t0 = 0 <= t = tau (and M_{t-1} = B_t):
    G(tau, 0) = (L_tau^{-1} + R_tau)^{-1},  L_tau = B_tau...B_1,  R_tau = B_Nt...B_{tau+1},
which equals B_tau...B_1 (1 + B_Nt...B_1)^{-1} (push-through identity).  G(0, 0) = G.

Modules:
  plain  -- B_tau...B_1 G straight from the definition (small beta only);
  stable -- Section 7 steps 7-9: the sum A1 + A2^{-1} with A1 = R_tau = X' D' Y'^{-1} and
            A2 = L_tau = X'' D'' Y''^{-1} is written X' [D' Y'^{-1} X'' + X'^{-1} Y'' D''^{-1}]
            X''^{-1}; the bracket is QR-decomposed (= Q D R) and
            (A1 + A2^{-1})^{-1} = (X'' R^{-1}) D^{-1} (Q^H X'^{-1}).
            Both products come from oracle.stable.udt_product (QR every n_stab slices).
"""
from __future__ import annotations

from typing import Iterable

import numpy as np

from . import plain as _plain
from . import stable as _stable


def green_tau_plain(E: np.ndarray, phi: np.ndarray) -> np.ndarray:
    nt, nx = phi.shape
    _, G = _plain.logdet_green(E, phi)
    out = np.empty((nt, nx, nx), dtype=complex)
    L = np.eye(nx, dtype=complex)
    for tau in range(nt):
        out[tau] = L @ G
        L = _plain.slice_matrix(E, phi[tau]) @ L
    return out


def green_tau_stable(E: np.ndarray, phi: np.ndarray, n_stab: int,
                     taus: Iterable[int] | None = None) -> dict:
    """{tau: G(tau, 0)} by Section 7 steps 7-9."""
    nt, nx = phi.shape
    taus = range(nt) if taus is None else taus
    out = {}
    for tau in taus:
        tau = int(tau)
        if tau == 0:
            out[0] = _stable.logdet_green(E, phi, n_stab)[1]
            continue
        # A1 = R_tau = B_Nt...B_{tau+1}: the slices tau+1..Nt (rows tau..Nt-1) act first to last
        X1, D1, T1 = _stable.udt_product(E, phi[tau:], n_stab)
        # A2 = L_tau = B_tau...B_1
        X2, D2, T2 = _stable.udt_product(E, phi[:tau], n_stab)
        Y1inv = T1                      # A1 = X1 D1 Y1^{-1}
        Y2 = np.linalg.inv(T2)          # A2 = X2 D2 Y2^{-1}, Y2 = T2^{-1}
        bracket = D1[:, None] * (Y1inv @ X2) + (X1.conj().T @ Y2) / D2[None, :]
        Q, R = np.linalg.qr(bracket)
        d = np.diag(R).copy()
        Rn = R / d[:, None]             # unit diagonal, bracket = Q diag(d) Rn
        out[tau] = (X2 @ np.linalg.inv(Rn)) @ np.diag(1.0 / d) @ (Q.conj().T @ X1.conj().T)
    return out
