"""Single-time observables from the Green's functions (Section 4.1).

* Fermion number (Eq. fermion_number): the response to the chemical potential,
      n = 1 - tr G / V,   G = (1 + B_Nt...B_1)^{-1},   V = Nx.
* Single-time response traces: the thermal trace of an operator O with the equal-time Green's
  function at every time slice (the reading of Eq. response_simple without its O(delta)
  shortcut),
      R[r] = tr(O G_r),   G_r = (1 + B_r...B_1 B_Nt...B_{r+1})^{-1},   r = 0..Nt-1  (G_0 = G).
  With O = e_x e_x^T this is [G_r]_xx (the force row F[r] = i (1 - diag G_r)).
* Hopping response: for B_t = E D_t with E = exp(delta kappa A), dB_t/dkappa = delta A B_t
  exactly (A commutes with E), and Jacobi's formula with the cyclic rewriting of
  Eq. response_result gives
      d log det / d kappa = delta sum_{t=1..Nt} tr(A (1 - G_t)) = -delta sum_r tr(A G_r)
  (tr A = 0 on the honeycomb lattice; G_Nt = G_0).

Each G_r is an independent stabilised evaluation on the rotated field (oracle.force.green_at):
slow and simple, on purpose.
"""
from __future__ import annotations

import numpy as np

from . import force as _force
from . import stable as _stable


def fermion_number(E: np.ndarray, phi: np.ndarray, n_stab: int) -> complex:
    _, G = _stable.logdet_green(E, phi, n_stab)
    return complex(1.0 - np.trace(G) / G.shape[0])


def response_traces(E: np.ndarray, phi: np.ndarray, n_stab: int, O: np.ndarray) -> np.ndarray:
    """R[r] = tr(O G_r), r = 0..Nt-1 (complex)."""
    nt = phi.shape[0]
    out = np.empty(nt, dtype=complex)
    for r in range(nt):
        out[r] = np.trace(O @ _force.green_at(E, phi, n_stab, r))
    return out


def hopping_response(E: np.ndarray, phi: np.ndarray, n_stab: int, A: np.ndarray,
                     delta: float) -> complex:
    """d log det / d kappa = delta sum_r tr(A (1 - G_r))."""
    R = response_traces(E, phi, n_stab, A)
    nt = phi.shape[0]
    return complex(delta * (nt * np.trace(A) - R.sum()))
