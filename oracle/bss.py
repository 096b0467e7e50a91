"""Local (BSS) updates of the auxiliary field at one time slice (Section 3, the BSS algorithm).

Sites x = 0..nx-1 of slice t (1-based; field row t-1) are visited in order.  At site x the
proposal phi[t-1, x] -> phi[t-1, x] + dphi[x] changes the determinant by the ratio
    r_x = det(1 + P') / det(1 + P),
and is accepted iff u[x] < |r_x| w[x]  (u: the caller's uniform random numbers, w > 0: the
caller's ratio of every other weight factor, e.g. the Gaussian weight of the auxiliary field; the
paper fixes neither, this is the Metropolis reading with the magnitude of the fermionic ratio).
An accepted proposal changes the field before the next site is visited.

The oracle takes every step from the definition: each r_x is the ratio of two stabilised
determinants of the full product (oracle.stable.logdet_green), and the Green's function that is
returned is G_{t-1} = (1 + B_{t-1}...B_1 B_Nt...B_t)^{-1} of the final field, evaluated from
scratch (oracle.force.green_at).  Slow and simple, on purpose; small sizes only.
"""
from __future__ import annotations

import numpy as np

from . import force as _force
from . import stable as _stable


def _wrap(z: complex) -> complex:
    im = float(np.angle(np.exp(1j * z.imag)))
    if im <= -np.pi:
        im += 2 * np.pi
    return complex(z.real, im)


def slice_update(E: np.ndarray, phi: np.ndarray, n_stab: int, t: int, dphi: np.ndarray,
                 u: np.ndarray, w: np.ndarray):
    """Returns (new field row t-1, accepted flags, sum of log r_x over accepted sites (imaginary
    part wrapped to (-pi, pi]), G_{t-1} of the final field, the ratios r_x of every proposal)."""
    phi = phi.copy()
    nx = phi.shape[1]
    ld, _ = _stable.logdet_green(E, phi, n_stab)
    accepted = np.zeros(nx, dtype=bool)
    ratios = np.zeros(nx, dtype=complex)
    total = 0j
    for x in range(nx):
        trial = phi.copy()
        trial[t - 1, x] += dphi[x]
        ld2, _ = _stable.logdet_green(E, trial, n_stab)
        logr = _wrap(ld2 - ld)
        ratios[x] = np.exp(logr)
        if u[x] < np.exp(logr.real) * w[x]:
            accepted[x] = True
            phi = trial
            ld = ld2
            total += logr
    G = _force.green_at(E, phi, n_stab, t - 1)
    return phi[t - 1].copy(), accepted, _wrap(total), G, ratios
