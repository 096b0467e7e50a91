"""Product form of the slice exponential for the intermediate-volume variant (Section 8).

Test infrastructure only (see the package header).

Section 8 replaces the slice exponential by the degree-n Taylor polynomial of exp written as a
product of n linear factors,
    T_n(K) = sum_{j=0}^{n} K^j / j!  =  prod_{k=1}^{n} (1 + gamma_k K),
so that applying it to a vector costs n products with the sparse K instead of one dense product
(O(n q V) per vector, q non-zeros per row).  The paper fixes the gamma_k by exactly this property
(the product equals the Taylor series to the same order n, error O(delta^{n+1})) and suggests
n = 4.  Since T_n(0) = 1, T_n(x) = prod_k (1 - x / x_k) over the n roots x_k of T_n, hence
gamma_k = -1 / x_k (real or complex-conjugate pairs).

For this model K = delta*kappa*A and the slice is B_t = T_n(K) diag(e^{i phi_t}): the Trotter
split of the paper's generic M_t keeps the field phase exact and approximates only the hopping
exponential.  T_n(K) is a real symmetric polynomial in A, so every quantity of the stabilised
method (log det, G) is the one of Section 7 with E replaced by T_n(K).
"""
from __future__ import annotations

import math

import numpy as np

from . import stable as _stable


def taylor_factors(n: int) -> np.ndarray:
    """gamma_1..gamma_n (complex) with prod_k (1 + gamma_k x) = sum_{j<=n} x^j / j!."""
    if n < 1:
        raise ValueError("n >= 1")
    # numpy.roots takes the coefficients from the highest power down
    coeffs = [1.0 / math.factorial(j) for j in range(n, -1, -1)]
    roots = np.roots(coeffs)
    return np.sort_complex(-1.0 / roots)


def taylor_matrix(K: np.ndarray, n: int) -> np.ndarray:
    """T_n(K) = sum_{j=0}^{n} K^j / j! (the definition, by powers)."""
    out = np.eye(K.shape[0])
    term = np.eye(K.shape[0])
    for j in range(1, n + 1):
        term = term @ K / j
        out = out + term
    return out


def product_form_matrix(K: np.ndarray, gammas) -> np.ndarray:
    """prod_k (1 + gamma_k K), multiplied out densely (complex; real up to rounding)."""
    out = np.eye(K.shape[0], dtype=complex)
    for g in gammas:
        out = out @ (np.eye(K.shape[0]) + g * K)
    return out


def slice_matrix(A: np.ndarray, delta: float, kappa: float, n: int) -> np.ndarray:
    """The hopping factor of a slice in the product form: T_n(delta*kappa*A), real symmetric."""
    return taylor_matrix(delta * kappa * A, n)


def logdet_green(A: np.ndarray, delta: float, kappa: float, n: int, phi: np.ndarray,
                 n_stab: int):
    """log det(1 + B_Nt...B_1) and G with B_t = T_n(delta*kappa*A) diag(e^{i phi_t}), by the
    stabilised method (the low-temperature variant of Section 9: slices applied in the product
    form, QR every n_stab slices)."""
    return _stable.logdet_green(slice_matrix(A, delta, kappa, n), phi, n_stab)
