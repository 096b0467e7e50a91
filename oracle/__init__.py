"""CPU oracle for the stabilised fermion determinant -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 (numpy/scipy, mpmath for the high-precision pin) implementation of what the
GPU library computes, written from the paper "Stable and Efficient Algorithms for the Fermion
Determinant" (arXiv 2604.02130).  It shares no code with the CUDA path and never imports it.
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may
import anything from here; the product path must not.

Quantities (Section 2, the "sausage"):
    B_t  = E diag(exp(i phi_t)),  E = exp(delta*kappa*A)          (time slice t = 1..Nt)
    P    = B_Nt ... B_2 B_1                                        (block-matrix order, see below)
    logdet = log det(1 + P),  G = (1 + P)^{-1}                      (Eq. hamiltonian_alg)
    F[t, x] = d logdet / d phi[t, x] = i (1 - [G_{t-1}]_{xx}),
    G_{t-1} = (1 + B_{t-1} ... B_1 B_Nt ... B_t)^{-1}               (Eq. response_result)

Modules:
    plain          -- the definitions written out (product, slogdet, inverse); small beta only.
    fermion_matrix -- brute force on the full (Nt*Nx)^2 fermion matrix M (Section 2).
    stable         -- the stabilised dense method of Section 7 (UDV form, QR re-orthogonalisation
                      every n_stab slices as in Section 9, scale-separated assembly).
    naive          -- the naive small-volume algorithm of Section 6 (eigen-decomposed product).
    free           -- closed form at phi = 0.
    force          -- the force from Eq. response_result, and central finite differences.
    highprec       -- the plain product in mpmath at 250 digits (low-temperature pin).
    unequal        -- the unequal-time Green's function G(tau, 0) (Section 4.2, Section 7
                      steps 7-9).
    observables    -- fermion number and single-time response traces tr(O G_r) (Section 4.1).
    bss            -- local (BSS) updates of the field at one time slice (Section 3).
    product_form   -- the slice exponential as a product of n linear factors in the sparse
                      hopping matrix (Section 8, the intermediate-volume variant).

Parity pins (tests/test_oracle_*.py) tie every module to something other than itself.
"""
from . import (plain, fermion_matrix, stable, naive, free, force, unequal, observables,  # noqa: F401
               bss, product_form)

__all__ = ["plain", "fermion_matrix", "stable", "naive", "free", "force", "unequal", "observables",
           "bss", "product_form", "wrap_phase"]


def wrap_phase(z):
    """Map the imaginary part of a complex log to (-pi, pi] (the log's branch, Section 7 step 5)."""
    import numpy as np

    z = np.asarray(z, dtype=complex)
    im = np.angle(np.exp(1j * z.imag))
    im = np.where(im <= -np.pi, im + 2 * np.pi, im)
    return z.real + 1j * im
