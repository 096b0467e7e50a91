"""Batched stabilised fermion determinants on NVIDIA GB300 (sm_103a).

log det(1 + B_Nt...B_1), the Green's function (1 + B_Nt...B_1)^{-1} and the HMC force
d log det / d phi, and the unequal-time Green's function G(tau, 0), for B_t = exp(delta*kappa*A) diag(exp(i phi_t)), by the stabilised dense method
of arXiv 2604.02130 (Section 7), computed by the CUDA library libfd.so through its C ABI
(include/fd.h).  Importing this package does not load the library; the first Context does, and
fails loudly if the CUDA library cannot be loaded (there is no CPU fallback).
"""
from .flops import force_flops, fwd_flops  # noqa: F401

__all__ = ["Context", "Batch", "logdet", "green", "force", "green_tau", "observables",
           "bss_update", "BssSlices", "green_sparse", "taylor_factors", "FermionLogDet",
           "fwd_flops", "force_flops"]


def __getattr__(name):
    if name in ("Context", "Batch", "logdet", "green", "force", "green_tau", "observables",
                "bss_update", "BssSlices", "green_sparse", "taylor_factors", "FermionLogDet",
                "Result",
                "FdError", "default_context"):
        from . import api

        return getattr(api, name)
    raise AttributeError(name)
