"""Shared helpers for the GPU parity tests (device transfer, oracle comparison)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

# Tolerances.  FP64 path: |d logdet| / |logdet| <= 1e-8 (the stated target), G and F compared
# element-wise in absolute terms (entries are O(1): |G_ij| <= ~1, |F| ~ 1).
LOGDET_RTOL_FP64 = 1e-8
G_ATOL_FP64 = 1e-8
F_ATOL_FP64 = 1e-8


def to_dev(probs, n_stab=None):
    dev = torch.device("cuda", 0)
    out = []
    for p in probs:
        out.append((torch.from_numpy(np.ascontiguousarray(p.E)).to(dev),
                    torch.from_numpy(np.ascontiguousarray(p.Einv)).to(dev),
                    torch.from_numpy(np.ascontiguousarray(p.phi)).to(dev),
                    p.n_stab if n_stab is None else n_stab))
    return out


def logdet_err(gpu: complex, ref: complex) -> float:
    """max(|d Re|, |d Im mod 2pi|) / max(1, |ref|)"""
    dre = abs(gpu.real - ref.real)
    dim = abs(np.angle(np.exp(1j * (gpu.imag - ref.imag))))
    return max(dre, dim) / max(1.0, abs(ref))
