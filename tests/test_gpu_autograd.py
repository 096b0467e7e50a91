"""The autograd function FermionLogDet (the binding's differentiable log det) against the oracle.

phi is real and log det complex; torch hands backward the conjugate-Wirtinger gradient of a real
loss, so d Re(logdet)/d phi = Re F and d Im(logdet)/d phi = Im F with F = d logdet / d phi (the
force of Eq. response_result).  Checked against oracle.force, and against central finite
differences of the library's own forward at a few entries.  The case keeps Im log det far from
the branch cut at +-pi.
"""
import numpy as np
import pytest

import fd_inputs as fi
from oracle import force as oforce
from oracle import stable

from gpu_helpers import F_ATOL_FP64, LOGDET_RTOL_FP64, logdet_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tensors(p):
    dev = torch.device("cuda", 0)
    E = torch.from_numpy(np.ascontiguousarray(p.E)).to(dev)
    Einv = torch.from_numpy(np.ascontiguousarray(p.Einv)).to(dev)
    phi = torch.from_numpy(np.ascontiguousarray(p.phi)).to(dev)
    return E, Einv, phi


def test_gradients_of_real_and_imaginary_parts():
    from paper_2604_02130_gb300 import api

    p = fi.make_problem(2, 16, 2.0, 2.0, 4, 1200, 1)
    ld_ref, _ = stable.logdet_green(p.E, p.phi, p.n_stab)
    assert abs(abs(ld_ref.imag) - np.pi) > 0.5
    F = oforce.force(p.E, p.phi, p.n_stab)
    E, Einv, phi0 = _tensors(p)
    for part, want in (("real", F.real), ("imag", F.imag)):
        phi = phi0.clone().requires_grad_(True)
        ld = api.FermionLogDet.apply(phi, E, Einv, p.n_stab)
        assert logdet_err(complex(ld.item()), ld_ref) <= LOGDET_RTOL_FP64
        getattr(ld, part).backward()
        torch.cuda.synchronize()
        assert np.abs(phi.grad.cpu().numpy() - want).max() <= F_ATOL_FP64, part


def test_gradient_matches_finite_differences_of_the_forward():
    from paper_2604_02130_gb300 import api

    p = fi.make_problem(2, 16, 2.0, 2.0, 4, 1200, 2)
    E, Einv, phi0 = _tensors(p)
    phi = phi0.clone().requires_grad_(True)
    ld = api.FermionLogDet.apply(phi, E, Einv, p.n_stab)
    ld.real.backward()
    g = phi.grad.cpu().numpy()
    h = 1e-5
    rng = np.random.default_rng(3)
    for _ in range(6):
        t, x = int(rng.integers(p.nt)), int(rng.integers(p.nx))
        vals = []
        for s in (+1, -1):
            q = phi0.clone()
            q[t, x] += s * h
            vals.append(complex(api.FermionLogDet.apply(q, E, Einv, p.n_stab).item()).real)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[t, x]) < 1e-6 * max(1.0, abs(g[t, x])), (t, x, fd, g[t, x])


def test_batched_gradient_and_lazy_forward():
    """A batch of fields through one call: the forward runs the log det kernels only (no force
    sweep, no checkpoints); the backward's force sweep gives every configuration's gradient."""
    from paper_2604_02130_gb300 import api

    probs = [fi.make_problem(3, 32, 4.0, 3.0, 8, 1201, c) for c in range(5)]
    E, Einv, _ = _tensors(probs[0])
    phi0 = torch.stack([_tensors(p)[2] for p in probs])
    ctx = api.default_context()
    ref_plan = api.Batch(ctx, [(E, Einv, phi0[k], 8) for k in range(5)], "logdet").plan()
    with torch.no_grad():
        ld = api.FermionLogDet.apply(phi0, E, Einv, 8)
    torch.cuda.synchronize()
    # the log det plan's launches only (chain segments and merge, or one log det kernel)
    assert ctx.last_launch_count() == len(ref_plan)
    assert all(r["kernel"] % 4 in (0, 1) or r["kernel"] == 8 for r in ref_plan)
    phi = phi0.clone().requires_grad_(True)
    ld2 = api.FermionLogDet.apply(phi, E, Einv, 8)
    assert torch.equal(ld, ld2.detach())
    w = torch.tensor([0.5 - 0.25j, 1.0, -2.0 + 1j, 0.0, 1j], dtype=torch.complex128,
                     device=phi.device)
    (ld2 * w).real.sum().backward()  # torch hands backward grad_out = conj(w)
    torch.cuda.synchronize()
    g = phi.grad.cpu().numpy()
    for c, p in enumerate(probs):
        ref_ld, _ = stable.logdet_green(p.E, p.phi, p.n_stab)
        assert logdet_err(complex(ld[c].item()), ref_ld) <= LOGDET_RTOL_FP64
        F = oforce.force(p.E, p.phi, p.n_stab)
        want = (w[c].item() * F).real  # d Re(w logdet) / d phi = Re(w F)
        assert np.abs(g[c] - want).max() <= F_ATOL_FP64, c
