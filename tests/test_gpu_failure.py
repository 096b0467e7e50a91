"""Failure detection on the GPU without a fault: the boundary and wrap tasks of the force wait on
progress flags with a bound.  With the chain launch skipped (fd_debug_skip_chains) nothing sets
the flags; the waits give up after ~4 s without progress, the kernels return, fd_status reports
FD_ERR_TIMEOUT, and the same context then computes a correct force."""
import time

import numpy as np
import pytest

import fd_inputs as fi
from oracle import force as oforce
from oracle import stable

from gpu_helpers import to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_waits_report_timeout_and_the_context_recovers():
    from paper_2604_02130_gb300 import api

    ctx = api.Context(0)
    probs = fi.workload("tiny8", batch=1)
    b = api.Batch(ctx, to_dev(probs), "force", "fp64")
    ctx.debug_skip_chains(True)
    t0 = time.perf_counter()
    b.run()
    st = ctx.status(1)
    dt = time.perf_counter() - t0
    ctx.debug_skip_chains(False)
    assert st == [-5]  # FD_ERR_TIMEOUT
    assert 2.0 < dt < 60.0  # the waits ran to their bound, and ended
    out = b.run()
    torch.cuda.synchronize()
    assert ctx.status(1) == [0]
    p = probs[0]
    ld, _ = stable.logdet_green(p.E, p.phi, p.n_stab)
    assert abs(complex(out.logdet[0].item()).real - ld.real) <= 1e-8 * abs(ld)
    F = oforce.force(p.E, p.phi, p.n_stab)
    assert np.abs(out.F[0].cpu().numpy() - F).max() < 1e-9
