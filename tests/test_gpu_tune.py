"""The QR-interval tuner (fd_tune_nstab_stats) on the low-temperature workload: beta = 64,
Nx = 72, Nt = 512, n_stab autotuned among {8, 16} (Section 9: stabilise every beta_0/delta
slices) under an error budget against FP64; the tuned call then matches the oracle within that
budget on the tuning configuration and within the mixed path's stated bounds on the others."""
import numpy as np
import pytest

import fd_inputs as fi
from oracle import stable

from gpu_helpers import MIXED_TOL, g_scaled_err, logdet_err, mixed_logdet_ok, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("budget", [1e-4, 1e-6])
def test_tune_cold72_nstab(budget):
    from paper_2604_02130_gb300 import api

    ctx = api.Context(0)
    probs = fi.workload("cold72", batch=4)
    tens = to_dev(probs)
    cands = [8, 16]
    best, err, ms = ctx.tune_nstab(tens[0], cands, budget, "3xtf32", stats=True)
    assert all(e >= 0 for e in err) and all(t > 0 for t in ms)
    ok = [c for c, e in zip(cands, err) if e <= budget]
    if not ok:
        assert best == 0
        ctx.close()
        return
    # the fastest candidate within the budget
    assert best == min(ok, key=lambda c: (ms[cands.index(c)], -c))
    b = api.Batch(ctx, [(E, Ei, phi, best) for (E, Ei, phi, _) in tens], "green", "3xtf32")
    r = b.run()
    torch.cuda.synchronize()
    assert all(s == 0 for s in b.status())
    for c, p in enumerate(probs):
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, p.n_stab)
        ld = complex(r.logdet[c].item())
        G = r.G[c].cpu().numpy()
        if c == 0:  # the tuning configuration: within the budget (plus the FP64 path's error)
            assert logdet_err(ld, ref_ld) <= budget + 1e-12
            assert g_scaled_err(G, ref_G) <= budget + 1e-12
        else:
            assert mixed_logdet_ok(ld, ref_ld, float(np.abs(ref_G).max()), "3xtf32")
            assert g_scaled_err(G, ref_G) <= MIXED_TOL["3xtf32"]["G_scaled"]
    ctx.close()
