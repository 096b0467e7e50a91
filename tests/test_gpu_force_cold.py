"""The force at low temperature and its finite-difference check at full size, in both paths.

* beta = 64 (Nx = 72, Nt = 512, n_stab = 16, the cold workload's configurations): sampled force
  rows against the oracle (each row a full stabilised evaluation on the rotated field), log det
  and G of the same configurations, and Im F = 1/2 on every entry of every configuration
  (Section 4, Eq. response_result, at Section 7's stabilisation).
* beta = 32 (Nx = 72, Nt = 256, n_stab = 8): all 16 seeded (t, x) entries of the force against
  central finite differences of the oracle's log det (h = 1e-6) on two configurations.
"""
import numpy as np
import pytest

import fd_inputs as fi
from oracle import force as oforce
from oracle import stable

from gpu_helpers import (F_ATOL_FP64, LOGDET_RTOL_FP64, MIXED_TOL, g_scaled_err, logdet_err,
                         mixed_logdet_ok, to_dev)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_02130_gb300 import api

    return api.Context(0)


def _force(ctx, probs, prec):
    from paper_2604_02130_gb300 import api

    b = api.Batch(ctx, to_dev(probs), "force+green", prec)
    r = b.run()
    torch.cuda.synchronize()
    st = b.status()
    assert all(s == 0 for s in st), st
    return (r.logdet.cpu().numpy(), [g.cpu().numpy() for g in r.G],
            [f.cpu().numpy() for f in r.F])


def _scale(M):
    return max(1.0, float(np.abs(M).max())) ** 2


@pytest.mark.parametrize("prec", ["fp64", "3xtf32"])
def test_force_beta64_sampled(ctx, prec):
    probs = fi.workload("cold72", batch=8)
    ld, G, F = _force(ctx, probs, prec)
    inv = 1e-10 if prec == "fp64" else MIXED_TOL[prec]["F_scaled"]
    for c, p in enumerate(probs):
        assert np.abs(F[c].imag - 0.5).max() <= inv * _scale(G[c]), c
    for c in (0, 5):
        p = probs[c]
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, p.n_stab)
        rows = [0, 15, 16, 255, 300, 511]  # block boundaries, inside blocks, the last slice
        ref = oforce.force_rows(p.E, p.phi, p.n_stab, rows)
        if prec == "fp64":
            assert logdet_err(complex(ld[c]), ref_ld) <= LOGDET_RTOL_FP64
            assert g_scaled_err(G[c], ref_G) <= 1e-10
            for r in rows:
                assert np.abs(F[c][r] - ref[r]).max() <= 1e-10 * _scale(ref_G), r
        else:
            tol = MIXED_TOL[prec]
            assert mixed_logdet_ok(complex(ld[c]), ref_ld, float(np.abs(ref_G).max()), prec)
            assert g_scaled_err(G[c], ref_G) <= tol["G_scaled"]
            for r in rows:
                assert np.abs(F[c][r] - ref[r]).max() <= tol["F_scaled"] * _scale(ref_G), r


@pytest.mark.parametrize("prec", ["fp64", "3xtf32"])
def test_force72_fd_all_entries(ctx, prec):
    probs = fi.workload("force72", batch=2)
    ld, G, F = _force(ctx, probs, prec)
    for c, p in enumerate(probs):
        rng = np.random.default_rng([1003, c])
        entries = [(int(rng.integers(p.nt)), int(rng.integers(p.nx))) for _ in range(16)]
        fd = oforce.finite_difference(p.E, p.phi, p.n_stab, entries, h=1e-6)
        got = np.array([F[c][r, x] for r, x in entries])
        # central differences: O(h^2) truncation plus ~1e-16 |log det| / h of rounding
        tol = 2e-6 if prec == "fp64" else 2e-6 + MIXED_TOL[prec]["F_scaled"] * _scale(G[c])
        assert np.abs(got - fd).max() <= tol, (c, np.abs(got - fd).max())
        assert np.abs(got.imag - 0.5).max() <= (F_ATOL_FP64 if prec == "fp64" else tol)
