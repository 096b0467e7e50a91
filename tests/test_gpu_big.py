"""The streamed tensor-core kernels (size classes whose TF32 operands do not fit the shared-memory
tensor tile: Nx = 98, 128, 288 in the split-TF32 mode) against the CPU oracle.

Log det and G through the time-parallel split (few configurations) and through one chain per
configuration (a batch larger than the SM count), and the force (chains on the tensor cores,
FP64 boundary Green's functions, wraps on the tensor cores), every entry compared, within the
mixed path's stated bounds (gpu_helpers.MIXED_TOL)."""
import numpy as np
import pytest

import fd_inputs as fi
from oracle import force as oforce
from oracle import stable

from gpu_helpers import MIXED_TOL, g_scaled_err, mixed_logdet_ok, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BIG = [  # L, nt, beta, U, n_stab
    (7, 32, 2.0, 3.0, 8),     # Nx = 98: one M-tile of E, ragged K (112)
    (8, 32, 2.0, 3.0, 16),    # Nx = 128
    (12, 32, 2.0, 3.0, 16),   # Nx = 288: three M-tiles of E, five of Y^T, two TMEM passes
]


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_02130_gb300 import api

    return api.Context(0)


def _run(ctx, probs, want, prec):
    from paper_2604_02130_gb300 import api

    b = api.Batch(ctx, to_dev(probs), want, prec)
    r = b.run()
    torch.cuda.synchronize()
    st = b.status()
    assert all(s == 0 for s in st), st
    return (b.plan(), r.logdet.cpu().numpy(), [g.cpu().numpy() for g in r.G] if r.G else None,
            [f.cpu().numpy() for f in r.F] if r.F else None)


def _check_ld_g(prec, p, ld, G):
    tol = MIXED_TOL[prec]
    ref_ld, ref_G = stable.logdet_green(p.E, p.phi, p.n_stab)
    assert mixed_logdet_ok(complex(ld), ref_ld, float(np.abs(ref_G).max()), prec), (p.nx, ld, ref_ld)
    assert g_scaled_err(G, ref_G) <= tol["G_scaled"], (p.nx, g_scaled_err(G, ref_G))
    return ref_G


@pytest.mark.parametrize("L,nt,beta,U,n_stab", BIG)
def test_streamed_plan_codes(ctx, L, nt, beta, U, n_stab):
    from paper_2604_02130_gb300 import api

    probs = [fi.make_problem(L, nt, beta, U, n_stab, 90, c) for c in range(2)]
    plan = api.Batch(ctx, to_dev(probs), "force+green", "3xtf32").plan()
    # chains 1 and wraps 3, +4 on the tensor cores, +16 streamed; the boundary Green's functions
    # (2) in double-float: 18
    assert [g["kernel"] for g in plan] == [21, 18, 23]


@pytest.mark.parametrize("prec", ["3xtf32", "tf32"])
@pytest.mark.parametrize("L,nt,beta,U,n_stab", BIG)
def test_streamed_logdet_green_split(ctx, prec, L, nt, beta, U, n_stab):
    probs = [fi.make_problem(L, nt, beta, U, n_stab, 91, c) for c in range(3)]
    _, ld, G, _ = _run(ctx, probs, "green", prec)
    for c, p in enumerate(probs):
        _check_ld_g(prec, p, ld[c], G[c])


def test_streamed_logdet_green_one_chain_per_config(ctx):
    # more configurations than SMs: no time-parallel split, one forward chain per configuration
    probs = [fi.make_problem(7, 16, 1.0, 3.0, 8, 92, c) for c in range(160)]
    plan, ld, G, _ = _run(ctx, probs, "green", "3xtf32")
    assert plan[0]["kernel"] == 21 and len(plan) == 1
    for c in range(0, 160, 23):
        _check_ld_g("3xtf32", probs[c], ld[c], G[c])


@pytest.mark.parametrize("prec", ["3xtf32", "tf32"])
@pytest.mark.parametrize("L,nt,beta,U,n_stab", BIG)
def test_streamed_force(ctx, prec, L, nt, beta, U, n_stab):
    probs = [fi.make_problem(L, nt, beta, U, n_stab, 93, c) for c in range(2)]
    _, ld, G, F = _run(ctx, probs, "force+green", prec)
    tol = MIXED_TOL[prec]
    for c, p in enumerate(probs):
        ref_G = _check_ld_g(prec, p, ld[c], G[c])
        ref_F = oforce.force(p.E, p.phi, p.n_stab)
        scale = max(1.0, float(np.abs(ref_G).max())) ** 2
        assert float(np.abs(F[c] - ref_F).max()) / scale <= tol["F_scaled"], (p.nx, c)
        assert float(np.abs(F[c].imag - 0.5).max()) <= tol["F_scaled"] * scale
