"""GPU parity of the unequal-time Green's function G(tau, 0) (Section 4.2) against the oracle.

Small lattices are compared block by block against the brute-force column of M^{-1}
(oracle.fermion_matrix.inverse_column) and the stabilised Section 7 steps 7-9 restatement
(oracle.unequal.green_tau_stable); the full-size workloads on sampled configurations and
time slices, plus properties that hold at any size (G(0, 0) = G of the same call, and one-slice
propagation G(t, 0) = B_t G(t-1, 0) where the forward and backward wraps of a block meet).
"""
import numpy as np
import pytest

import fd_inputs as fi
from oracle import fermion_matrix, stable, unequal
from oracle import force as oforce
from oracle import plain

from gpu_helpers import MIXED_TOL, logdet_err, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP64: |dG(tau, 0)| <= 1e-8 max(1, max|G(tau, 0)|)^2 (the conditioning of the boundary solve
# grows like |G|^2, as for the equal-time G).
GT_TOL_FP64 = 1e-8


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_02130_gb300 import api

    return api.Context(0)


def _run(ctx, probs, want, prec="fp64"):
    from paper_2604_02130_gb300 import api

    b = api.Batch(ctx, to_dev(probs), want, prec)
    r = b.run()
    torch.cuda.synchronize()
    st = b.status()
    assert all(s == 0 for s in st), st
    out = {"logdet": r.logdet.cpu().numpy(),
           "Gtau": [g.cpu().numpy() for g in r.Gtau]}
    if r.G is not None:
        out["G"] = [g.cpu().numpy() for g in r.G]
    if r.F is not None:
        out["F"] = [f.cpu().numpy() for f in r.F]
    return out


def _scaled(a, ref):
    return float(np.abs(a - ref).max()) / max(1.0, float(np.abs(ref).max())) ** 2


SMALL = [  # L, nt, beta, U, n_stab
    (2, 16, 2.0, 2.0, 4),      # the tiny workload shape
    (2, 16, 2.0, 2.0, 1),      # every slice a block boundary (no wraps)
    (2, 16, 2.0, 2.0, 16),     # a single block (no boundary solve; 1 - G at the top)
    (2, 12, 1.5, 2.0, 6),      # even n_stab: backward wraps one longer than forward
    (3, 24, 3.0, 3.0, 8),      # Nx = 18
    (4, 16, 2.0, 3.0, 4),      # Nx = 32
    (5, 16, 2.0, 3.0, 8),      # Nx = 50: ragged tiles
]


@pytest.mark.parametrize("L,nt,beta,U,n_stab", SMALL)
def test_gtau_brute_force(ctx, L, nt, beta, U, n_stab):
    probs = [fi.make_problem(L, nt, beta, U, n_stab, 91, c) for c in range(2)]
    out = _run(ctx, probs, "gtau+green")
    for c, p in enumerate(probs):
        ref = fermion_matrix.inverse_column(p.E, p.phi, 0)
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, n_stab)
        assert logdet_err(complex(out["logdet"][c]), ref_ld) <= 1e-8
        assert np.abs(out["G"][c] - ref_G).max() <= 1e-8
        assert out["Gtau"][c].shape == (nt, p.nx, p.nx)
        for tau in range(nt):
            assert _scaled(out["Gtau"][c][tau], ref[tau]) <= GT_TOL_FP64, tau


@pytest.mark.parametrize("L,nt,beta,U,n_stab", [(2, 16, 2.0, 2.0, 4), (3, 24, 3.0, 3.0, 8),
                                                (6, 16, 4.0, 3.0, 8)])
def test_gtau_with_force(ctx, L, nt, beta, U, n_stab):
    """G(tau, 0), G and F from one call (the boundary solve with two right-hand sides)."""
    probs = [fi.make_problem(L, nt, beta, U, n_stab, 92, c) for c in range(2)]
    out = _run(ctx, probs, "gtau+force+green")
    for c, p in enumerate(probs):
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, n_stab)
        ref_F = oforce.force(p.E, p.phi, n_stab)
        ref = unequal.green_tau_stable(p.E, p.phi, n_stab)
        assert logdet_err(complex(out["logdet"][c]), ref_ld) <= 1e-8
        assert np.abs(out["G"][c] - ref_G).max() <= 1e-8
        assert np.abs(out["F"][c] - ref_F).max() <= 1e-8
        for tau in range(nt):
            assert _scaled(out["Gtau"][c][tau], ref[tau]) <= GT_TOL_FP64, tau


def _meeting_propagation(p, Gt, worst):
    """|G(m, 0) - B_m G(m-1, 0)| in every block at m = t0 + (n_stab-1)//2 + 1, where G(m-1, 0)
    comes from forward wraps off the block's lower boundary and G(m, 0) from backward wraps off
    its upper one (1 - G for the last block): two independent routes."""
    h = (p.n_stab - 1) // 2
    for t0 in range(0, p.nt, p.n_stab):
        m = t0 + h + 1
        if m >= t0 + p.n_stab:
            continue
        prop = plain.slice_matrix(p.E, p.phi[m - 1]) @ Gt[m - 1]
        worst = max(worst, _scaled(Gt[m], prop))
    return worst


def test_gtau_batch18_sampled(ctx):
    """The 256-configuration Nx = 18 workload: three configurations against the oracle on
    every slice; all of them on G(0, 0) = G and on the propagation check inside every block."""
    probs = fi.workload("batch18")
    out = _run(ctx, probs, "gtau+green")
    worst = 0.0
    for c, p in enumerate(probs):
        assert np.abs(out["Gtau"][c][0] - out["G"][c]).max() == 0.0
        worst = _meeting_propagation(p, out["Gtau"][c], worst)
    assert worst <= 1e-9
    for c in (0, 101, 255):
        p = probs[c]
        ref = unequal.green_tau_stable(p.E, p.phi, p.n_stab)
        for tau in range(p.nt):
            assert _scaled(out["Gtau"][c][tau], ref[tau]) <= GT_TOL_FP64, (c, tau)


@pytest.mark.parametrize("name,taus", [("force72", (0, 1, 4, 5, 8, 100, 131, 255)),
                                       ("cold72", (0, 7, 8, 9, 16, 250, 511))])
def test_gtau_nx72_sampled(ctx, name, taus):
    probs = fi.workload(name, batch=2)
    out = _run(ctx, probs, "gtau")
    p = probs[1]
    ref = unequal.green_tau_stable(p.E, p.phi, p.n_stab, taus=taus)
    for tau in taus:
        assert _scaled(out["Gtau"][1][tau], ref[tau]) <= GT_TOL_FP64, tau
    assert _meeting_propagation(p, out["Gtau"][1], 0.0) <= 1e-9


@pytest.mark.parametrize("prec", ["3xtf32", "tf32"])
@pytest.mark.parametrize("L,nt,beta,U,n_stab", [(2, 16, 2.0, 2.0, 4), (3, 64, 8.0, 3.0, 8),
                                                (6, 32, 4.0, 3.0, 8)])
def test_gtau_mixed(ctx, prec, L, nt, beta, U, n_stab):
    """Tensor-core chains, FP64 boundary solves and G(tau, 0) wraps."""
    probs = [fi.make_problem(L, nt, beta, U, n_stab, 93, c) for c in range(2)]
    out = _run(ctx, probs, "gtau+force", prec)
    tol = MIXED_TOL[prec]
    for c, p in enumerate(probs):
        ref = unequal.green_tau_stable(p.E, p.phi, n_stab)
        for tau in range(nt):
            assert _scaled(out["Gtau"][c][tau], ref[tau]) <= tol["G_scaled"], tau
        ref_F = oforce.force(p.E, p.phi, n_stab)
        scale = max(1.0, float(np.abs(ref_F).max())) ** 2
        assert float(np.abs(out["F"][c] - ref_F).max()) / scale <= tol["F_scaled"]


def test_gtau_uneven_classes(ctx):
    """Several size classes in one call (concurrent branches), FP64."""
    shapes = [(2, 32, 8), (3, 16, 4), (4, 16, 8), (2, 8, 8), (5, 8, 2)]
    probs = [fi.make_problem(L, nt, nt / 16.0, 3.0, ns, 94, c)
             for c, (L, nt, ns) in enumerate(shapes)]
    out = _run(ctx, probs, "gtau")
    for c, p in enumerate(probs):
        ref = fermion_matrix.inverse_column(p.E, p.phi, 0)
        for tau in range(p.nt):
            assert _scaled(out["Gtau"][c][tau], ref[tau]) <= GT_TOL_FP64, (c, tau)


def test_gtau_validation(ctx):
    from paper_2604_02130_gb300 import api

    p = fi.make_problem(2, 16, 2.0, 2.0, 4, 95, 0)
    (E, Einv, phi, ns), = to_dev([p])
    with pytest.raises(api.FdError):
        api.Batch(ctx, [(E, None, phi, ns)], "gtau").run()  # E^{-1} is needed
    b = api.Batch(ctx, [(E, Einv, phi, ns)], "gtau")
    with pytest.raises(ValueError):
        b.graph()
    lib = ctx.lib
    ld = torch.empty(2, dtype=torch.float64, device="cuda")
    rc = lib.fd_green_tau(ctx.h, 1, b.problems, ld.data_ptr(), None, None, None, 0, None)
    assert rc == -1  # FD_ERR_INVALID: null Gtau array
