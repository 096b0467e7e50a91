"""GPU parity of the single-time observables of Section 4.1 (fd_observables) against the oracle.

Fermion number n = 1 - tr G / V and response traces R[r] = tr(O G_r) for the hopping matrix A
and for random non-symmetric operators: element-wise against oracle.observables on small and
sampled full-size configurations, plus properties that hold at any size (tr G_r independent of
r and equal to V (1 - n); -delta sum_r tr(A G_r) = d log det / d kappa by finite differences of
the oracle's log det).
"""
import numpy as np
import pytest

import fd_inputs as fi
from oracle import force as oforce
from oracle import observables, stable

from gpu_helpers import MIXED_TOL, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_02130_gb300 import api

    return api.Context(0)


def _ops(probs, kind, seed=7):
    dev = torch.device("cuda", 0)
    out = []
    for c, p in enumerate(probs):
        if kind == "A":
            O = p.A
        elif kind == "I":
            O = np.eye(p.nx)
        else:
            O = np.random.default_rng([seed, c]).normal(size=(p.nx, p.nx))
        out.append(torch.from_numpy(np.ascontiguousarray(O)).to(dev))
    return out


def _run(ctx, probs, want, prec="fp64", ops=None):
    from paper_2604_02130_gb300 import api

    b = api.Batch(ctx, to_dev(probs), want, prec, ops)
    r = b.run()
    torch.cuda.synchronize()
    st = b.status()
    assert all(s == 0 for s in st), st
    out = {"logdet": r.logdet.cpu().numpy()}
    if r.nferm is not None:
        out["nferm"] = r.nferm.cpu().numpy()
    if r.R is not None:
        out["R"] = [x.cpu().numpy() for x in r.R]
    if r.F is not None:
        out["F"] = [x.cpu().numpy() for x in r.F]
    if r.G is not None:
        out["G"] = [x.cpu().numpy() for x in r.G]
    return out


def _ref_traces(p, O):
    """tr(O G_r) and max_r max|G_r| from independent stabilised evaluations."""
    R, gmax = [], 0.0
    for r in range(p.nt):
        Gr = oforce.green_at(p.E, p.phi, p.n_stab, r)
        R.append(np.trace(O @ Gr))
        gmax = max(gmax, float(np.abs(Gr).max()))
    return np.array(R), gmax


SMALL = [  # L, nt, beta, U, n_stab
    (2, 16, 2.0, 2.0, 4),
    (2, 16, 2.0, 2.0, 1),
    (2, 16, 2.0, 2.0, 16),
    (3, 24, 3.0, 3.0, 8),
    (5, 16, 2.0, 3.0, 8),
    (6, 16, 4.0, 3.0, 8),
]


@pytest.mark.parametrize("L,nt,beta,U,n_stab", SMALL)
@pytest.mark.parametrize("op", ["A", "rand"])
def test_response_fp64(ctx, L, nt, beta, U, n_stab, op):
    probs = [fi.make_problem(L, nt, beta, U, n_stab, 101, c) for c in range(2)]
    ops = _ops(probs, op)
    out = _run(ctx, probs, "nferm+response", ops=ops)
    for c, p in enumerate(probs):
        O = ops[c].cpu().numpy()
        ref, gmax = _ref_traces(p, O)
        scale = max(1.0, float(np.abs(O).sum(axis=1).max()))
        assert np.abs(out["R"][c] - ref).max() <= 1e-8 * scale * max(1.0, gmax) ** 2
        n_ref = observables.fermion_number(p.E, p.phi, n_stab)
        assert abs(out["nferm"][c] - n_ref) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "3xtf32", "tf32"])
def test_nferm_single_kernel(ctx, prec):
    """n alone runs the log det/G kernel; batch18 (256 configurations), every one compared."""
    probs = fi.workload("batch18")
    out = _run(ctx, probs, "nferm+green", prec)
    tol = 1e-10 if prec == "fp64" else MIXED_TOL[prec]["G_scaled"]
    worst = 0.0
    for c, p in enumerate(probs):
        _, G = stable.logdet_green(p.E, p.phi, p.n_stab)
        n_ref = 1.0 - np.trace(G) / p.nx
        worst = max(worst, abs(out["nferm"][c] - n_ref) / max(1.0, float(np.abs(G).max())) ** 2)
        # the same call's G gives the same n
        assert abs(out["nferm"][c] - (1.0 - np.trace(out["G"][c]) / p.nx)) <= 1e-12
    assert worst <= tol


def test_response_with_force_and_green(ctx):
    probs = [fi.make_problem(3, 24, 3.0, 3.0, 8, 102, c) for c in range(3)]
    ops = _ops(probs, "rand")
    out = _run(ctx, probs, "force+green+nferm+response", ops=ops)
    for c, p in enumerate(probs):
        ref_F = oforce.force(p.E, p.phi, 8)
        _, ref_G = stable.logdet_green(p.E, p.phi, 8)
        assert np.abs(out["F"][c] - ref_F).max() <= 1e-8
        assert np.abs(out["G"][c] - ref_G).max() <= 1e-8
        ref, gmax = _ref_traces(p, ops[c].cpu().numpy())
        assert np.abs(out["R"][c] - ref).max() <= 1e-8 * p.nx * max(1.0, gmax) ** 2


def test_trace_invariance_batch18(ctx):
    """O = 1: tr G_r = V (1 - n) for every slice r and every configuration (any size)."""
    probs = fi.workload("batch18")
    out = _run(ctx, probs, "nferm+response", ops=_ops(probs, "I"))
    worst = 0.0
    for c, p in enumerate(probs):
        R = out["R"][c]
        target = p.nx * (1.0 - out["nferm"][c])
        worst = max(worst, float(np.abs(R - target).max()))
    assert worst <= 1e-9


def _kappa_derivative(p, h=1e-4):
    def ld(kappa):
        return stable.logdet_green(fi.hopping_exp(p.A, p.delta, kappa), p.phi, p.n_stab)[0]

    f0 = ld(1.0)
    vals = []
    for k in (-2, -1, 1, 2):
        v = ld(1.0 + k * h)
        vals.append((v.real - f0.real) + 1j * np.angle(np.exp(1j * (v.imag - f0.imag))))
    return (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)


@pytest.mark.parametrize("prec", ["fp64", "3xtf32"])
def test_hopping_response_force72(ctx, prec):
    """Nx = 72, beta = 32, Nt = 256: -delta sum_r tr(A G_r) against d log det / d kappa."""
    probs = fi.workload("force72", batch=2)
    out = _run(ctx, probs, "force+response", prec, ops=_ops(probs, "A"))
    p = probs[1]
    got = -p.delta * out["R"][1].sum()
    ref = _kappa_derivative(p)
    tol = 1e-7 if prec == "fp64" else 1e-3
    assert abs(got - ref) <= tol * max(1.0, abs(ref))
    # sampled slices element-wise
    for r in (0, 3, 4, 5, 8, 131, 255):
        Gr = oforce.green_at(p.E, p.phi, p.n_stab, r)
        ref_r = np.trace(p.A @ Gr)
        t = 1e-8 if prec == "fp64" else MIXED_TOL[prec]["G_scaled"]
        assert abs(out["R"][1][r] - ref_r) <= t * p.nx * max(1.0, float(np.abs(Gr).max())) ** 2


@pytest.mark.parametrize("prec", ["3xtf32", "tf32"])
@pytest.mark.parametrize("L,nt,beta,U,n_stab", [(2, 16, 2.0, 2.0, 4), (3, 64, 8.0, 3.0, 8),
                                                (6, 32, 4.0, 3.0, 8)])
def test_response_mixed(ctx, prec, L, nt, beta, U, n_stab):
    probs = [fi.make_problem(L, nt, beta, U, n_stab, 103, c) for c in range(2)]
    ops = _ops(probs, "rand")
    out = _run(ctx, probs, "nferm+response", prec, ops=ops)
    tol = MIXED_TOL[prec]["G_scaled"]
    for c, p in enumerate(probs):
        O = ops[c].cpu().numpy()
        ref, gmax = _ref_traces(p, O)
        scale = float(np.abs(O).sum(axis=1).max())
        assert np.abs(out["R"][c] - ref).max() <= tol * scale * max(1.0, gmax) ** 2


def test_observables_validation(ctx):
    from paper_2604_02130_gb300 import api

    p = fi.make_problem(2, 16, 2.0, 2.0, 4, 104, 0)
    (E, Einv, phi, ns), = to_dev([p])
    ops = _ops([p], "A")
    with pytest.raises(ValueError):
        api.Batch(ctx, [(E, Einv, phi, ns)], "response")  # no operators
    with pytest.raises(ValueError):
        api.Batch(ctx, [(E, Einv, phi, ns)], "gtau+nferm")
    with pytest.raises(api.FdError):
        api.Batch(ctx, [(E, None, phi, ns)], "response", operators=ops).run()  # needs E^{-1}
    b = api.Batch(ctx, [(E, Einv, phi, ns)], "nferm+response", operators=ops)
    lib = ctx.lib
    ld = torch.empty(2, dtype=torch.float64, device="cuda")
    # O without R
    rc = lib.fd_observables(ctx.h, 1, b.problems, ld.data_ptr(), None, None, None, b._Op, None,
                            0, None)
    assert rc == -1
