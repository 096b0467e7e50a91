"""GPU parity of the FP64 path against the CPU oracle, through the C ABI (via the binding).

Small sizes are compared element by element (log det, every entry of G and of F); the full-size
workloads are compared on sampled configurations (all outputs) plus exact invariants on every
configuration (particle-hole phase of log det, Re G_xx = 1/2, Im F = 1/2).
"""
import numpy as np
import pytest

import fd_inputs as fi
from oracle import force as oforce
from oracle import free, stable

from gpu_helpers import F_ATOL_FP64, G_ATOL_FP64, LOGDET_RTOL_FP64, logdet_err, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_02130_gb300 import api

    return api.Context(0)


def _run(ctx, probs, want, prec="fp64", n_stab=None):
    from paper_2604_02130_gb300 import api

    b = api.Batch(ctx, to_dev(probs, n_stab), want, prec)
    r = b.run()
    torch.cuda.synchronize()
    st = b.status()
    assert all(s == 0 for s in st), st
    ld = r.logdet.cpu().numpy()
    G = [g.cpu().numpy() for g in r.G] if r.G is not None else None
    F = [f.cpu().numpy() for f in r.F] if r.F is not None else None
    return ld, G, F


SMALL = [  # L, nt, beta, U, n_stab
    (2, 16, 2.0, 2.0, 4),      # the tiny workload shape
    (2, 16, 2.0, 2.0, 1),      # QR after every slice
    (2, 16, 2.0, 2.0, 16),     # a single block
    (3, 24, 3.0, 3.0, 8),      # Nx = 18
    (4, 16, 2.0, 3.0, 4),      # Nx = 32: one full warp of rows
    (5, 16, 2.0, 3.0, 8),      # Nx = 50: ragged
    (6, 16, 4.0, 3.0, 8),      # Nx = 72
    (7, 8, 1.0, 3.0, 4),       # Nx = 98: buffers spill to global scratch
]


@pytest.mark.parametrize("L,nt,beta,U,n_stab", SMALL)
def test_logdet_green_small(ctx, L, nt, beta, U, n_stab):
    probs = [fi.make_problem(L, nt, beta, U, n_stab, 77, c) for c in range(3)]
    ld, G, _ = _run(ctx, probs, "green")
    for c, p in enumerate(probs):
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, n_stab)
        assert logdet_err(complex(ld[c]), ref_ld) <= LOGDET_RTOL_FP64
        assert np.abs(G[c] - ref_G).max() <= G_ATOL_FP64


@pytest.mark.parametrize("L,nt,beta,U,n_stab", SMALL[:6])
def test_force_small(ctx, L, nt, beta, U, n_stab):
    probs = [fi.make_problem(L, nt, beta, U, n_stab, 78, c) for c in range(2)]
    ld, G, F = _run(ctx, probs, "force+green")
    for c, p in enumerate(probs):
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, n_stab)
        ref_F = oforce.force(p.E, p.phi, n_stab)
        assert logdet_err(complex(ld[c]), ref_ld) <= LOGDET_RTOL_FP64
        assert np.abs(G[c] - ref_G).max() <= G_ATOL_FP64
        assert np.abs(F[c] - ref_F).max() <= F_ATOL_FP64


def test_tiny_workload(ctx):
    probs = fi.workload("tiny8")
    ld, G, F = _run(ctx, probs, "force+green")
    p = probs[0]
    ref_ld, ref_G = stable.logdet_green(p.E, p.phi, p.n_stab)
    assert logdet_err(complex(ld[0]), ref_ld) <= LOGDET_RTOL_FP64
    assert np.abs(G[0] - ref_G).max() <= G_ATOL_FP64
    assert np.abs(F[0] - oforce.force(p.E, p.phi, p.n_stab)).max() <= F_ATOL_FP64


def _inv_tol(M):
    # FP64 element tolerance of G (and of F = i (1 - diag G_t)): G = (1 + P)^{-1} moves by
    # -G dP G under a relative perturbation dP of the product, so element errors scale with
    # max|G|^2 (single beta = 64 configurations reach max|G| ~ 300)
    return max(1e-10, 1e-12 * max(1.0, float(np.abs(M).max())) ** 2)


def _invariants(probs, ld, G=None, F=None):
    for c, p in enumerate(probs):
        r = (ld[c].imag - 0.5 * p.phi.sum()) / np.pi
        assert abs(r - round(r)) < 1e-8
        if G is not None:
            assert np.abs(np.diag(G[c]).real - 0.5).max() < _inv_tol(G[c])
        if F is not None:
            assert np.abs(F[c].imag - 0.5).max() < _inv_tol(F[c])


def test_batch18_full(ctx):
    probs = fi.workload("batch18")
    ld, G, F = _run(ctx, probs, "force+green")
    _invariants(probs, ld, G, F)
    for c, p in enumerate(probs):
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, p.n_stab)
        assert logdet_err(complex(ld[c]), ref_ld) <= LOGDET_RTOL_FP64
        assert np.abs(G[c] - ref_G).max() <= G_ATOL_FP64
    for c in (0, 101, 255):
        p = probs[c]
        rows = [0, 7, 8, 31, 63]
        ref = oforce.force_rows(p.E, p.phi, p.n_stab, rows)
        for r in rows:
            assert np.abs(F[c][r] - ref[r]).max() <= F_ATOL_FP64


def test_cold72_sampled(ctx):
    probs = fi.workload("cold72")
    ld, G, _ = _run(ctx, probs, "green")
    _invariants(probs, ld, G)
    for c in (0, 37, 63):
        p = probs[c]
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, p.n_stab)
        assert logdet_err(complex(ld[c]), ref_ld) <= LOGDET_RTOL_FP64
        assert np.abs(G[c] - ref_G).max() <= G_ATOL_FP64


def test_free_field_beta64(ctx):
    probs = [fi.make_problem(6, 512, 64.0, 3.5, 16, 0, 0, zero_field=True),
             fi.make_problem(2, 512, 64.0, 3.5, 8, 0, 0, zero_field=True)]
    ld, G, _ = _run(ctx, probs, "green")
    for c, p in enumerate(probs):
        ref_ld, ref_G = free.logdet_green(p.A, 64.0)
        assert logdet_err(complex(ld[c]), ref_ld) <= LOGDET_RTOL_FP64
        assert np.abs(G[c] - ref_G).max() <= G_ATOL_FP64


def test_force72_fd_sampled(ctx):
    probs = fi.workload("force72", batch=4)
    ld, _, F = _run(ctx, probs, "force")
    _invariants(probs, ld, None, F)
    rng = np.random.default_rng(1003)
    p = probs[0]
    entries = [(int(rng.integers(p.nt)), int(rng.integers(p.nx))) for _ in range(16)]
    fd = oforce.finite_difference(p.E, p.phi, p.n_stab, entries[:4], h=1e-6)
    got = np.array([F[0][r, x] for r, x in entries[:4]])
    assert np.abs(got - fd).max() <= 2e-6
    rows = sorted({r for r, _ in entries[:6]})
    ref = oforce.force_rows(p.E, p.phi, p.n_stab, rows)
    for r in rows:
        assert np.abs(F[0][r] - ref[r]).max() <= F_ATOL_FP64


def test_uneven_mix(ctx):
    # several sizes in one call (one launch per size class), ragged nt, different n_stab
    probs = []
    for c, (L, nt, ns) in enumerate([(2, 32, 16), (3, 64, 16), (4, 32, 8), (2, 128, 16),
                                     (5, 32, 16), (3, 32, 32), (6, 32, 16), (2, 16, 2)]):
        probs.append(fi.make_problem(L, nt, nt / 16.0, 3.0, ns, 1004, c))
    ld, G, F = _run(ctx, probs, "force+green")
    for c, p in enumerate(probs):
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, p.n_stab)
        assert logdet_err(complex(ld[c]), ref_ld) <= LOGDET_RTOL_FP64
        assert np.abs(G[c] - ref_G).max() <= G_ATOL_FP64
        rows = [0, p.nt // 2, p.nt - 1]
        ref = oforce.force_rows(p.E, p.phi, p.n_stab, rows)
        for r in rows:
            assert np.abs(F[c][r] - ref[r]).max() <= F_ATOL_FP64


def test_degenerate_sizes(ctx):
    # nx = 1 (a 1x1 "lattice") and nx = 2 with generic symmetric E; nt = n_stab = 1
    rng = np.random.default_rng(5)
    probs = []
    for nx, nt, ns in [(1, 1, 1), (1, 7, 7), (2, 3, 1), (2, 4, 2)]:
        A = rng.normal(size=(nx, nx))
        A = 0.5 * (A + A.T)
        E = fi.hopping_exp(A, 0.3)
        Einv = fi.hopping_exp(A, 0.3, sign=-1.0)
        phi = rng.normal(size=(nt, nx))
        probs.append(fi.Problem(L=0, nt=nt, n_stab=ns, beta=0.3 * nt, U=1.0, kappa=1.0, E=E,
                                Einv=Einv, phi=phi, A=A))
    from paper_2604_02130_gb300 import api

    dev = torch.device("cuda", 0)
    tens = [(torch.from_numpy(p.E).to(dev), torch.from_numpy(p.Einv).to(dev),
             torch.from_numpy(p.phi).to(dev), p.n_stab) for p in probs]
    r = api.Batch(ctx, tens, "force+green").run()
    torch.cuda.synchronize()
    for c, p in enumerate(probs):
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, p.n_stab)
        assert logdet_err(complex(r.logdet[c].item()), ref_ld) <= LOGDET_RTOL_FP64
        assert np.abs(r.G[c].cpu().numpy() - ref_G).max() <= G_ATOL_FP64
        ref_F = oforce.force(p.E, p.phi, p.n_stab)
        assert np.abs(r.F[c].cpu().numpy() - ref_F).max() <= F_ATOL_FP64


def test_host_validation(ctx):
    from paper_2604_02130_gb300 import _lib as L
    from paper_2604_02130_gb300 import api

    p = fi.make_problem(2, 16, 2.0, 2.0, 4, 1, 0)
    good = to_dev([p])
    with pytest.raises(api.FdError) as e:  # nt % n_stab != 0
        api.Batch(ctx, [(good[0][0], good[0][1], good[0][2], 5)], "logdet").run()
    assert e.value.code == L.FD_ERR_INVALID
    with pytest.raises(api.FdError) as e:  # force without E^{-1}
        api.Batch(ctx, [(good[0][0], None, good[0][2], 4)], "force").run()
    assert e.value.code == L.FD_ERR_INVALID
    # empty batch is a no-op
    r = api.Batch(ctx, [], "logdet").run()
    assert r.logdet.numel() == 0


# ------------------------------------------------------------------ mixed precision
from gpu_helpers import MIXED_TOL, g_scaled_err  # noqa: E402

MIXED_CASES = [  # L, nt, beta, U, n_stab
    (2, 16, 2.0, 2.0, 4),
    (3, 64, 8.0, 3.0, 8),
    (4, 32, 4.0, 3.0, 8),
    (5, 32, 4.0, 3.0, 16),
    (6, 64, 8.0, 3.0, 16),
]


@pytest.mark.parametrize("prec", ["3xtf32", "tf32"])
@pytest.mark.parametrize("L,nt,beta,U,n_stab", MIXED_CASES)
def test_mixed_logdet_green(ctx, prec, L, nt, beta, U, n_stab):
    probs = [fi.make_problem(L, nt, beta, U, n_stab, 55, c) for c in range(3)]
    ld, G, _ = _run(ctx, probs, "green", prec)
    tol = MIXED_TOL[prec]
    for c, p in enumerate(probs):
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, n_stab)
        assert logdet_err(complex(ld[c]), ref_ld) * max(1.0, abs(ref_ld)) / abs(ref_ld) \
            <= tol["logdet_rel"]
        assert g_scaled_err(G[c], ref_G) <= tol["G_scaled"]


@pytest.mark.parametrize("prec", ["3xtf32", "tf32"])
def test_mixed_cold72_sampled(ctx, prec):
    probs = fi.workload("cold72", batch=8)
    ld, G, _ = _run(ctx, probs, "green", prec)
    tol = MIXED_TOL[prec]
    for c in (0, 5):
        p = probs[c]
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, p.n_stab)
        assert logdet_err(complex(ld[c]), ref_ld) * max(1.0, abs(ref_ld)) / abs(ref_ld) \
            <= tol["logdet_rel"]
        assert g_scaled_err(G[c], ref_G) <= tol["G_scaled"]


def test_mixed_oversize_class_runs_streamed(ctx):
    # Nx = 288 exceeds the shared-memory tensor tile: that size class runs on the streamed
    # tensor-core kernel (operands in global memory), the Nx = 18 class of the same call on the
    # shared-memory one
    from paper_2604_02130_gb300 import api

    probs = [fi.make_problem(12, 16, 1.0, 3.0, 16, 1, 0), fi.make_problem(3, 16, 1.0, 3.0, 8, 1, 1)]
    b = api.Batch(ctx, to_dev(probs), "green", "3xtf32")
    first = {}
    for g in b.plan():  # the first launch of a class does the slice products
        first.setdefault(g["nx"], g["kernel"])
    # kernel codes: 0 log det/G, 1 chains (time-parallel segments), +4 on the tensor cores,
    # +16 streamed
    assert first[288] in (20, 21) and first[18] in (4, 5)
    ld, G, _ = _run(ctx, probs, "green", "3xtf32")
    tol = MIXED_TOL["3xtf32"]
    for c, p in enumerate(probs):
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, p.n_stab)
        assert logdet_err(complex(ld[c]), ref_ld) <= tol["logdet_rel"]
        assert g_scaled_err(G[c], ref_G) <= tol["G_scaled"]


@pytest.mark.parametrize("prec", ["3xtf32", "tf32"])
@pytest.mark.parametrize("L,nt,beta,U,n_stab", [(2, 16, 2.0, 2.0, 4), (3, 64, 8.0, 3.0, 8),
                                                (4, 32, 4.0, 3.0, 8), (6, 32, 4.0, 3.0, 8)])
def test_mixed_force(ctx, prec, L, nt, beta, U, n_stab):
    probs = [fi.make_problem(L, nt, beta, U, n_stab, 56, c) for c in range(2)]
    ld, G, F = _run(ctx, probs, "force+green", prec)
    tol = MIXED_TOL[prec]
    for c, p in enumerate(probs):
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, n_stab)
        assert logdet_err(complex(ld[c]), ref_ld) * max(1.0, abs(ref_ld)) / abs(ref_ld) \
            <= tol["logdet_rel"]
        assert g_scaled_err(G[c], ref_G) <= tol["G_scaled"]
        ref_F = oforce.force(p.E, p.phi, n_stab)
        scale = max(1.0, float(np.abs(ref_F).max())) ** 2
        assert float(np.abs(F[c] - ref_F).max()) / scale <= tol["F_scaled"]


# ------------------------------------------------------------------ graphs and uneven batches
def _uneven_small(seed=1004):
    # every honeycomb size of the uneven workload (Nx = 8 ... 288), short Nt, delta = 1/16
    probs = []
    shapes = [(2, 64), (3, 32), (4, 64), (5, 32), (6, 32), (7, 16), (8, 16), (12, 16),
              (2, 128), (3, 64), (4, 32), (6, 64)]
    for c, (L, nt) in enumerate(shapes):
        probs.append(fi.make_problem(L, nt, nt / 16.0, 3.0, min(16, nt), seed, c))
    return probs


@pytest.mark.parametrize("prec", ["fp64", "3xtf32"])
def test_uneven_graph_replay(ctx, prec):
    """An uneven batch captured into one CUDA graph; two replays with a field update between."""
    from paper_2604_02130_gb300 import api

    probs = _uneven_small()
    tens = to_dev(probs)
    b = api.Batch(ctx, tens, "force+green", prec)
    g = b.graph()
    for rep in range(2):
        if rep == 1:  # update the fields in place and replay
            for p, t in zip(probs, tens):
                p.phi = p.phi[::-1].copy()
                t[2].copy_(torch.from_numpy(p.phi))
        g.launch()
        torch.cuda.synchronize()
        assert all(s == 0 for s in g.status())
        for c, p in enumerate(probs):
            ref_ld, ref_G = stable.logdet_green(p.E, p.phi, p.n_stab)
            got = complex(b.logdet_buf[c, 0].item(), b.logdet_buf[c, 1].item())
            Gc = b.G[c].cpu().numpy()
            if prec == "fp64":
                assert logdet_err(got, ref_ld) <= LOGDET_RTOL_FP64
                assert np.abs(Gc - ref_G).max() <= G_ATOL_FP64
            else:
                tol = MIXED_TOL[prec]
                assert logdet_err(got, ref_ld) * max(1.0, abs(ref_ld)) / abs(ref_ld) \
                    <= tol["logdet_rel"]
                assert g_scaled_err(Gc, ref_G) <= tol["G_scaled"]
            rows = [0, p.nt - 1]
            ref = oforce.force_rows(p.E, p.phi, p.n_stab, rows)
            Fc = b.F[c].cpu().numpy()
            for r in rows:
                if prec == "fp64":
                    assert np.abs(Fc[r] - ref[r]).max() <= F_ATOL_FP64
                else:
                    scale = max(1.0, float(np.abs(ref[r]).max())) ** 2
                    assert float(np.abs(Fc[r] - ref[r]).max()) / scale <= MIXED_TOL[prec]["F_scaled"]
    g.close()


def test_graph_matches_direct_call(ctx):
    from paper_2604_02130_gb300 import api

    probs = fi.workload("batch18", batch=40)
    tens = to_dev(probs)
    direct = api.Batch(ctx, tens, "force", "3xtf32").run()
    torch.cuda.synchronize()
    ld0 = direct.logdet.clone()
    F0 = [f.clone() for f in direct.F]
    b = api.Batch(ctx, tens, "force", "3xtf32")
    g = b.graph()
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(b.logdet_buf.view(-1, 2), torch.view_as_real(ld0))
    assert all(torch.equal(a, c) for a, c in zip(b.F, F0))
    g.close()
