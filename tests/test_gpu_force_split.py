"""Time-parallel force chains (fd_set_force_split).  Halves: each chain of a configuration runs
as two halves in parallel, the boundary phase merges a second half's checkpoint with the first
half's last one (Section 7's stabilised product of two factored matrices, FP64) and forms log det
and G_0 from the forward halves.  Segments (the mixed path): segments run from the identity,
their prefixes are formed by merges (double-float in the streamed size classes, FP64 in the
shared-memory ones) and the segments re-run from them.  Compared with the whole chains and with the CPU oracle, every entry, in FP64 (buffers in
shared memory and in global scratch) and in both mixed modes; odd block counts; short streamed
chains stay whole; the automatic rule on the force workloads."""
import numpy as np
import pytest

import fd_inputs as fi
from oracle import force as oforce
from oracle import stable

from gpu_helpers import (F_ATOL_FP64, G_ATOL_FP64, LOGDET_RTOL_FP64, MIXED_TOL, g_scaled_err,
                         logdet_err, mixed_logdet_ok, to_dev)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_02130_gb300 import api

    c = api.Context(0)
    yield c
    c.set_force_split(-1)


def _run(ctx, probs, prec, mode):
    from paper_2604_02130_gb300 import api

    ctx.set_force_split(mode)
    b = api.Batch(ctx, to_dev(probs), "force+green", prec)
    plan = b.plan()
    r = b.run()
    torch.cuda.synchronize()
    st = b.status()
    ctx.set_force_split(-1)
    assert all(s == 0 for s in st), st
    return (plan, r.logdet.cpu().numpy(), [g.cpu().numpy() for g in r.G],
            [f.cpu().numpy() for f in r.F])


def _chain_tasks(plan):
    return sum(g["configs"] for g in plan if g["kernel"] % 4 == 1)


FP64_CASES = [  # L, nt, beta, U, n_stab: nb = nt / n_stab blocks, split at nb // 2
    (2, 64, 4.0, 3.0, 8),     # Nx = 8, nb = 8
    (3, 40, 5.0, 3.0, 8),     # Nx = 18, nb = 5 (odd: halves of 2 and 3 blocks)
    (6, 64, 8.0, 3.0, 16),    # Nx = 72, nb = 4
]


@pytest.mark.parametrize("L,nt,beta,U,n_stab", FP64_CASES)
def test_split_fp64_matches_unsplit_and_oracle(ctx, L, nt, beta, U, n_stab):
    probs = [fi.make_problem(L, nt, beta, U, n_stab, 97, c) for c in range(3)]
    plan1, ld1, G1, F1 = _run(ctx, probs, "fp64", 1)
    plan0, ld0, G0, F0 = _run(ctx, probs, "fp64", 0)
    assert _chain_tasks(plan1) == 4 * len(probs) and _chain_tasks(plan0) == 2 * len(probs)
    for c, p in enumerate(probs):
        # the merge re-factors at rounding level only
        assert logdet_err(complex(ld1[c]), complex(ld0[c])) <= 1e-12
        assert np.abs(G1[c] - G0[c]).max() <= 1e-10 * max(1.0, np.abs(G0[c]).max()) ** 2
        assert np.abs(F1[c] - F0[c]).max() <= 1e-10 * max(1.0, np.abs(G0[c]).max()) ** 2
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, p.n_stab)
        ref_F = oforce.force(p.E, p.phi, p.n_stab)
        assert logdet_err(complex(ld1[c]), ref_ld) <= LOGDET_RTOL_FP64
        assert np.abs(G1[c] - ref_G).max() <= G_ATOL_FP64
        assert np.abs(F1[c] - ref_F).max() <= F_ATOL_FP64


def test_split_mixed_against_oracle(ctx):
    prec = "3xtf32"
    tol = MIXED_TOL[prec]
    probs = [fi.make_problem(6, 64, 8.0, 3.0, 8, 98, c) for c in range(2)]  # Nx = 72
    plan1, ld1, G1, F1 = _run(ctx, probs, prec, 1)
    _, ld0, G0, F0 = _run(ctx, probs, prec, 0)
    assert _chain_tasks(plan1) == 4 * len(probs)
    for c, p in enumerate(probs):
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, p.n_stab)
        ref_F = oforce.force(p.E, p.phi, p.n_stab)
        gmax = float(np.abs(ref_G).max())
        scale = max(1.0, gmax) ** 2
        for ld, G, F in ((ld1[c], G1[c], F1[c]), (ld0[c], G0[c], F0[c])):
            assert mixed_logdet_ok(complex(ld), ref_ld, gmax, prec), (c, ld, ref_ld)
            assert g_scaled_err(G, ref_G) <= tol["G_scaled"], c
            assert float(np.abs(F - ref_F).max()) / scale <= tol["F_scaled"], c
            assert float(np.abs(F.imag - 0.5).max()) <= tol["F_scaled"] * scale


def test_streamed_mixed_class_short_chains_stay_whole(ctx):
    from paper_2604_02130_gb300 import api

    # Nx = 98 in the mixed path runs the streamed kernels (double-float boundary): never split
    # in halves, and 8 blocks are too few for segments of at least 4 blocks (S >= 4)
    probs = [fi.make_problem(7, 64, 8.0, 3.0, 8, 98, c) for c in range(2)]
    ctx.set_force_split(1)
    plan = api.Batch(ctx, to_dev(probs), "force+green", "3xtf32").plan()
    ctx.set_force_split(-1)
    assert _chain_tasks(plan) == 2 * len(probs)


# Nx = 98, nb = 16 blocks, forced segments S = 4 of 4 blocks -- pass 1 (3 + 3 tasks), two prefix
# tasks, pass 2 (3 + 3) per configuration.  Split TF32 runs it on the streamed kernels
# (double-float merges), plain TF32 fits the shared-memory tile (FP64 merges).
@pytest.mark.parametrize("prec,kernels,per", [("3xtf32", [21, 18, 23], 14), ("tf32", [5, 2, 7], 14)])
def test_segmented_streamed_chains(ctx, prec, kernels, per):
    tol = MIXED_TOL[prec]
    probs = [fi.make_problem(7, 128, 8.0, 3.0, 8, 100, c) for c in range(2)]
    plan1, ld1, G1, F1 = _run(ctx, probs, prec, 1)
    _, ld0, G0, F0 = _run(ctx, probs, prec, 0)
    assert [g["kernel"] for g in plan1] == kernels
    assert _chain_tasks(plan1) == per * len(probs)
    for c, p in enumerate(probs):
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, p.n_stab)
        ref_F = oforce.force(p.E, p.phi, p.n_stab)
        gmax = float(np.abs(ref_G).max())
        scale = max(1.0, gmax) ** 2
        for ld, G, F in ((ld1[c], G1[c], F1[c]), (ld0[c], G0[c], F0[c])):
            assert mixed_logdet_ok(complex(ld), ref_ld, gmax, prec), (c, ld, ref_ld)
            assert g_scaled_err(G, ref_G) <= tol["G_scaled"], c
            assert float(np.abs(F - ref_F).max()) / scale <= tol["F_scaled"], c


def test_split_fp64_streamed_class(ctx):
    # Nx = 98 in FP64 runs the FP64 kernels with buffers in global scratch
    probs = [fi.make_problem(7, 32, 2.0, 3.0, 8, 99, c) for c in range(2)]
    _, ld, G, F = _run(ctx, probs, "fp64", 1)
    for c, p in enumerate(probs):
        ref_ld, ref_G = stable.logdet_green(p.E, p.phi, p.n_stab)
        ref_F = oforce.force(p.E, p.phi, p.n_stab)
        assert logdet_err(complex(ld[c]), ref_ld) <= LOGDET_RTOL_FP64
        assert np.abs(G[c] - ref_G).max() <= G_ATOL_FP64
        assert np.abs(F[c] - ref_F).max() <= F_ATOL_FP64


def test_split_rule_on_force_workloads(ctx):
    from paper_2604_02130_gb300 import api

    def tasks(name, prec):
        return _chain_tasks(api.Batch(ctx, to_dev(fi.workload(name)), "force+green", prec).plan())

    # FP64 force72: 32 configurations, 4 * 32 <= 152 SMs -> every chain split
    assert tasks("force72", "fp64") == 4 * 32
    # more configurations: whole chains
    assert tasks("cold72", "fp64") == 2 * 64
    # mixed force72: one chain is 152 / 64 = 2.4 times an SM's share -> segments S = 4 of 8
    # blocks; mixed cold72 (1.2 times) keeps whole chains
    assert tasks("force72", "3xtf32") == 14 * 32
    assert tasks("cold72", "3xtf32") == 2 * 64
    # never
    ctx.set_force_split(0)
    n0 = tasks("force72", "fp64")
    ctx.set_force_split(-1)
    assert n0 == 2 * 32
    # uneven512, mixed: the Nx = 288 chains of Nt = 512 (32 blocks, S = 4) and Nt = 1024 (64
    # blocks, S = 8) are segmented, the shorter ones stay whole
    per = {512: 6 + 2 + 6, 1024: 14 + 2 + 14}
    want = sum(per.get(nt, 2) for L, nt in fi.uneven_sizes(512) if L == 12)
    plan = api.Batch(ctx, to_dev(fi.workload("uneven512")), "force+green", "3xtf32").plan()
    got = [g["configs"] for g in plan if g["nx"] == 288 and g["kernel"] % 4 == 1]
    assert got == [want]
