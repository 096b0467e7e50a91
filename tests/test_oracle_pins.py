"""Pins that tie the CPU oracle to things other than itself.

* brute force on the full (Nt*Nx)^2 fermion matrix (Section 2): log det and every diagonal block
  of M^{-1} (G and all equal-time G_tau, hence the force);
* the free-field closed form at phi = 0, any beta up to 64;
* 250-digit mpmath evaluation of the plain product at beta = 64 (stored golden values, made by
  tests/golden/make_golden.py from oracle.highprec);
* exact invariants: cyclic slice shift, product-order reversal, and the particle-hole identities
  of the bipartite honeycomb lattice, Im log det = (1/2) sum phi (mod pi) and Re [G_tau]_xx = 1/2;
* the naive algorithm of Section 6 and the literal assembly of Section 7 at small beta;
* central finite differences (h = 1e-6) for the force.
"""
import json
import os

import numpy as np
import pytest

import fd_inputs as fi
from oracle import fermion_matrix, force, free, naive, plain, stable

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dlog(a, b):
    """|a - b| for complex logs, imaginary part compared mod 2 pi."""
    return abs(a.real - b.real) + abs(np.angle(np.exp(1j * (a.imag - b.imag))))


def _rand_problem(L, nt, beta, U, n_stab, c=0, seed=7):
    return fi.make_problem(L, nt, beta, U, n_stab, seed, c)


SMALL = [
    # L, nt, beta, U, n_stab
    (2, 16, 2.0, 2.0, 4),
    (2, 16, 2.0, 2.0, 1),
    (2, 12, 4.0, 3.0, 5),    # last block shorter than n_stab
    (3, 8, 1.0, 3.0, 8),
    (2, 24, 6.0, 4.0, 3),
]


@pytest.mark.parametrize("L,nt,beta,U,n_stab", SMALL)
def test_stable_matches_brute_force(L, nt, beta, U, n_stab):
    p = _rand_problem(L, nt, beta, U, n_stab)
    ld, G = stable.logdet_green(p.E, p.phi, n_stab)
    ld_bf = fermion_matrix.logdet(p.E, p.phi)
    Gb = fermion_matrix.green_blocks(p.E, p.phi)
    assert _dlog(ld, ld_bf) < 1e-11 * max(1, abs(ld_bf))
    assert np.abs(G - Gb[0]).max() < 1e-12


@pytest.mark.parametrize("L,nt,beta,U,n_stab", SMALL[:3])
def test_plain_definition_matches_brute_force(L, nt, beta, U, n_stab):
    p = _rand_problem(L, nt, beta, U, n_stab)
    ld, G = plain.logdet_green(p.E, p.phi)
    assert _dlog(ld, fermion_matrix.logdet(p.E, p.phi)) < 1e-11
    assert np.abs(G - fermion_matrix.green_blocks(p.E, p.phi)[0]).max() < 1e-12


@pytest.mark.parametrize("L,nt,beta,n_stab", [(2, 512, 64.0, 16), (6, 512, 64.0, 16),
                                              (3, 64, 8.0, 8), (4, 256, 32.0, 8)])
def test_free_field_closed_form(L, nt, beta, n_stab):
    p = fi.make_problem(L, nt, beta, 3.0, n_stab, 0, 0, zero_field=True)
    ld, G = stable.logdet_green(p.E, p.phi, n_stab)
    ld_cf, G_cf = free.logdet_green(p.A, beta)
    # the closed form from the momentum-space bands, independent of any eigen-solver
    ld_k = free.logdet_from_spectrum(fi.honeycomb_spectrum(L), beta)
    assert abs(ld_cf.real - ld_k) < 1e-10 * ld_k
    assert _dlog(ld, ld_cf) < 1e-12 * abs(ld_cf)
    assert np.abs(G - G_cf).max() < 1e-12


def test_highprec_golden_beta64():
    with open(os.path.join(GOLDEN, "highprec_beta64.json")) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        p = fi.make_problem(case["L"], case["nt"], case["beta"], case["U"], case["n_stab"],
                            case["seed"], case["c"])
        ld, G = stable.logdet_green(p.E, p.phi, case["n_stab"])
        ld_ref = complex(*case["logdet"])
        G_ref = np.array(case["G_re"]) + 1j * np.array(case["G_im"])
        assert _dlog(ld, ld_ref) < 1e-12 * abs(ld_ref)
        assert np.abs(G - G_ref).max() < 1e-10


@pytest.mark.slow
def test_highprec_live():
    pytest.importorskip("mpmath")
    from oracle import highprec

    p = _rand_problem(2, 96, 24.0, 3.0, 8)
    ld_mp, G_mp = highprec.logdet_green(p.E, p.phi, dps=120)
    ld, G = stable.logdet_green(p.E, p.phi, 8)
    assert _dlog(ld, ld_mp) < 1e-12 * abs(ld_mp)
    assert np.abs(G - G_mp).max() < 1e-11


@pytest.mark.parametrize("L,nt,beta,n_stab", [(2, 64, 8.0, 8), (3, 128, 16.0, 8),
                                              (2, 512, 64.0, 16)])
def test_cyclic_shift_and_reversal(L, nt, beta, n_stab):
    p = _rand_problem(L, nt, beta, 3.0, n_stab)
    ld, G = stable.logdet_green(p.E, p.phi, n_stab)
    for s in (1, 5, nt // 2):
        ld_s, G_s = stable.logdet_green(p.E, np.roll(p.phi, -s, axis=0), n_stab)
        assert _dlog(ld, ld_s) < 1e-11 * abs(ld)
    # rolled by one slice: G' = B_1 G B_1^{-1}
    ld_1, G_1 = stable.logdet_green(p.E, np.roll(p.phi, -1, axis=0), n_stab)
    B1 = plain.slice_matrix(p.E, p.phi[0])
    B1inv = np.exp(-1j * p.phi[0])[:, None] * p.Einv
    assert np.abs(G_1 - B1 @ G @ B1inv).max() < 1e-9
    # order reversal (A real symmetric, D diagonal): log det unchanged
    ld_r, _ = stable.logdet_green(p.E, p.phi[::-1].copy(), n_stab)
    assert _dlog(ld, ld_r) < 1e-11 * abs(ld)


@pytest.mark.parametrize("L,nt,beta,n_stab", [(2, 16, 2.0, 4), (3, 64, 8.0, 8),
                                              (6, 512, 64.0, 16)])
def test_particle_hole_invariants(L, nt, beta, n_stab):
    p = _rand_problem(L, nt, beta, 3.5, n_stab)
    ld, G = stable.logdet_green(p.E, p.phi, n_stab)
    half = 0.5 * p.phi.sum()
    r = (ld.imag - half) / np.pi
    assert abs(r - round(r)) < 1e-10
    assert np.abs(np.diag(G).real - 0.5).max() < 1e-10
    S = np.diag([(-1.0) ** (i % 2) for i in range(p.nx)])
    assert np.abs(S @ G @ S - (np.eye(p.nx) - G.conj().T)).max() < 1e-10


@pytest.mark.parametrize("L,nt,beta,U", [(2, 16, 2.0, 2.0), (2, 24, 4.0, 3.0),
                                         (3, 16, 3.0, 3.0)])
def test_naive_section6_matches(L, nt, beta, U):
    p = _rand_problem(L, nt, beta, U, 4)
    ld, G = stable.logdet_green(p.E, p.phi, 4)
    ld_n, G_n = naive.logdet_green(p.E, p.phi)
    assert _dlog(ld, ld_n) < 1e-10
    assert np.abs(G - G_n).max() < 1e-10


@pytest.mark.parametrize("beta", [1.0, 4.0, 8.0])
def test_literal_assembly_matches_scale_separated(beta):
    p = _rand_problem(2, 32, beta, 3.0, 8)
    X, D, T = stable.udt_product(p.E, p.phi, 8)
    ld, G = stable.assemble(X, D, T)
    ld_l, G_l = stable.assemble_literal(X, D, T)
    assert _dlog(ld, ld_l) < 1e-10
    assert np.abs(G - G_l).max() < 1e-9


@pytest.mark.parametrize("L,nt,beta,U,n_stab", [(2, 16, 2.0, 2.0, 4), (2, 12, 3.0, 3.0, 4),
                                                (3, 8, 1.0, 3.0, 2)])
def test_force_matches_brute_force_blocks(L, nt, beta, U, n_stab):
    p = _rand_problem(L, nt, beta, U, n_stab)
    F = force.force(p.E, p.phi, n_stab)
    Gb = fermion_matrix.green_blocks(p.E, p.phi)
    F_bf = np.stack([1j * (1 - np.diag(Gb[t - 1])) for t in range(1, nt + 1)])
    assert np.abs(F - F_bf).max() < 1e-11
    assert np.abs(F.imag - 0.5).max() < 1e-11


@pytest.mark.parametrize("L,nt,beta,U,n_stab", [(2, 16, 2.0, 2.0, 4), (3, 64, 8.0, 3.0, 8),
                                                (2, 256, 32.0, 3.0, 8)])
def test_force_matches_finite_differences(L, nt, beta, U, n_stab):
    p = _rand_problem(L, nt, beta, U, n_stab)
    rng = np.random.default_rng(1003)
    entries = [(int(rng.integers(nt)), int(rng.integers(p.nx))) for _ in range(6)]
    rows = force.force_rows(p.E, p.phi, n_stab, {r for r, _ in entries})
    F = np.array([rows[r][x] for r, x in entries])
    Ffd = force.finite_difference(p.E, p.phi, n_stab, entries, h=1e-6)
    assert np.abs(F - Ffd).max() < 2e-6 * max(1.0, np.abs(F).max())


@pytest.mark.parametrize("name,nseg", [("cold72", 4), ("cold72", 8), ("force72", 2)])
def test_segmented_product_matches_chain(name, nseg):
    """The time-parallel order (segments from the identity, merged by the stabilised product of
    two UDV factors) gives the log det and G of the sequential chain at beta = 64 and 32."""
    p = fi.workload(name, batch=1)[0]
    ref_ld, ref_G = stable.logdet_green(p.E, p.phi, p.n_stab)
    ld, G = stable.assemble(*stable.segmented_product(p.E, p.phi, p.n_stab, nseg))
    assert abs(ld.real - ref_ld.real) <= 1e-12 * abs(ref_ld)
    assert abs(np.angle(np.exp(1j * (ld.imag - ref_ld.imag)))) <= 1e-12 * abs(ref_ld)
    assert np.abs(G - ref_G).max() <= 1e-10 * max(1.0, float(np.abs(ref_G).max())) ** 2
