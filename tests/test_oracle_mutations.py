"""Plant plausible mistakes in copies of the oracle's steps and check that the pins catch them.

Each mutant below is a wrong variant of one oracle step (a dropped term, a wrong order, a wrong
sign or index, a missing permutation).  The test asserts that at least one independent pin
(brute force, free field, particle-hole invariant, finite differences) rejects it, so the pins
are strong enough to hold the real oracle to the paper.
"""
import numpy as np
import pytest
import scipy.linalg

import fd_inputs as fi
from oracle import fermion_matrix, free, plain, stable


def _mut_udt(E, phi, n_stab, *, order="fwd", perm=True, phase=+1, scale_t=True):
    nt, nx = phi.shape
    X = np.eye(nx, dtype=complex)
    D = np.ones(nx)
    T = np.eye(nx, dtype=complex)
    rng = range(nt) if order == "fwd" else range(nt - 1, -1, -1)
    rows = list(rng)
    for b in range(0, nt, n_stab):
        for s in rows[b:b + n_stab]:
            X = (E * np.exp(phase * 1j * phi[s])[None, :]) @ X
        Z = X * D[None, :]
        Q, R, p = scipy.linalg.qr(Z, pivoting=True)
        d = np.abs(np.diag(R))
        Tp = T[p, :] if perm else T
        X, D, T = Q, d, ((R / d[:, None]) if scale_t else R) @ Tp
    return X, D, T


def _assemble_drop_ds(X, D, T):
    Db = np.maximum(D, 1.0)
    XH = X.conj().T
    C = XH / Db[:, None] + T          # D_s dropped
    sx, lx = np.linalg.slogdet(X)
    sc, lc = np.linalg.slogdet(C)
    ld = lx + lc + np.sum(np.log(Db)) + 1j * (np.angle(sx) + np.angle(sc))
    return ld, np.linalg.solve(C, XH / Db[:, None])


def _assemble_no_detx(X, D, T):
    Db = np.maximum(D, 1.0)
    Ds = np.minimum(D, 1.0)
    XH = X.conj().T
    C = XH / Db[:, None] + Ds[:, None] * T
    sc, lc = np.linalg.slogdet(C)
    ld = lc + np.sum(np.log(Db)) + 1j * np.angle(sc)   # log det X forgotten
    return ld, np.linalg.solve(C, XH / Db[:, None])


def _pins_fail(ld, G, p):
    """True if any independent pin rejects (ld, G) for problem p."""
    ld_bf = fermion_matrix.logdet(p.E, p.phi)
    G_bf = fermion_matrix.green_blocks(p.E, p.phi)[0]
    bad_bf = (abs(ld.real - ld_bf.real) > 1e-8
              or abs(np.angle(np.exp(1j * (ld.imag - ld_bf.imag)))) > 1e-8
              or np.abs(G - G_bf).max() > 1e-8)
    half = 0.5 * p.phi.sum()
    r = (ld.imag - half) / np.pi
    bad_ph = abs(r - round(r)) > 1e-8 or np.abs(np.diag(G).real - 0.5).max() > 1e-8
    return bad_bf or bad_ph


@pytest.fixture(scope="module")
def prob():
    return fi.make_problem(2, 16, 4.0, 3.0, 4, 11, 0)


def test_real_oracle_passes(prob):
    ld, G = stable.logdet_green(prob.E, prob.phi, 4)
    assert not _pins_fail(ld, G, prob)


@pytest.mark.parametrize("kw", [dict(order="rev"), dict(perm=False), dict(phase=-1),
                                dict(scale_t=False)])
def test_product_mutants_are_caught(prob, kw):
    ld, G = stable.assemble(*_mut_udt(prob.E, prob.phi, 4, **kw))
    assert _pins_fail(ld, G, prob), kw


@pytest.mark.parametrize("fn", [_assemble_drop_ds, _assemble_no_detx])
def test_assembly_mutants_are_caught(prob, fn):
    ld, G = fn(*stable.udt_product(prob.E, prob.phi, 4))
    assert _pins_fail(ld, G, prob)


def test_transposed_green_is_caught(prob):
    ld, G = stable.logdet_green(prob.E, prob.phi, 4)
    assert _pins_fail(ld, G.T, prob)


def test_force_index_mutant_is_caught(prob):
    # using G_t instead of G_{t-1} for slice t
    from oracle import force

    nt = prob.phi.shape[0]
    F_wrong = np.stack([1j * (1 - np.diag(force.green_at(prob.E, prob.phi, 4, t % nt)))
                        for t in range(1, nt + 1)])
    entries = [(3, 1), (9, 5)]
    Ffd = force.finite_difference(prob.E, prob.phi, 4, entries)
    assert np.abs(np.array([F_wrong[r, x] for r, x in entries]) - Ffd).max() > 1e-4


def test_free_field_catches_wrong_exponent_sign():
    p = fi.make_problem(3, 64, 8.0, 3.0, 8, 0, 0, zero_field=True)
    ld_cf, _ = free.logdet_green(p.A, 8.0)
    ld, _ = stable.logdet_green(p.Einv, p.phi, 8)   # e^{-delta kappa A}: bipartite => same det!
    # the spectrum is symmetric, so log det alone cannot see the sign; G can.
    _, G = stable.logdet_green(p.Einv, p.phi, 8)
    _, G_cf = free.logdet_green(p.A, 8.0)
    assert np.abs(G - G_cf).max() > 1e-3
    assert abs(ld - ld_cf) < 1e-9


def test_plain_vs_brute_force_orders(prob):
    # the product in the other order gives the same log det but a different G
    P_rev = np.eye(prob.nx, dtype=complex)
    for t in range(prob.nt - 1, -1, -1):
        P_rev = plain.slice_matrix(prob.E, prob.phi[t]) @ P_rev
    G_rev = np.linalg.inv(np.eye(prob.nx) + P_rev)
    G_bf = fermion_matrix.green_blocks(prob.E, prob.phi)[0]
    assert np.abs(G_rev - G_bf).max() > 1e-3
