"""Pins for the single-time observables of Section 4.1 (oracle.observables).

Independent references: the diagonal blocks of the inverse full fermion matrix (brute force),
finite differences of log det in the chemical potential (B_t -> e^{delta mu} B_t) and in the
hopping kappa (E = exp(delta kappa A)), the free-field closed forms, and the cyclic invariance of
tr G_r.  Planted mistakes (transposed operator, slice index off by one, dropped delta, wrong sign)
are each rejected by one of them.
"""
import numpy as np
import pytest

import fd_inputs as fi
from oracle import fermion_matrix, observables, stable
from oracle import force as oforce


def _rand_op(nx, seed):
    return np.random.default_rng(seed).normal(size=(nx, nx))  # not symmetric


@pytest.mark.parametrize("L,nt,beta,U,n_stab", [(2, 16, 2.0, 2.0, 4), (2, 12, 3.0, 3.0, 3)])
def test_traces_match_brute_force(L, nt, beta, U, n_stab):
    p = fi.make_problem(L, nt, beta, U, n_stab, 31, 0)
    O = _rand_op(p.nx, 5)
    Gb = fermion_matrix.green_blocks(p.E, p.phi)
    ref = np.array([np.trace(O @ Gb[r]) for r in range(nt)])
    got = observables.response_traces(p.E, p.phi, n_stab, O)
    assert np.abs(got - ref).max() < 1e-11


def _deriv5(f, x, h):
    """Five-point central difference of a complex log det (imaginary parts on the principal
    branch relative to f(x))."""
    f0 = f(x)
    vals = []
    for k in (-2, -1, 1, 2):
        v = f(x + k * h)
        vals.append((v.real - f0.real) + 1j * np.angle(np.exp(1j * (v.imag - f0.imag))))
    return (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)


def _logdet_scaled_E(p, s):
    return stable.logdet_green(p.E * s, p.phi, p.n_stab)[0]


def test_fermion_number_is_mu_derivative():
    # B_t(mu) = e^{delta mu} B_t: d log det / d mu at mu = 0 equals beta V n
    p = fi.make_problem(3, 32, 4.0, 3.0, 8, 32, 0)
    d = _deriv5(lambda mu: _logdet_scaled_E(p, np.exp(p.delta * mu)), 0.0, 3e-5)
    n = observables.fermion_number(p.E, p.phi, p.n_stab)
    assert abs(d / (p.beta * p.nx) - n) < 1e-9


def test_hopping_response_is_kappa_derivative():
    p = fi.make_problem(3, 32, 4.0, 3.0, 8, 33, 0)

    def ld(kappa):
        return stable.logdet_green(fi.hopping_exp(p.A, p.delta, kappa), p.phi, p.n_stab)[0]

    d = _deriv5(ld, 1.0, 1e-4)
    got = observables.hopping_response(p.E, p.phi, p.n_stab, p.A, p.delta)
    assert abs(got - d) < 1e-9 * max(1.0, abs(d))


def test_free_field_closed_forms():
    # phi = 0: n = 1 - (1/V) sum_k 1/(1 + e^{beta lam_k}),
    #          d log det / d kappa = sum_k beta lam_k / (1 + e^{-beta lam_k})
    L, nt, beta = 3, 64, 8.0
    p = fi.make_problem(L, nt, beta, 3.0, 8, 0, 0, zero_field=True)
    lam = fi.honeycomb_spectrum(L)
    x = beta * lam
    fermi = 0.5 * (1.0 - np.tanh(0.5 * x))
    n_ref = 1.0 - fermi.sum() / p.nx
    assert abs(observables.fermion_number(p.E, p.phi, 8) - n_ref) < 1e-13
    k_ref = np.sum(beta * lam * (1.0 - fermi))
    got = observables.hopping_response(p.E, p.phi, 8, p.A, p.delta)
    assert abs(got - k_ref) < 1e-10 * max(1.0, abs(k_ref))


def test_trace_of_green_is_slice_independent():
    # G_r is similar to G (cyclic rotation of the product), so tr G_r = tr G for every r
    p = fi.make_problem(3, 32, 4.0, 3.0, 8, 34, 0)
    R = observables.response_traces(p.E, p.phi, 8, np.eye(p.nx))
    assert np.abs(R - R[0]).max() < 1e-11
    assert abs(1.0 - R[0] / p.nx - observables.fermion_number(p.E, p.phi, 8)) < 1e-13


def test_diagonal_operator_matches_force():
    p = fi.make_problem(2, 16, 2.0, 2.0, 4, 35, 0)
    w = np.random.default_rng(6).normal(size=p.nx)
    R = observables.response_traces(p.E, p.phi, 4, np.diag(w))
    F = oforce.force(p.E, p.phi, 4)
    # F[r] = i (1 - diag G_r)  =>  diag G_r = 1 + i F[r]
    assert np.abs(R - (1.0 + 1j * F) @ w).max() < 1e-12


# ------------------------------------------------------------------ planted mistakes
def _traces_transposed(E, phi, n_stab, O):
    return np.array([np.trace(O.T @ oforce.green_at(E, phi, n_stab, r))
                     for r in range(phi.shape[0])])


def _traces_shifted(E, phi, n_stab, O):
    nt = phi.shape[0]
    return np.array([np.trace(O @ oforce.green_at(E, phi, n_stab, (r + 1) % nt))
                     for r in range(nt)])


@pytest.mark.parametrize("mutant", [_traces_transposed, _traces_shifted])
def test_trace_mutants_are_caught(mutant):
    p = fi.make_problem(2, 16, 2.0, 2.0, 4, 31, 0)
    O = _rand_op(p.nx, 5)
    Gb = fermion_matrix.green_blocks(p.E, p.phi)
    ref = np.array([np.trace(O @ Gb[r]) for r in range(p.nt)])
    assert np.abs(mutant(p.E, p.phi, 4, O) - ref).max() > 1e-3


@pytest.mark.parametrize("scale", [1.0, -1.0])  # delta dropped (delta = 1/8 here) / sign flipped
def test_hopping_mutants_are_caught(scale):
    p = fi.make_problem(3, 32, 4.0, 3.0, 8, 33, 0)

    def ld(kappa):
        return stable.logdet_green(fi.hopping_exp(p.A, p.delta, kappa), p.phi, p.n_stab)[0]

    d = _deriv5(ld, 1.0, 1e-4)
    R = observables.response_traces(p.E, p.phi, p.n_stab, p.A)
    mutant = scale * (-R.sum())  # no delta factor (scale 1) or the sign of delta flipped
    if scale < 0:
        mutant = -p.delta * (-R.sum())
    assert abs(mutant - d) > 1e-2 * max(1.0, abs(d))
