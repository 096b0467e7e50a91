"""Pins for the product form of the slice exponential (oracle.product_form, Section 8).

Independent references: the closed forms of the factors for n = 1, 2; multiplying the linear
factors out (polynomial convolution) must give the Taylor coefficients 1/j!; the dense product
of the factors equals the power sum T_n(K); T_n converges to scipy's expm with order n+1 in
delta; the stabilised log det with T_n equals the brute-force determinant of the full fermion
matrix built with the same slice matrix, and converges to the exact-exponential log det with
order n in delta at fixed beta.  Planted mistakes (gamma_k = +1/x_k, one factor dropped) are
rejected by the expansion pin.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import fd_inputs as fi
from oracle import fermion_matrix, product_form, stable


def _expand(gammas):
    """Coefficients (lowest power first) of prod_k (1 + gamma_k x)."""
    c = np.array([1.0 + 0j])
    for g in gammas:
        c = np.convolve(c, np.array([1.0, g]))
    return c


def test_factors_closed_forms():
    assert np.allclose(product_form.taylor_factors(1), [1.0])
    g2 = product_form.taylor_factors(2)  # 1 + x + x^2/2 has roots -1 +- i
    assert np.allclose(sorted(g2, key=lambda z: z.imag), [0.5 - 0.5j, 0.5 + 0.5j])


@pytest.mark.parametrize("n", range(1, 9))
def test_factors_expand_to_taylor(n):
    c = _expand(product_form.taylor_factors(n))
    want = np.array([1.0 / math.factorial(j) for j in range(n + 1)])
    assert np.abs(c - want).max() < 1e-12
    if n >= 2:  # planted mistakes
        g = product_form.taylor_factors(n)
        assert np.abs(_expand(-g) - want).max() > 1e-3
        assert len(_expand(g[1:])) != len(want)


def test_product_matrix_is_the_power_sum_and_converges_to_expm():
    A = fi.honeycomb_adjacency(3)
    for n in (2, 4):
        g = product_form.taylor_factors(n)
        errs = []
        for delta in (0.2, 0.1):
            K = delta * A
            P = product_form.product_form_matrix(K, g)
            T = product_form.taylor_matrix(K, n)
            assert np.abs(P - T).max() < 1e-13
            assert np.abs(T - T.T).max() < 1e-15  # symmetric, as the library requires of E
            errs.append(np.abs(T - expm(K)).max())
        order = np.log2(errs[0] / errs[1])
        assert abs(order - (n + 1)) < 0.3, order


def test_logdet_against_brute_force_full_matrix():
    p = fi.make_problem(2, 12, 1.5, 2.0, 4, 77, 0)
    E4 = product_form.slice_matrix(p.A, p.delta, p.kappa, 4)
    ld, G = product_form.logdet_green(p.A, p.delta, p.kappa, 4, p.phi, p.n_stab)
    ref = fermion_matrix.logdet(E4, p.phi)
    assert abs(ld.real - ref.real) < 1e-10
    assert abs(np.angle(np.exp(1j * (ld.imag - ref.imag)))) < 1e-10
    assert np.abs(G - fermion_matrix.green_blocks(E4, p.phi)[0]).max() < 1e-10  # block (0, 0)


def test_logdet_converges_with_order_n():
    """At fixed beta the product-form log det differs from the exact one by O(Nt delta^{n+1})
    = O(beta delta^n): halving delta divides the error by ~2^n.  Odd n: for even n the leading
    term of the error in log det cancels on this bipartite lattice (the error then falls faster
    than delta^n), so the order is checked with n = 3."""
    n, beta, L = 3, 2.0, 2
    errs = []
    for nt in (64, 128):
        p = fi.make_problem(L, nt, beta, 0.0, 4, 5, 0, zero_field=True)
        rng = np.random.default_rng(9)
        # a smooth field, the same function of imaginary time on both grids
        tau = (np.arange(nt) + 0.5) / nt
        phi = np.outer(np.sin(2 * np.pi * tau), rng.normal(size=p.nx)) * 0.5
        exact, _ = stable.logdet_green(p.E, phi, 4)
        approx, _ = product_form.logdet_green(p.A, p.delta, p.kappa, n, phi, 4)
        errs.append(abs(approx - exact))
    order = np.log2(errs[0] / errs[1])
    assert abs(order - n) < 0.15, (errs, order)
