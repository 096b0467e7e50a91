"""Pins for the synthetic input generator (lattice, hopping exponential, fields)."""
import numpy as np
import pytest
import scipy.linalg

import fd_inputs as fi


@pytest.mark.parametrize("L", [2, 3, 4, 6, 12])
def test_honeycomb_structure(L):
    A = fi.honeycomb_adjacency(L)
    nx = 2 * L * L
    assert A.shape == (nx, nx)
    assert np.array_equal(A, A.T)
    assert np.all(A.sum(axis=1) == 3)          # coordination number 3
    assert np.trace(A) == 0
    S = np.diag([(-1.0) ** (i % 2) for i in range(nx)])  # sublattice sign
    assert np.array_equal(S @ A @ S, -A)         # bipartite


@pytest.mark.parametrize("L", [2, 3, 5, 6, 8])
def test_honeycomb_spectrum_matches_momentum_space(L):
    lam = np.linalg.eigvalsh(fi.honeycomb_adjacency(L))
    assert np.allclose(lam, fi.honeycomb_spectrum(L), atol=1e-12)


@pytest.mark.parametrize("delta", [0.125, 0.0625, 0.5])
def test_hopping_exp_matches_pade(delta):
    A = fi.honeycomb_adjacency(3)
    E = fi.hopping_exp(A, delta, 1.0)
    Einv = fi.hopping_exp(A, delta, 1.0, -1.0)
    assert np.allclose(E, scipy.linalg.expm(delta * A), rtol=1e-13, atol=1e-14)
    assert np.allclose(E @ Einv, np.eye(A.shape[0]), atol=1e-13)
    assert np.array_equal(E, E.T)


def test_field_law_and_seeding():
    phi = fi.field(1001, 0, 4000, 18, 0.125, 3.0)
    assert phi.shape == (4000, 18)
    assert abs(phi.mean()) < 0.01
    assert abs(phi.var() / (0.125 * 3.0) - 1.0) < 0.02       # variance delta*U
    assert np.array_equal(phi, fi.field(1001, 0, 4000, 18, 0.125, 3.0))
    assert not np.array_equal(phi, fi.field(1001, 1, 4000, 18, 0.125, 3.0))


def test_workload_shapes():
    w = fi.workload("batch18", batch=3)
    assert [p.nx for p in w] == [18] * 3 and w[0].nt == 64 and w[0].n_stab == 8
    assert abs(w[0].delta - 0.125) < 1e-15
    u = fi.workload("uneven512")
    assert len(u) == 512
    pairs = {(p.nx, p.nt) for p in u}
    assert len(pairs) == 48
    assert all(abs(p.delta - 1 / 16) < 1e-15 for p in u)


def test_sparse_rows_reproduce_the_matrix():
    A = fi.honeycomb_adjacency(4)
    col, val = fi.sparse_rows(A)
    assert col.dtype == np.int32 and col.shape == (32, 3)
    B = np.zeros_like(A, dtype=float)
    for i in range(A.shape[0]):
        for m in range(col.shape[1]):
            B[i, col[i, m]] += val[i, m]
    assert np.array_equal(B, A)
    col4, val4 = fi.sparse_rows(A, 4)  # padded: (col = i, val = 0)
    assert np.all(col4[:, 3] == np.arange(32)) and np.all(val4[:, 3] == 0)
    with pytest.raises(ValueError):
        fi.sparse_rows(A, 2)


def test_bss_proposals_law_and_sharding():
    d, u, w = fi.bss_proposals("batch18", 3)
    assert d.shape == u.shape == w.shape == (256, 18)
    assert abs(d.var() / (0.125 * 3.0) - 1.0) < 0.05 and 0.0 <= u.min() and u.max() < 1.0
    assert np.all(w == 1.0)
    d2, u2, _ = fi.bss_proposals("batch18", 3, first=100, count=7)
    assert np.array_equal(d2, d[100:107]) and np.array_equal(u2, u[100:107])
    assert not np.array_equal(d, fi.bss_proposals("batch18", 4)[0])
