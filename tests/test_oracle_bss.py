"""Pins for the local (BSS) slice update of oracle.bss.

Independent references: determinant ratios from the full fermion matrix of Section 2 (brute
force), the matrix determinant lemma r_x = 1 + delta_x (1 - [G_{t-1}]_xx) with delta_x =
e^{i dphi_x} - 1 and G_{t-1} the diagonal block of the inverse full matrix, and the two limits
(every proposal accepted / rejected).  A planted mistake (the proposal applied to the wrong field
row) is rejected.
"""
import numpy as np
import pytest

import fd_inputs as fi
from oracle import bss, fermion_matrix, stable
from oracle import force as oforce


def _case(L=2, nt=8, beta=1.0, n_stab=4, seed=41):
    p = fi.make_problem(L, nt, beta, 2.0, n_stab, seed, 0)
    rng = np.random.default_rng(seed)
    dphi = rng.normal(0.0, 0.8, size=p.nx)
    u = rng.uniform(size=p.nx)
    w = np.exp(rng.normal(0.0, 0.3, size=p.nx))
    return p, dphi, u, w


@pytest.mark.parametrize("t", [1, 3, 8])
def test_ratios_match_brute_force_and_lemma(t):
    p, dphi, u, w = _case()
    row, acc, total, G, ratios = bss.slice_update(p.E, p.phi, p.n_stab, t, dphi, u, w)
    phi = p.phi.copy()
    for x in range(p.nx):
        Gb = fermion_matrix.green_blocks(p.E, phi)[t - 1]
        delta = np.exp(1j * dphi[x]) - 1.0
        lemma = 1.0 + delta * (1.0 - Gb[x, x])
        trial = phi.copy()
        trial[t - 1, x] += dphi[x]
        brute = np.exp(fermion_matrix.logdet(p.E, trial) - fermion_matrix.logdet(p.E, phi))
        assert abs(ratios[x] - brute) < 1e-10 * max(1.0, abs(brute))
        assert abs(ratios[x] - lemma) < 1e-10 * max(1.0, abs(lemma))
        if acc[x]:
            phi = trial
    assert np.allclose(row, phi[t - 1])
    assert np.abs(G - fermion_matrix.green_blocks(p.E, phi)[t - 1]).max() < 1e-10
    assert 0 < acc.sum() < p.nx  # the case exercises both outcomes


def test_all_accepted_and_all_rejected():
    p, dphi, u, _ = _case(L=3, nt=16, beta=2.0, seed=42)
    t = 5
    row, acc, total, G, _ = bss.slice_update(p.E, p.phi, p.n_stab, t, dphi, u,
                                             np.full(p.nx, 1e300))
    assert acc.all()
    phi2 = p.phi.copy()
    phi2[t - 1] += dphi
    ld0, _ = stable.logdet_green(p.E, p.phi, p.n_stab)
    ld1, _ = stable.logdet_green(p.E, phi2, p.n_stab)
    d = ld1 - ld0
    assert abs(total.real - d.real) < 1e-10 * max(1.0, abs(d))
    assert abs(np.angle(np.exp(1j * (total.imag - d.imag)))) < 1e-10 * max(1.0, abs(d))
    assert np.abs(G - oforce.green_at(p.E, phi2, p.n_stab, t - 1)).max() < 1e-10
    row, acc, total, G, _ = bss.slice_update(p.E, p.phi, p.n_stab, t, dphi, u, np.zeros(p.nx))
    assert not acc.any() and total == 0 and np.array_equal(row, p.phi[t - 1])
    assert np.abs(G - oforce.green_at(p.E, p.phi, p.n_stab, t - 1)).max() < 1e-13


def test_wrong_row_mutant_is_caught():
    p, dphi, u, w = _case()
    t = 3
    Gb = fermion_matrix.green_blocks(p.E, p.phi)[t - 1]
    delta = np.exp(1j * dphi[0]) - 1.0
    lemma = 1.0 + delta * (1.0 - Gb[0, 0])
    trial = p.phi.copy()
    trial[t, 0] += dphi[0]  # row t instead of t-1
    wrong = np.exp(fermion_matrix.logdet(p.E, trial) - fermion_matrix.logdet(p.E, p.phi))
    assert abs(wrong - lemma) > 1e-3
