"""Pins for the unequal-time Green's function G(tau, 0) (Section 4.2, Section 7 steps 7-9)."""
import json
import os

import numpy as np
import pytest

import fd_inputs as fi
from oracle import fermion_matrix, stable, unequal

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("L,nt,beta,U,n_stab", [(2, 16, 2.0, 2.0, 4), (2, 12, 4.0, 3.0, 3),
                                                (3, 8, 1.0, 3.0, 8)])
def test_green_tau_matches_brute_force(L, nt, beta, U, n_stab):
    p = fi.make_problem(L, nt, beta, U, n_stab, 21, 0)
    bf = fermion_matrix.inverse_column(p.E, p.phi, 0)
    st = unequal.green_tau_stable(p.E, p.phi, n_stab)
    pl = unequal.green_tau_plain(p.E, p.phi)
    for tau in range(nt):
        assert np.abs(st[tau] - bf[tau]).max() < 1e-11
        assert np.abs(pl[tau] - bf[tau]).max() < 1e-11


def test_green_tau_zero_is_green():
    p = fi.make_problem(3, 32, 4.0, 3.0, 8, 22, 0)
    _, G = stable.logdet_green(p.E, p.phi, 8)
    assert np.abs(unequal.green_tau_stable(p.E, p.phi, 8, [0])[0] - G).max() < 1e-14


def test_green_tau_golden_beta32():
    gold = json.load(open(os.path.join(GOLDEN, "highprec_gtau.json")))
    case = gold["case"]
    p = fi.make_problem(case["L"], case["nt"], case["beta"], case["U"], case["n_stab"],
                        case["seed"], case["c"])
    st = unequal.green_tau_stable(p.E, p.phi, case["n_stab"], case["taus"])
    for t in case["taus"]:
        ref = np.array(gold["G_re"][str(t)]) + 1j * np.array(gold["G_im"][str(t)])
        assert np.abs(st[t] - ref).max() < 1e-10 * max(1.0, np.abs(ref).max())


def test_green_tau_free_field_closed_form():
    # phi = 0: G(tau, 0) = U diag(e^{tau delta kappa lam} / (1 + e^{beta kappa lam})) U^T
    L, nt, beta = 3, 64, 16.0
    p = fi.make_problem(L, nt, beta, 3.0, 8, 0, 0, zero_field=True)
    lam, U = np.linalg.eigh(p.A)
    st = unequal.green_tau_stable(p.E, p.phi, 8, [0, 5, 33, 63])
    for tau, Gt in st.items():
        x = np.exp(tau * (beta / nt) * lam - np.logaddexp(0.0, beta * lam))
        assert np.abs(Gt - (U * x[None, :]) @ U.T).max() < 1e-12
