"""Writes tests/golden/highprec_beta64.json from oracle.highprec (mpmath, 250 digits).

The stored values are log det(1 + B_Nt...B_1) and G = (1 + B_Nt...B_1)^{-1} of the plain
definition (Section 2) evaluated with 250 significant digits on seeded honeycomb inputs, so that
FP64 paths can be checked at beta = 64 without mpmath.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import fd_inputs as fi  # noqa: E402
from oracle import highprec  # noqa: E402

CASES = [
    dict(L=2, nt=512, beta=64.0, U=3.5, n_stab=16, seed=1002, c=0),
    dict(L=2, nt=512, beta=64.0, U=3.5, n_stab=8, seed=1002, c=1),
    dict(L=2, nt=256, beta=32.0, U=3.0, n_stab=8, seed=1003, c=0),
]


def main():
    out = {"source": "oracle.highprec (mpmath, dps=250), plain product of Section 2",
           "cases": []}
    for case in CASES:
        p = fi.make_problem(case["L"], case["nt"], case["beta"], case["U"], case["n_stab"],
                            case["seed"], case["c"])
        ld, G = highprec.logdet_green(p.E, p.phi, dps=250)
        out["cases"].append(dict(case, logdet=[ld.real, ld.imag], G_re=G.real.tolist(),
                                 G_im=G.imag.tolist()))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "highprec_beta64.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    # unequal-time Green's function G(tau, 0) = (L_tau^{-1} + R_tau)^{-1} at beta = 32
    case = dict(L=2, nt=256, beta=32.0, U=3.0, n_stab=8, seed=1003, c=1, taus=[1, 37, 128, 255])
    p = fi.make_problem(case["L"], case["nt"], case["beta"], case["U"], case["n_stab"],
                        case["seed"], case["c"])
    gt = highprec.green_tau(p.E, p.phi, case["taus"], dps=250)
    out2 = {"source": "oracle.highprec.green_tau (mpmath, dps=250), Section 4.2", "case": case,
            "G_re": {str(t): gt[t].real.tolist() for t in case["taus"]},
            "G_im": {str(t): gt[t].imag.tolist() for t in case["taus"]}}
    path2 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "highprec_gtau.json")
    with open(path2, "w") as f:
        json.dump(out2, f, indent=1)


if __name__ == "__main__":
    main()
