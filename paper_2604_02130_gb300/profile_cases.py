"""Small, self-checking cases for profiler captures of single kernels (a few GB on the device at
most, launches of a few hundred ms), run as ``python -m paper_2604_02130_gb300.profile_cases
<case>``.  Each case calls the public API twice (a capture skips the first launch) and checks
the per-configuration status.

Cases:
  chain_big288  the streamed chain kernel: 152 configurations of Nx = 288 (honeycomb L = 12),
                Nt = 128, beta = 8, n_stab = 16 -- eight blocks (128 slice products on the
                tensor cores, 8 double-float QRs) and the assembly per configuration; log det,
                split TF32.
"""
import sys

import torch

import fd_inputs as fi

from . import api

CASES = {
    "chain_big288": dict(L=12, nt=128, beta=8.0, U=3.0, n_stab=16, batch=152, want="logdet",
                         prec="3xtf32"),
}


def run(case: str) -> list:
    c = CASES[case]
    dev = torch.device("cuda", 0)
    probs = [fi.make_problem(c["L"], c["nt"], c["beta"], c["U"], c["n_stab"], 96, k)
             for k in range(c["batch"])]
    E = torch.from_numpy(probs[0].E).to(dev)
    Einv = torch.from_numpy(probs[0].Einv).to(dev)
    t = [(E, Einv, torch.from_numpy(p.phi).to(dev), p.n_stab) for p in probs]
    ctx = api.Context(0)
    b = api.Batch(ctx, t, c["want"], c["prec"])
    for _ in range(2):
        b.run()
    torch.cuda.synchronize()
    st = b.status()
    if any(s != 0 for s in st):
        raise RuntimeError("status %s" % st)
    return b.plan()


if __name__ == "__main__":
    print("ok", run(sys.argv[1] if len(sys.argv) > 1 else "chain_big288"))
