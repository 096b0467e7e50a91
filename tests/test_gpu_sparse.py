"""GPU parity of the intermediate-volume variant (fd_green_sparse, Sections 8-9) against
oracle.product_form: log det and G with every slice's hopping factor applied as the product of
n linear factors of the sparse K = delta*kappa*A, QR every n_stab slices.

Cases span several size classes in one call (Nx = 8 ... 72), n = 1, 2, 4, 8 factors, a padded
row width (q = 4 with one zero entry per row), a configuration above one tensor tile and the
shared-memory placement (Nx = 288, matrices in the CTA's global scratch), log det without G, and
a column index outside the matrix (flagged FD_ERR_NUMERIC, no access).  Tolerances are those of
the FP64 path: log det relative 1e-10, G 1e-10 max(1, max|G|)^2.
"""
import numpy as np
import pytest

import fd_inputs as fi
from oracle import product_form

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(L, nt, beta, U, n_stab, seed, c, nfac, q=None):
    p = fi.make_problem(L, nt, beta, U, n_stab, seed, c)
    col, val = fi.sparse_rows(p.A, q)
    ld, G = product_form.logdet_green(p.A, p.delta, p.kappa, nfac, p.phi, p.n_stab)
    return p, col, val * (p.delta * p.kappa), ld, G


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.device("cuda", 0))


def _check(ld, G, ref_ld, ref_G):
    d = complex(ld) - ref_ld
    assert abs(d.real) <= 1e-10 * max(1.0, abs(ref_ld))
    assert abs(np.angle(np.exp(1j * d.imag))) <= 1e-10 * max(1.0, abs(ref_ld))
    if G is not None:
        scale = max(1.0, float(np.abs(ref_G).max())) ** 2
        assert np.abs(G.cpu().numpy() - ref_G).max() <= 1e-10 * scale


@pytest.mark.parametrize("nfac", [1, 2, 4, 8])
def test_sparse_matches_oracle_mixed_sizes(nfac):
    from paper_2604_02130_gb300 import api

    cases = [_case(2, 16, 2.0, 2.0, 4, 901, 0, nfac), _case(3, 24, 3.0, 3.0, 8, 902, 1, nfac),
             _case(4, 16, 2.0, 3.0, 4, 903, 2, nfac), _case(6, 16, 2.0, 3.0, 8, 904, 3, nfac),
             _case(3, 16, 4.0, 3.0, 4, 905, 4, nfac, q=4)]
    probs = [(_dev(p.phi), p.n_stab) for p, *_ in cases]
    hops = [(_dev(col), _dev(val)) for _, col, val, _, _ in cases]
    ld, G = api.green_sparse(probs, hops, nfac=nfac)
    torch.cuda.synchronize()
    ctx = api.default_context()
    assert all(s == 0 for s in ctx.status(len(cases)))
    ld = ld.cpu().numpy()
    for k, (p, col, val, rld, rG) in enumerate(cases):
        _check(ld[k], G[k], rld, rG)


def test_sparse_large_nx_and_logdet_only():
    from paper_2604_02130_gb300 import api

    p, col, val, rld, rG = _case(12, 8, 1.0, 3.0, 4, 906, 0, 4)
    assert p.nx == 288
    probs = [(_dev(p.phi), p.n_stab)]
    hops = [(_dev(col), _dev(val))]
    ld, G = api.green_sparse(probs, hops, nfac=4)
    ld2, none = api.green_sparse(probs, hops, nfac=4, with_green=False)
    torch.cuda.synchronize()
    assert none is None
    _check(ld.cpu().numpy()[0], G[0], rld, rG)
    _check(ld2.cpu().numpy()[0], None, rld, None)


def test_sparse_equals_dense_with_taylor_E():
    """The same arithmetic through fd_green with the dense E = T_n(K): agreement to rounding."""
    from paper_2604_02130_gb300 import api

    p, col, val, rld, _ = _case(3, 32, 4.0, 3.0, 8, 907, 0, 4)
    E4 = product_form.slice_matrix(p.A, p.delta, p.kappa, 4)
    ld_d, G_d = api.green([(_dev(E4), None, _dev(p.phi), p.n_stab)], prec="fp64")
    ld_s, G_s = api.green_sparse([(_dev(p.phi), p.n_stab)], [(_dev(col), _dev(val))], nfac=4)
    torch.cuda.synchronize()
    assert abs(complex(ld_d.cpu()[0]) - complex(ld_s.cpu()[0])) < 1e-10 * max(1.0, abs(rld))
    scale = max(1.0, G_d[0].abs().max().item()) ** 2
    assert (G_d[0] - G_s[0]).abs().max().item() < 1e-10 * scale


def test_sparse_bad_column_is_flagged():
    from paper_2604_02130_gb300 import api

    p, col, val, _, _ = _case(2, 8, 1.0, 2.0, 4, 908, 0, 2)
    col = col.copy()
    col[3, 1] = p.nx + 5  # outside the matrix
    ld, G = api.green_sparse([(_dev(p.phi), p.n_stab)], [(_dev(col), _dev(val))], nfac=2)
    torch.cuda.synchronize()
    assert api.default_context().status(1) == [-4]  # FD_ERR_NUMERIC


def test_sparse_validation():
    from paper_2604_02130_gb300 import api

    p, col, val, _, _ = _case(2, 8, 1.0, 2.0, 4, 909, 0, 2)
    probs = [(_dev(p.phi), p.n_stab)]
    hops = [(_dev(col), _dev(val))]
    for nfac in (0, 9):
        with pytest.raises(api.FdError):
            api.green_sparse(probs, hops, nfac=nfac)
