"""The hand-written FP64 refinements of the QR and LU steps against IEEE results, on the GPU.

rcp64, rsqrt64 and sqrt64 (an FP32 hardware estimate refined by two Newton steps) and the
Householder reflector's reciprocals (reflector_math: FP32 seeds refined by one third-order step of
Householder's iteration) replace IEEE division and square root in the serial steps of Section 7's
QR re-orthogonalisation.  fd_check_fp64_refinements evaluates them beside CUDA's correctly rounded
operations over a sweep of arguments that crosses the FP32 range edges (where they switch to the
IEEE operation), and the test bounds the distance in units in the last place (ulp):
  rcp64  <= 1 ulp from CUDA's correctly rounded 1/x,
  rsqrt64 <= 2 ulp and sqrt64 <= 2 ulp from the exact value (extended precision on the host),
  reflector (alpha, 1/c, tau) <= 8 ulp relative to the exact formula,
and requires identical results where the reference is 0, infinite or NaN."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


def _run(x, y, z):
    from paper_2604_02130_gb300 import _lib as L

    lib = L.load()
    dev = torch.device("cuda", 0)
    tx, ty, tz = (torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
                  for a in (x, y, z))
    out = torch.empty(16 * len(x), dtype=torch.float64, device=dev)
    rc = lib.fd_check_fp64_refinements(ctypes.c_void_p(tx.data_ptr()), ctypes.c_void_p(ty.data_ptr()),
                                       ctypes.c_void_p(tz.data_ptr()), len(x),
                                       ctypes.c_void_p(out.data_ptr()), None)
    assert rc == L.FD_OK
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(len(x), 16)


def _ulps(a, b):
    """Distance in ulps between finite doubles of the same sign."""
    ia = np.asarray(a, dtype=np.float64).view(np.int64)
    ib = np.asarray(b, dtype=np.float64).view(np.int64)
    return np.abs(ia - ib)


def _arguments():
    vals = []
    for e in range(-1074, 1024, 7):
        for m in (1.0, 1.2345678901234567, 1.5, 1.9999999999999998):
            vals.append(np.ldexp(m, e))
    # the FP32 range edges where the refinements hand over to the IEEE operations
    f32_min, f32_max = float(np.finfo(np.float32).tiny), float(np.finfo(np.float32).max)
    for v in (1e-36, 1e36, 1e-38, 1e38, f32_min, f32_max, 1e-45, 1e-40, 1e-300, 1e300,
              5e-324, 2.2250738585072014e-308, 1.7976931348623157e308):
        vals += [v, np.nextafter(v, 0.0), np.nextafter(v, np.inf)]
    rng = np.random.default_rng(11)
    vals += list(np.exp(rng.uniform(-80, 80, size=2000)))
    vals = np.array(vals, dtype=np.float64)
    vals = vals[np.isfinite(vals)]
    return np.concatenate([vals, -vals[::7], [0.0, -0.0]])


def test_rcp_rsqrt_sqrt_against_ieee():
    x = _arguments()
    o = _run(x, np.zeros_like(x), np.ones_like(x))
    # rcp64 against CUDA's correctly rounded reciprocal
    ref = o[:, 1]
    fin = np.isfinite(ref) & (ref != 0)
    assert _ulps(o[fin, 0], ref[fin]).max() <= 1
    assert np.array_equal(o[~fin, 0], ref[~fin])  # inf, 0 and signs as IEEE
    # rsqrt64 and sqrt64 against the exact value (extended precision)
    pos = (x > 0)
    xl = x[pos].astype(np.longdouble)
    rs_exact = (1 / np.sqrt(xl)).astype(np.float64)
    sq_exact = np.sqrt(xl).astype(np.float64)
    fr = np.isfinite(rs_exact) & (rs_exact != 0)
    assert _ulps(o[pos, 2][fr], rs_exact[fr]).max() <= 2
    assert _ulps(o[pos, 4], sq_exact).max() <= 2
    # CUDA's own operations on the same arguments (the reference the refinements replace)
    assert _ulps(o[pos, 5], sq_exact).max() == 0
    assert _ulps(o[pos, 3][fr], rs_exact[fr]).max() <= 1
    # non-positive arguments: the refinements fall back to the IEEE operations
    neg = x < 0
    assert np.all(np.isnan(o[neg, 2])) and np.all(np.isnan(o[neg, 3]))
    zero = x == 0
    assert np.all(np.isinf(o[zero, 2])) and np.all(o[zero, 4] == 0)


def test_reflector_against_exact_formula():
    rng = np.random.default_rng(12)
    n = 4000
    mag = np.exp(rng.uniform(-60, 60, size=n))
    ang = rng.uniform(0, 2 * np.pi, size=n)
    a, b = mag * np.cos(ang), mag * np.sin(ang)
    z = (mag * np.exp(rng.uniform(-30, 30, size=n))) ** 2
    # edges: FP32 range limits of |x|^2 and of the norm, a zero leading entry, a zero column, and
    # a leading entry near the bottom of the FP64 range (|x|^2 still a normal double)
    extra = [(1e-19, 0.0, 1.0), (1e-18, 0.0, 0.0), (1e18, 0.0, 0.0), (1e17, 1e17, 1e36),
             (0.0, 0.0, 4.0), (0.0, 0.0, 0.0), (1e-150, 1e-150, 1e-300), (3.0, -4.0, 0.0)]
    a = np.concatenate([a, [e[0] for e in extra]])
    b = np.concatenate([b, [e[1] for e in extra]])
    z = np.concatenate([z, [e[2] for e in extra]])
    o = _run(a, b, z)
    al, bl, zl = (v.astype(np.longdouble) for v in (a, b, z))
    x2 = al * al + bl * bl
    ax = np.sqrt(x2)
    nrm = np.sqrt(x2 + zl)
    zero_col = (x2 + zl) == 0
    assert np.array_equal(o[:, 11] == 1.0, zero_col)
    ok = ~zero_col
    with np.errstate(divide="ignore", invalid="ignore"):
        ux = np.where(ax > 0, al / ax, 1.0)
        uy = np.where(ax > 0, bl / ax, 0.0)
        alpha_re, alpha_im = -ux * nrm, -uy * nrm
        den = np.where(ax > 0, ax * (ax + nrm), nrm)
        cinv_re = np.where(ax > 0, al / den, 1.0 / nrm)
        cinv_im = np.where(ax > 0, -bl / den, 0.0)
        tau = 1 + ax / nrm

    def rel(got, re, im):
        mag = np.sqrt(re * re + im * im)
        return (np.abs(got[0] - re) + np.abs(got[1] - im)) / mag

    e_alpha = rel((o[ok, 6], o[ok, 7]), alpha_re[ok], alpha_im[ok])
    e_cinv = rel((o[ok, 8], o[ok, 9]), cinv_re[ok], cinv_im[ok])
    e_tau = np.abs(o[ok, 10] - tau[ok]) / tau[ok]
    assert float(e_alpha.max()) <= 8 * EPS
    assert float(e_cinv.max()) <= 8 * EPS
    assert float(e_tau.max()) <= 8 * EPS
