"""Host checks of the double-float helpers (csrc/fd_df.cuh) that the BSS kernel uses to hold G.

The helpers are compiled for the host with g++ (no FP contraction, so every FP32 step rounds as
written, as the intrinsics do on the GPU) and driven through tests/host/df_check.cpp.  Expected
values are exact rational arithmetic (fractions.Fraction) on the same inputs:
* split: hi keeps the leading 24 bits of d, |d - hi - lo| < 2^-46 |d|, join(split(d)) close to d;
* widen: exact for normal FP32 values, subnormals flushed to zero;
* cms (g - a b for complex pairs): error below 2^-43 of |g| + |a||b| per component, including
  cancellations;
* add_re: the real part gains c with the same bound;
* abs2, recip, scale (the decision of a local update in double-float): relative errors below
  2^-44; greater agrees with the exact comparison wherever the operands differ by more than
  2^-44 of their size, including pairs that differ only in the low part.
A planted mistake (the conjugate product) is rejected by the same bound.
"""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "host", "df_check.cpp")


@pytest.fixture(scope="module")
def df_exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("df") / "df_check")
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-std=c++17", SRC, "-o", exe], check=True)
    return exe


def _run(exe, lines):
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.split("\n")
    return [[float.fromhex(t) for t in ln.split()] for ln in out if ln.strip()]


def _f32(x):
    return float(np.float32(x))


def _pair(rng, scale):
    """A normalised df pair (hi, lo) of magnitude ~scale."""
    d = rng.normal() * scale
    hi = _f32(d)
    lo = _f32(d - hi)
    return hi, lo


def test_split_join_widen(df_exe):
    rng = np.random.default_rng(3)
    vals = list(rng.normal(size=200) * np.exp(rng.uniform(-60, 60, size=200)))
    vals += [0.0, -0.0, 1.0, -1.5, 0.1, 2.0 ** -126, 2.0 ** -127, 3.0e38, 1e-300]
    res = _run(df_exe, ["s %s" % float(v).hex() for v in vals])
    for v, (hi, lo) in zip(vals, res):
        if abs(v) < 2.0 ** -126:
            assert hi == 0.0 and lo == 0.0
            continue
        assert _f32(hi) == hi and _f32(lo) == lo
        # hi: v truncated to 24 significant bits
        m, e = np.frexp(v)
        assert hi == np.ldexp(np.trunc(m * 2.0 ** 24), int(e) - 24)
        err = abs(Fraction(v) - Fraction(hi) - Fraction(lo))
        assert err < Fraction(2) ** -46 * abs(Fraction(v))
    joined = _run(df_exe, ["j %s %s" % (hi.hex(), lo.hex()) for hi, lo in res])
    for v, (hi, lo), (d,) in zip(vals, res, joined):
        assert d == hi + lo
        if abs(v) >= 2.0 ** -126:
            assert abs(d - v) <= 2.0 ** -45 * abs(v)
    fl = [_f32(x) for x in rng.normal(size=50) * np.exp(rng.uniform(-80, 80, size=50))]
    fl += [0.0, 1.0, -2.0, 1e-45, -1e-40]
    wide = _run(df_exe, ["w %s" % x.hex() for x in fl])
    for x, (d,) in zip(fl, wide):
        assert d == (0.0 if abs(x) < 2.0 ** -126 else x)


def _exact_cms(g, a, b):
    G = (Fraction(g[0]) + Fraction(g[1]), Fraction(g[2]) + Fraction(g[3]))
    A = (Fraction(a[0]) + Fraction(a[1]), Fraction(a[2]) + Fraction(a[3]))
    B = (Fraction(b[0]) + Fraction(b[1]), Fraction(b[2]) + Fraction(b[3]))
    re = G[0] - (A[0] * B[0] - A[1] * B[1])
    im = G[1] - (A[0] * B[1] + A[1] * B[0])
    size_re = abs(G[0]) + abs(A[0] * B[0]) + abs(A[1] * B[1])
    size_im = abs(G[1]) + abs(A[0] * B[1]) + abs(A[1] * B[0])
    return re, im, size_re, size_im


def _cases(rng, k):
    out = []
    for _ in range(k):
        sg, sa, sb = np.exp(rng.uniform(-8, 8, size=3))
        g = [*_pair(rng, sg), *_pair(rng, sg)]
        a = [*_pair(rng, sa), *_pair(rng, sa)]
        b = [*_pair(rng, sb), *_pair(rng, sb)]
        out.append((g, a, b))
    # cancellations: g equal to the product up to the last bits
    for _ in range(k // 4):
        a = [*_pair(rng, 1.0), *_pair(rng, 1.0)]
        b = [*_pair(rng, 1.0), *_pair(rng, 1.0)]
        re, im, _, _ = _exact_cms([0, 0, 0, 0], a, b)
        pr, pi = -float(re), -float(im)  # a b in FP64
        g = [_f32(pr), _f32(pr - _f32(pr)), _f32(pi), _f32(pi - _f32(pi))]
        out.append((g, a, b))
    return out


def _fmt(v):
    return " ".join(float(x).hex() for x in v)


def test_complex_multiply_subtract(df_exe):
    rng = np.random.default_rng(5)
    cases = _cases(rng, 400)
    res = _run(df_exe, ["m %s %s %s" % (_fmt(g), _fmt(a), _fmt(b)) for g, a, b in cases])
    bound = Fraction(2) ** -43
    for (g, a, b), r in zip(cases, res):
        re, im, sre, sim = _exact_cms(g, a, b)
        assert abs(Fraction(r[0]) + Fraction(r[1]) - re) <= bound * sre
        assert abs(Fraction(r[2]) + Fraction(r[3]) - im) <= bound * sim
        assert abs(r[1]) <= abs(r[0]) * 2.0 ** -23 and abs(r[3]) <= abs(r[2]) * 2.0 ** -23


def test_conjugate_product_mutant_is_rejected(df_exe):
    """The bound distinguishes g - a b from g - conj(a) b (a sign slip in the kernel's update)."""
    rng = np.random.default_rng(6)
    cases = _cases(rng, 40)
    res = _run(df_exe, ["m %s %s %s" % (_fmt(g), _fmt([a[0], a[1], -a[2], -a[3]]), _fmt(b))
                        for g, a, b in cases])
    bound = Fraction(2) ** -43
    caught = 0
    for (g, a, b), r in zip(cases, res):
        re, im, sre, sim = _exact_cms(g, a, b)
        if (abs(Fraction(r[0]) + Fraction(r[1]) - re) > bound * sre
                or abs(Fraction(r[2]) + Fraction(r[3]) - im) > bound * sim):
            caught += 1
    assert caught == len(cases)


def test_add_real(df_exe):
    rng = np.random.default_rng(7)
    gs = [[*_pair(rng, s), *_pair(rng, s)] for s in np.exp(rng.uniform(-3, 3, size=100))]
    cs = [_f32(x) for x in rng.normal(size=100)]
    res = _run(df_exe, ["r %s %s" % (_fmt(g), c.hex()) for g, c in zip(gs, cs)])
    for g, c, r in zip(gs, cs, res):
        want = Fraction(g[0]) + Fraction(g[1]) + Fraction(c)
        size = abs(Fraction(g[0])) + abs(Fraction(c))
        assert abs(Fraction(r[0]) + Fraction(r[1]) - want) <= Fraction(2) ** -45 * size
        assert r[2] == g[2] and r[3] == g[3]


def _fr(h, l):
    return Fraction(h) + Fraction(l)


def test_abs2_recip_scale_greater(df_exe):
    rng = np.random.default_rng(8)
    rs = [[*_pair(rng, s), *_pair(rng, s)] for s in np.exp(rng.uniform(-20, 20, size=200))]
    res = _run(df_exe, ["a %s" % _fmt(r) for r in rs])
    for r, (th, tl) in zip(rs, res):
        want = _fr(r[0], r[1]) ** 2 + _fr(r[2], r[3]) ** 2
        assert abs(_fr(th, tl) - want) <= Fraction(2) ** -44 * want
    ts = [_pair(rng, s) for s in np.exp(rng.uniform(-40, 40, size=200))]
    ts = [(abs(h), abs(l) if h >= 0 else -abs(l)) for h, l in ts]
    res = _run(df_exe, ["q %s %s" % (h.hex(), l.hex()) for h, l in ts])
    for (h, l), (yh, yl) in zip(ts, res):
        assert abs(_fr(yh, yl) * _fr(h, l) - 1) <= Fraction(2) ** -44
    ys = [_pair(rng, s) for s in np.exp(rng.uniform(-5, 5, size=100))]
    res = _run(df_exe, ["c %s %s %s" % (_fmt(a), y[0].hex(), y[1].hex()) for a, y in zip(rs, ys)])
    for a, y, r in zip(rs, ys, res):
        for k in (0, 2):
            want = _fr(a[k], a[k + 1]) * _fr(*y)
            assert abs(_fr(r[k], r[k + 1]) - want) <= Fraction(2) ** -44 * abs(want)
    pairs = []
    for _ in range(300):
        a = _pair(rng, 1.0)
        kind = rng.integers(3)
        if kind == 0:
            b = _pair(rng, 1.0)
        elif kind == 1:  # same high part, different low parts
            b = (a[0], _f32(a[1] * (1 + rng.normal())))
        else:  # nearby values
            d = a[0] + a[1] + rng.normal() * 1e-12 * abs(a[0])
            b = (_f32(d), _f32(d - _f32(d)))
        pairs.append((a, b))
    res = _run(df_exe, ["g %s %s %s %s" % (a[0].hex(), a[1].hex(), b[0].hex(), b[1].hex())
                        for a, b in pairs])
    checked = 0
    for (a, b), (g,) in zip(pairs, res):
        fa, fb = _fr(*a), _fr(*b)
        if abs(fa - fb) > Fraction(2) ** -44 * max(abs(fa), abs(fb)):
            assert bool(g) == (fa > fb)
            checked += 1
    assert checked > 200
