"""The fixed-point products of the element-wise evaluation (csrc/fixrot.cuh),
compiled for the host from the same header: E = v_o e^{j(theta_o - theta_q)}
and G = conj(Yc) E against 50-digit references, the rounding to double
against exact rational arithmetic, and the FP64 fallback (non-finite angles,
v or Yc outside the fixed-point range) against the IEEE products."""
import math
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2302_10736_gb300", "csrc")
EPS = 2.0 ** -53


@pytest.fixture(scope="module")
def host(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("fixrot") / "fixrot_host")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                           os.path.join(os.path.dirname(__file__), "fixrot_host.cpp")])

    def run(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             check=True).stdout
        return out.splitlines()

    return run


def _E(host, cases):
    out = host(["E %r %r %r" % (float(v), float(a), float(b)) for v, a, b in cases])
    return np.array([[float(t) for t in ln.split()] for ln in out])


def test_product_against_50_digit_reference(host):
    """|E - E_ref| <= (2^-53 + 2^-56) |v_o| per component (one rounding plus
    the fixed-point truncations)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(5)
    n = 4000
    vo = np.concatenate([rng.uniform(0.9, 1.1, n), 10.0 ** rng.uniform(-250, 250, n) * rng.choice([-1, 1], n)])
    tho = np.concatenate([rng.normal(0, 0.3, n), rng.uniform(-65535, 65535, n)])
    thq = np.concatenate([tho[:n] + rng.normal(0, 0.05, n), rng.uniform(-65535, 65535, n)])
    # nearly equal and nearly opposite angles (tiny components of E)
    tho[:200] = thq[:200] + np.pi / 2 + rng.normal(0, 1e-9, 200)
    tho[200:400] = thq[200:400]
    r = _E(host, zip(vo, tho, thq))
    for k in range(vo.size):
        d = mp.mpf(tho[k]) - mp.mpf(thq[k])
        er, ei = mp.mpf(vo[k]) * mp.cos(d), mp.mpf(vo[k]) * mp.sin(d)
        bound = (EPS + 2.0 ** -56) * abs(vo[k])
        assert abs(float(mp.mpf(r[k, 0]) - er)) <= bound, k
        assert abs(float(mp.mpf(r[k, 1]) - ei)) <= bound, k
    # equal angles give a real E = v_o to within its rounding
    assert np.all(np.abs(r[200:400, 0] - vo[200:400]) <= EPS * np.abs(vo[200:400]))
    assert np.all(np.abs(r[200:400, 1]) <= 2.0 ** -56 * np.abs(vo[200:400]))


def test_rounding_to_double_is_exact(host):
    """fix_to_double(x, e1) = x 2^(e1 - 1085) rounded to nearest (ties away
    from zero), checked with exact rationals, ties included."""
    rng = np.random.default_rng(9)
    xs = [int(v) for v in rng.integers(-(1 << 62), 1 << 62, 3000)]
    xs += [1, -1, 3, (1 << 62) - 1, -(1 << 62) + 1, (1 << 53) + 1, ((1 << 53) + 1) << 9, (3 << 52) + 1]
    xs += [((1 << 52) + k) * 2 + 1 for k in range(50)] + [-(((1 << 52) + k) * 2 + 1) for k in range(50)]   # ties
    es = [int(v) for v in rng.integers(70, 2000, len(xs))]
    out = host(["D %d %d" % (x, e) for x, e in zip(xs, es)])
    for x, e, h in zip(xs, es, out):
        got = struct.unpack("<d", bytes.fromhex(h)[::-1])[0]
        exact = Fraction(x) * Fraction(2) ** (e - 1085)
        lo = float(exact)   # nearest, ties to even
        if Fraction(lo) != exact:
            # the two neighbours of the exact value; ours must be the nearer, a tie the larger magnitude
            other = math.nextafter(lo, math.inf if Fraction(lo) < exact else -math.inf)
            dl, do = abs(Fraction(lo) - exact), abs(Fraction(other) - exact)
            want = lo if dl < do else other if do < dl else (lo if abs(lo) > abs(other) else other)
        else:
            want = lo
        assert got == want, (x, e, got, want)
    assert host(["D 0 1023"]) == ["0000000000000000"]


def test_fallback_keeps_ieee_semantics(host):
    """v_o zero, subnormal, huge, negative; angles inf and NaN: the FP64
    products (NaN propagates, zero gives zero)."""
    nan = float("nan")
    cases = [(0.0, 0.3, -0.2), (5e-324, 0.3, -0.2), (1e300, 0.3, -0.2), (-1.05, 0.3, -0.2),
             (1.0, nan, 0.1), (1.0, 0.1, nan), (1.0, math.inf, 0.1), (nan, 0.1, 0.2), (math.inf, 0.1, 0.1)]
    r = _E(host, cases)
    assert r[0, 0] == 0.0 and r[0, 1] == 0.0
    for k in (1, 2, 3):
        v, a, b = cases[k]
        ref = (v * math.cos(a - b), v * math.sin(a - b))
        tol = max(4 * EPS * abs(v), 2 * 5e-324)
        assert abs(r[k, 0] - ref[0]) <= tol and abs(r[k, 1] - ref[1]) <= tol, k
    assert np.isnan(r[4:8]).all()
    # inf v_o: (inf, inf) conj(U_q) by FP64 products gives inf + j NaN
    assert r[8, 0] == math.inf and np.isnan(r[8, 1])


def test_coupling_product_against_50_digit_reference(host):
    """G = conj(Yc) E with Yc in block floating point: |G - G_ref| <= 2.25 *
    2^-53 |Yc| |v_o| per component (fixed-point truncations below about 2^-53
    |G|, plus one rounding of at most 2^-53 |G|); Yc of every magnitude, one
    component zero or tiny."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(7)
    n = 6000
    vo = np.concatenate([rng.uniform(0.9, 1.1, n), 10.0 ** rng.uniform(-200, 200, n)])
    tho = np.concatenate([rng.normal(0, 0.3, n), rng.uniform(-6e4, 6e4, n)])
    thq = np.concatenate([tho[:n] + rng.normal(0, 0.05, n), rng.uniform(-6e4, 6e4, n)])
    yr = np.concatenate([rng.normal(0, 20, n), 10.0 ** rng.uniform(-200, 200, n) * rng.choice([-1, 1], n)])
    yi = np.concatenate([rng.normal(0, 20, n), 10.0 ** rng.uniform(-200, 200, n) * rng.choice([-1, 1], n)])
    yr[:100] = 0.0
    yi[100:200] = 1e-30 * yr[100:200]
    out = host(["G %r %r %r %r %r" % tuple(map(float, c)) for c in zip(vo, tho, thq, yr, yi)])
    r = np.array([[float(t) for t in ln.split()] for ln in out])
    for k in range(vo.size):
        d = mp.mpf(tho[k]) - mp.mpf(thq[k])
        er, ei = mp.mpf(vo[k]) * mp.cos(d), mp.mpf(vo[k]) * mp.sin(d)
        gr = mp.mpf(yr[k]) * er + mp.mpf(yi[k]) * ei   # conj(Yc) E
        gi = mp.mpf(yr[k]) * ei - mp.mpf(yi[k]) * er
        bound = 2.25 * EPS * float(abs(vo[k]) * mp.sqrt(mp.mpf(yr[k]) ** 2 + mp.mpf(yi[k]) ** 2))
        assert abs(float(mp.mpf(r[k, 0]) - gr)) <= bound, k
        assert abs(float(mp.mpf(r[k, 1]) - gi)) <= bound, k


def test_coupling_fallback(host):
    """Yc zero, subnormal or non-finite, and products beyond the double range:
    the FP64 products."""
    nan, inf = float("nan"), math.inf
    cases = [(1.0, 0.2, -0.1, 0.0, 0.0), (1.0, 0.2, -0.1, 5e-324, 0.0), (1.0, 0.2, -0.1, nan, 1.0),
             (1.0, 0.2, -0.1, inf, 0.0), (1e200, 0.2, -0.1, 1e200, 1.0), (1e-200, 0.2, -0.1, 1e-200, 1e-201)]
    out = host(["G %r %r %r %r %r" % c for c in cases])
    r = np.array([[float(t) for t in ln.split()] for ln in out])
    assert r[0, 0] == 0.0 and r[0, 1] == 0.0
    assert abs(r[1, 0]) <= 1e-323 and abs(r[1, 1]) <= 1e-323
    assert np.isnan(r[2]).all()
    assert r[3, 0] == inf and np.isinf(r[3, 1])
    assert r[4, 0] == inf                                   # 1e400 overflows, as the FP64 product does
    assert abs(r[5, 0]) <= 1e-320 and abs(r[5, 1]) <= 1e-320   # 1e-400 underflows
