"""The integer-pipe sine/cosine of the phasor step (csrc/isincos.cuh) on the
CPU: every constant recomputed from first principles in exact integer
arithmetic (pi by Machin's formula, the table by Taylor series), and the
algorithm itself, compiled for the host from the same header, against the
C library's sin and cos."""
import math
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2302_10736_gb300", "csrc")
HEADER = os.path.join(CSRC, "isincos.cuh")
BITS = 400   # working precision of the integer references


def _header():
    return open(HEADER).read()


def _const(name):
    m = re.search(r"constexpr uint64_t %s = (0x[0-9a-f]+)ull;" % name, _header())
    assert m, name
    return int(m.group(1), 16)


def _table():
    body = re.search(r"kITrigTable\[kITrigN\] = \{(.*?)\};", _header(), re.S).group(1)
    pairs = re.findall(r"\{(0x[0-9a-f]+)ull, (0x[0-9a-f]+)ull\}", body)
    return [(int(c, 16), int(s, 16)) for c, s in pairs]


def _arctan_inv(x, one):
    """arctan(1/x) * one by its Taylor series (integer arithmetic)."""
    total, term, n, sign = 0, one // x, 1, 1
    while term:
        total += sign * (term // n)
        term //= x * x
        n += 2
        sign = -sign
    return total


ONE = 1 << BITS
PI = 16 * _arctan_inv(5, ONE) - 4 * _arctan_inv(239, ONE)   # Machin's formula, pi * 2^BITS


def _rdiv(num, den):
    return (2 * num + den) // (2 * den)


def _sincos_fixed(a):
    """sin and cos of a / 2^BITS (0 <= a < 2 * 2^BITS) by Taylor series, * 2^BITS."""
    s, c, term, n = 0, 0, ONE, 0
    while term:
        if n % 4 == 0:
            c += term
        elif n % 4 == 1:
            s += term
        elif n % 4 == 2:
            c -= term
        else:
            s -= term
        n += 1
        term = term * a // ONE // n
    return s, c


def test_pi_reference():
    assert abs(PI / ONE - math.pi) < 1e-15


def test_reduction_constants():
    c = (_const("kInv2PiHi") << 64) | _const("kInv2PiLo")
    assert c == (1 << 129) * ONE // PI                            # floor(2^129 / pi)
    assert _const("kTwoPi61") == _rdiv(2 * PI << 61, ONE)          # round(2 pi 2^61)


def test_polynomial_constants():
    assert _const("kInv6") == _rdiv(1 << 64, 6)
    assert _const("kInv24") == _rdiv(1 << 64, 24)
    assert _const("kInv120") == _rdiv(1 << 64, 120)
    assert _const("kInv720_54") == _rdiv(1 << 54, 720)
    assert _const("kInv5040_54") == _rdiv(1 << 54, 5040)


def test_table_entries():
    tab = _table()
    assert len(tab) == 64
    for j, (c, s) in enumerate(tab):
        sj, cj = _sincos_fixed(2 * PI * j // 256)
        assert c == _rdiv(cj << 62, ONE), j
        assert s == _rdiv(sj << 62, ONE), j


@pytest.fixture(scope="module")
def host_sincos(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("isc") / "isincos_host")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                           os.path.join(os.path.dirname(__file__), "isincos_host.cpp")])

    def run(x):
        out = subprocess.run([exe], input="\n".join("%.17g" % v for v in x), capture_output=True, text=True,
                             check=True).stdout
        return np.array([[float(t) for t in ln.split()] for ln in out.splitlines()])

    return run


def test_algorithm_on_the_host(host_sincos):
    """Within 2 ulp of 1 of libm's sin/cos over normal, wide, tiny angles, the
    table nodes and midpoints, and quadrant boundaries (|x| < 2^16)."""
    rng = np.random.default_rng(11)
    step = 2 * np.pi / 256
    x = np.concatenate([rng.normal(0, 0.25, 20000), rng.uniform(-65535.9, 65535.9, 20000),
                        rng.uniform(-1e-3, 1e-3, 2000), 10.0 ** rng.uniform(-300, -3, 2000),
                        np.arange(-500, 500) * step, np.arange(-500, 500) * step + step / 2,
                        np.arange(-300, 300) * (np.pi / 2), [0.0, -0.0, 5e-324, np.pi, -np.pi, 65535.99]])
    r = host_sincos(x)
    eps = np.finfo(np.float64).eps
    s_ref = np.array([math.sin(v) for v in x])
    c_ref = np.array([math.cos(v) for v in x])
    assert np.max(np.abs(r[:, 0] - s_ref)) <= 2 * eps
    assert np.max(np.abs(r[:, 1] - c_ref)) <= 2 * eps
    # away from zero the results are within about one rounding (relative)
    big = np.abs(s_ref) >= 0.5
    assert np.max(np.abs(r[big, 0] - s_ref[big]) / np.abs(s_ref[big])) <= 2 * eps
