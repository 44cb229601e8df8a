"""The constants written into the double-word exponential of csrc/dwarith.cuh (and the
ln 10 pairs of csrc/k_prior.cu) are the float pairs nearest the mathematical values, and
the Cody-Waite split of ln2/16 has the bit budget its exactness argument needs.  Parsed
from the sources and checked against 60-digit values; no GPU."""
import os
import re

import mpmath as mp
import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2607_06834_b300", "csrc")
mp.mp.dps = 60


def _src(name):
    with open(os.path.join(CSRC, name)) as f:
        return f.read()


def _f(tok):
    return float.fromhex(tok.rstrip("f")) if "0x" in tok else float(tok.rstrip("f"))


def _nearest_pair(v):
    h = float(np.float32(float(v)))
    l = float(np.float32(float(v - mp.mpf(h))))
    return h, l


def _bits(x):
    """significant bits of a float (from its binary mantissa)."""
    if x == 0.0:
        return 0
    m = int(np.float32(abs(x)).view(np.uint32)) & 0x7FFFFF
    m |= 0x800000
    while m % 2 == 0:
        m //= 2
    return m.bit_length()


def test_exp2_sixteenth_table():
    s = _src("dwarith.cuh")
    body = s[s.index("kExp2Sixteenth[16] = {"):]
    body = body[:body.index("};")]
    pairs = re.findall(r"\{\s*([-0-9a-fx.p+]+f?)\s*,\s*([-0-9a-fx.p+]+f?)\s*\}", body)
    assert len(pairs) == 16
    for j, (h, l) in enumerate(pairs):
        exact = mp.mpf(2) ** (mp.mpf(j) / 16)
        assert (_f(h), _f(l)) == _nearest_pair(exact), j
        assert abs(mp.mpf(_f(h)) + mp.mpf(_f(l)) - exact) < mp.mpf(2) ** -48


def test_cody_waite_split_and_series():
    s = _src("dwarith.cuh")
    m = re.search(r"kC1 = ([-0-9a-fx.p+]+f), kC2 = ([-0-9a-fx.p+]+f), kC3 = ([-0-9a-fx.p+]+f), kInv = ([-0-9a-fx.p+]+f)", s)
    c1, c2, c3, inv = (_f(t) for t in m.groups())
    l16 = mp.log(2) / 16
    # n C1 and n C2 exact for |n| < 2^12: at most 12 significant bits each
    assert _bits(c1) <= 12 and _bits(c2) <= 12
    # the split's residual times the largest n of the reduction's range (|a| < 170) stays
    # below 2^-45 absolute in r, and n C1, n C2 stay exact there (|n| < 2^12)
    nmax = 170 * 16 / mp.log(2)
    assert nmax < 2 ** 12
    assert abs(mp.mpf(c1) + mp.mpf(c2) + mp.mpf(c3) - l16) * nmax < mp.mpf(2) ** -45
    assert inv == float(np.float32(float(16 / mp.log(2))))
    # 1/6 as a pair, 1/24, 1/120, 1/720 as floats
    sixth = re.search(r"make_float2\(([-0-9a-fx.p+]+f), ([-0-9a-fx.p+]+f)\), dw_mulf\(r, tail\)", s).groups()
    assert tuple(_f(t) for t in sixth) == _nearest_pair(mp.mpf(1) / 6)
    tail = re.search(r"__fmaf_rn\(__fmaf_rn\(r\.x, ([-0-9a-fx.p+]+f), ([-0-9a-fx.p+]+f)\), r\.x, ([-0-9a-fx.p+]+f)\)", s)
    assert [_f(t) for t in tail.groups()] == [float(np.float32(1 / k)) for k in (720.0, 120.0, 24.0)]
    # truncation of the series at r^6 for |r| <= ln2/32 (plus a rounding margin in n)
    r = 1.1 * float(mp.log(2) / 32)
    assert r ** 7 / 5040 < 2.0 ** -46


@pytest.mark.parametrize("name", ["kLn10 = ", "kHalfLn10 = "])
def test_ln10_pairs(name):
    s = _src("k_prior.cu")
    m = re.search(name + r"\{([-0-9a-fx.p+]+f), ([-0-9a-fx.p+]+f)\}", s)
    exact = mp.log(10) if name.startswith("kLn10") else mp.log(10) / 2
    assert tuple(_f(t) for t in m.groups()) == _nearest_pair(exact)
