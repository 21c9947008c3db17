"""Integer rules the GPU kernels use in place of fp64 operations (GB300's fp64 pipe is narrow),
checked against IEEE-754 double arithmetic on the host:
- the enforcer's sum of two halved row scales in [1/4, 1): X = h 2^54 is an integer, the
  exact sum C = X_i + X_j lies in [2^53, 2^55) and is rounded to 53 bits, ties to even;
- its fixed-point row-sum term floor(v 2^-U) from the bits of a non-negative v."""
import math
import random
import struct


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _dbl(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def _fixed(h):
    b = _bits(h)
    e = b >> 52
    assert e in (1021, 1022)  # h in [1/4, 1)
    return ((b & ((1 << 52) - 1)) | (1 << 52)) << (e - 1021)


def _fixed_sum_rn(hi, hj):
    c = _fixed(hi) + _fixed(hj)
    k = 1 + (c >> 54)
    q = (c + (k - 1) + ((c >> k) & 1)) >> k
    return _dbl(((1021 + k) << 52) + q - (1 << 52))


def test_fixed_point_sum_is_the_ieee_sum():
    rng = random.Random(7)
    cases = [(0.25, 0.25), (0.5, 0.5), (0.25, 0.9999999999999999), (0.9999999999999999, 0.9999999999999999),
             (0.5, 0.4999999999999999), (0.75, 0.25)]
    for _ in range(200000):
        a = rng.uniform(0.25, 1.0)
        b = rng.uniform(0.25, 1.0) if rng.random() < 0.5 else _dbl(_bits(a) ^ rng.getrandbits(3))
        if 0.25 <= b < 1.0:
            cases.append((a, b))
    for a, b in cases:
        assert _fixed_sum_rn(a, b) == a + b, (a, b)


def _term(v, U):
    """floor(v 2^-U) as the enforcer forms it: the significand moved to the top of 64 bits
    (M = m 2^11) and shifted right by 1086 + U - e; zero and subnormals give 0."""
    b = _bits(v)
    e = b >> 52
    if e == 0:
        return 0
    M = ((b & ((1 << 52) - 1)) | (1 << 52)) << 11
    s = 1086 + U - e
    assert s >= 1  # v < 2^(U + 63)
    return M >> s if s < 64 else 0


def test_fixed_point_term_is_the_floor():
    rng = random.Random(11)
    for _ in range(100000):
        U = rng.randint(-1000, 900)
        v = math.ldexp(rng.random(), U + rng.randint(-80, 62))
        if v < 2.0 ** -1022:
            continue
        exact = math.floor(math.ldexp(v, -U)) if v >= 2.0 ** U else 0
        assert _term(v, U) == exact
