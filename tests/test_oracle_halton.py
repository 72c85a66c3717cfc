"""Pins for the oracle's Halton ray directions (Sec. III-E, Eq. halton).

Checked against things other than the oracle itself: exact rational prefixes of the
radical-inverse sequence, its stratification property, exact nearest-float rounding
(Python Fractions), libm sin/cos in FP64, and identities of the sphere mapping.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden", "halton_prefix.json")
M3 = 3 ** 20


def nearest_f32(fr: Fraction) -> np.float32:
    """The float32 nearest to an exact rational (ties cannot occur for our inputs)."""
    g = np.float32(float(fr))
    cands = [np.nextafter(g, np.float32(-1)), g, np.nextafter(g, np.float32(2))]
    return min(cands, key=lambda c: abs(Fraction(float(c)) - fr))


def test_prefixes_match_textbook_values(orc):
    gold = json.load(open(GOLD))
    n = len(gold["base3"])
    u, v, num = orc.halton(n, offset=1)
    for i, (p, q) in enumerate(gold["base2"]):
        assert Fraction(float(u[i])) == Fraction(p, q)
    for i, (p, q) in enumerate(gold["base3"]):
        assert Fraction(int(num[i]), M3) == Fraction(p, q)
        assert v[i] == nearest_f32(Fraction(p, q))


def test_offset_zero_gives_the_pole():
    import oracle
    u, v, num = oracle.halton(1, offset=0)
    assert u[0] == 0.0 and v[0] == 0.0 and num[0] == 0
    d = oracle.ray_dirs(1, offset=0)[0]
    assert tuple(d) == (0.0, 0.0, 1.0)


@pytest.mark.parametrize("m", [1, 4, 8, 12])
def test_base2_stratified(orc, m):
    """The first 2^m - 1 base-2 values are exactly {k / 2^m : k = 1 .. 2^m - 1}."""
    u, _, _ = orc.halton(2 ** m - 1, offset=1)
    ks = sorted(int(Fraction(float(x)) * 2 ** m) for x in u)
    assert ks == list(range(1, 2 ** m))
    assert all(Fraction(float(x)) * 2 ** m == int(Fraction(float(x)) * 2 ** m) for x in u)


@pytest.mark.parametrize("m", [1, 3, 6, 9])
def test_base3_stratified(orc, m):
    """The first 3^m - 1 base-3 numerators are exactly {k 3^(20-m) : k = 1 .. 3^m - 1}."""
    _, _, num = orc.halton(3 ** m - 1, offset=1)
    step = 3 ** (20 - m)
    assert all(int(x) % step == 0 for x in num)
    assert sorted(int(x) // step for x in num) == list(range(1, 3 ** m))


def test_powers(orc):
    for k in range(0, 15):
        u, _, _ = orc.halton(1, offset=2 ** k)
        assert Fraction(float(u[0])) == Fraction(1, 2 ** (k + 1))
    for k in range(0, 15):
        _, _, num = orc.halton(1, offset=3 ** k)
        assert Fraction(int(num[0]), M3) == Fraction(1, 3 ** (k + 1))


def test_base3_float_is_nearest(orc):
    rng = np.random.default_rng(5)
    idx = np.concatenate([np.arange(1, 3000), rng.integers(1, 2 ** 24, 3000)])
    for i in idx:
        _, v, num = orc.halton(1, offset=int(i))
        assert v[0] == nearest_f32(Fraction(int(num[0]), M3)), i


def test_sincos_within_two_ulp_of_libm(orc):
    _, v, _ = orc.halton(65536, offset=1)
    grid = (np.arange(0, 1 << 16, dtype=np.float64) / (1 << 16)).astype(np.float32)
    for vs in (v, grid):
        c, s = orc.sincos_turns(vs)
        ang = 2.0 * np.pi * vs.astype(np.float64)
        for got, ref in ((c, np.cos(ang)), (s, np.sin(ang))):
            ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
            err = np.abs(got.astype(np.float64) - ref)
            # below 2^-20 the result's own ulp is tiny; there the bound is absolute
            bound = np.maximum(2.0 * ulp, 2.0 ** -45)
            assert np.all(err <= bound), (np.max(err / ulp))


def test_sincos_special_angles(orc):
    c, s = orc.sincos_turns(np.array([0.0, 0.25, 0.5, 0.75, 0.125], np.float32))
    assert (c[0], s[0]) == (1.0, 0.0)
    assert (abs(c[1]), s[1]) == (0.0, 1.0)
    assert (c[2], abs(s[2])) == (-1.0, 0.0)
    assert (abs(c[3]), s[3]) == (0.0, -1.0)
    h = math.sqrt(0.5)
    assert abs(c[4] - h) <= 2 * np.spacing(np.float32(h)) and abs(s[4] - h) <= 2 * np.spacing(np.float32(h))


def test_directions_unit_and_close_to_exact(orc):
    n = 65536
    d = orc.ray_dirs(n, 1).astype(np.float64)
    assert np.all(np.abs(np.linalg.norm(d, axis=1) - 1.0) <= 3 * 2.0 ** -24)
    u, v, num = orc.halton(n, 1)
    uu = u.astype(np.float64)                        # exact dyadic
    vv = num.astype(np.float64) / M3                 # exact value, rounded once to FP64
    z = 1.0 - 2.0 * uu
    st = np.sqrt(np.maximum(1.0 - z * z, 0.0))
    ref = np.stack([st * np.cos(2 * np.pi * vv), st * np.sin(2 * np.pi * vv), z], axis=1)
    # FP32 pipeline: RN(v) (<= 2^-25 turn -> 1.9e-7 rad), RN(pi/4), a few roundings
    assert np.max(np.abs(d - ref)) <= 4e-7
    assert np.all(d[:, 2] == z)                      # z = 1 - 2u is exact


def test_polar_strata_sum_to_zero(orc):
    """z = 1 - 2u over the first 2^m - 1 rays is an exact symmetric set: sums to 0."""
    for m in (4, 10, 16):
        d = orc.ray_dirs(2 ** m - 1, 1).astype(np.float64)
        assert math.fsum(d[:, 2]) == 0.0


def test_direction_quantisation(orc):
    d = orc.ray_dirs(4096, 1)
    D = orc.quantize_dirs(d)
    scaled = d.astype(np.float64) * 2.0 ** 24
    assert np.all(np.abs(D - scaled) <= 0.5)
    assert np.all(np.abs(D) <= 2 ** 24)
