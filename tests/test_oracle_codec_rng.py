"""Pins of the oracle's address codec and random-number source (not GPU)."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.ed as ED
from conftest import golden


def test_paper_bitstrings():
    g = golden("bitstrings.json")
    for case in g["cases"]:
        occ = case["occ"]
        m = O.Model(O.REAL_1D, len(occ), 1, case["N"], 1.0, 1.0)
        key = m.encode(occ)
        assert format(key, "b") == case["bits"]
        assert list(m.decode(key)) == occ


def test_roundtrip_all_6x6_states_and_order():
    m = O.Model(O.REAL_1D, 6, 1, 6, 1.0, 6.0)
    occs = ED.all_compositions(6, 6)
    assert len(occs) == math.comb(11, 6) == 462
    keys = [m.encode(o) for o in occs]
    assert len(set(keys)) == 462
    for o, k in zip(occs, keys):
        assert k < (1 << m.nbits)
        assert bin(k).count("1") == 6
        assert np.array_equal(m.decode(k), o)


@pytest.mark.parametrize("kind,Lx,Ly,N", [(O.REAL_2D, 8, 8, 64), (O.REAL_2D, 4, 3, 7),
                                          (O.MOM_1D, 32, 1, 32), (O.REAL_1D, 30, 1, 30)])
def test_roundtrip_random_states(kind, Lx, Ly, N):
    m = O.Model(kind, Lx, Ly, N, 1.0, 1.0)
    rng = np.random.default_rng(7)
    for _ in range(300):
        occ = np.bincount(rng.integers(0, m.M, N), minlength=m.M).astype(np.uint8)
        k = m.encode(occ)
        assert k.bit_length() <= N + m.M - 1
        assert np.array_equal(m.decode(k), occ)
    # 127-bit addresses of the 8x8, N = 64 model use the high word
    if m.nbits > 64:
        assert m.encode(np.r_[np.zeros(m.M - 1), N].astype(np.uint8)) >> 64 != 0


def test_decode_rejects_invalid():
    m = O.Model(O.REAL_1D, 6, 1, 6, 1.0, 6.0)
    with pytest.raises(ValueError):
        m.decode((1 << 11) | 0b11111)       # bit beyond N + M - 1
    with pytest.raises(ValueError):
        m.decode(0b11111)                   # five bosons


def test_philox_known_answers():
    g = golden("philox_kat.json")
    for case in g["cases"]:
        ctr = [int(x, 16) for x in case["ctr"]]
        key = [int(x, 16) for x in case["key"]]
        assert O.philox4x32_10(ctr, key) == tuple(int(x, 16) for x in case["out"])


def test_philox_counter_and_key_sensitivity():
    base = O.philox4x32_10([5, 6, 7, 8], [9, 10])
    for i in range(4):
        c = [5, 6, 7, 8]
        c[i] ^= 1
        assert O.philox4x32_10(c, [9, 10]) != base
    assert O.philox4x32_10([5, 6, 7, 8], [9, 11]) != base
    # the 128 output bits over many counters are balanced
    bits = 0
    for i in range(2000):
        for w in O.philox4x32_10([i, 0, 0, 0], [1, 2]):
            bits += bin(w).count("1")
    frac = bits / (2000 * 128)
    assert abs(frac - 0.5) < 0.005
