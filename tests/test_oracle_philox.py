"""Pins of the oracle's Philox generator: the published known-answer vectors (4x32)
and numpy's independent Philox-4x64-10 bit generator (same round structure)."""
import os

import numpy as np

from oracle.philox import philox4x32_10, philox4x64_10_scalar, uniform53

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox4x32_known_answers():
    n = 0
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(s, 16) for s in line.split()]
        out = philox4x32_10(v[0:4], v[4:6])
        assert [int(o) for o in out] == v[6:10]
        n += 1
    assert n == 3


def test_philox4x64_matches_numpy():
    for key in ([0, 0], [3, 5], [0xDEADBEEF12345678, 0x0123456789ABCDEF]):
        bg = np.random.Philox(counter=np.array([7, 0, 0, 0], dtype=np.uint64),
                              key=np.array(key, dtype=np.uint64))
        raw = [int(r) for r in bg.random_raw(8)]
        # numpy increments the counter before each block
        assert raw[:4] == philox4x64_10_scalar([8, 0, 0, 0], key)
        assert raw[4:] == philox4x64_10_scalar([9, 0, 0, 0], key)


def test_philox_vectorised_equals_scalar_counters():
    ctr0 = np.arange(100, dtype=np.uint32)
    out = philox4x32_10((ctr0, 5, 7, 1), (11, 13))
    for i in (0, 37, 99):
        single = philox4x32_10((i, 5, 7, 1), (11, 13))
        assert [int(o[i]) for o in out] == [int(s) for s in single]


def test_uniform53_range_and_resolution():
    assert uniform53(0, 0) == 0.0
    top = uniform53(0xFFFFFFFF, 0xFFFFFFFF)
    assert top == 1.0 - 2.0 ** -53
    assert uniform53(0, 1 << 6) == 2.0 ** -53
