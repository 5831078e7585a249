"""The seeded input generators (CPU only).

SplitMix64 is pinned to the first outputs of the published generator seeded
with 0 (Steele, Lea and Flood 2014): the k-th output is the mix of k * gamma + gamma.
"""
import numpy as np

from synth import batched_problems, box_dims, splitmix64, sweep_ks, uniform_pm1

GAMMA = 0x9E3779B97F4A7C15


def test_splitmix64_published_sequence():
    states = np.array([(k * GAMMA) & 0xFFFFFFFFFFFFFFFF for k in range(3)], dtype=np.uint64)
    out = [int(v) for v in splitmix64(states)]
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_range_and_key():
    v = uniform_pm1(0, np.arange(100000))
    assert v.min() >= -1.0 and v.max() < 1.0 and abs(v.mean()) < 0.01
    np.testing.assert_array_equal(uniform_pm1(3, [5, 9]), uniform_pm1(3, np.array([5, 9])))
    assert not np.array_equal(uniform_pm1(0, [1, 2]), uniform_pm1(1, [1, 2]))


def test_box_dims_and_sweep():
    for k in range(0, 22):
        d = box_dims(k)
        assert d[0] * d[1] * d[2] == 2 ** k and max(d) <= 2 * min(d)
    assert sweep_ks(7) == list(range(5, 19))
    assert sweep_ks(3) == list(range(9, 22))


def test_batched_draws():
    p = batched_problems()
    assert len(p) == 256
    assert all(2 <= q["k"] <= 16 and q["N"] in (3, 5, 7) and 0 <= q["amp"] <= 0.1 for q in p)
    assert p == batched_problems()
