"""Seeded input generator: SplitMix64 pinned to its published stream."""
import numpy as np

import synth


def test_splitmix64_published_seed0_stream():
    # SplitMix64 started from state 0: the first outputs of the reference
    # generator (Steele, Lea, Flood 2014; public-domain reference code).
    got = synth.splitmix64(np.arange(4, dtype=np.uint64))
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [int(v) for v in got] == want


def test_splitmix64_sequential_equals_counter():
    # the counter form must equal stepping the state by GAMMA one draw at a time
    M = (1 << 64) - 1
    s = 0
    seq = []
    for _ in range(16):
        s = (s + 0x9E3779B97F4A7C15) & M
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        seq.append(z ^ (z >> 31))
    got = synth.splitmix64(np.arange(16, dtype=np.uint64))
    assert [int(v) for v in got] == seq


def test_uniform_range_and_exact_fp32():
    u = synth.uniform_pm1(0, 0, (8, 8, 8))
    assert u.dtype == np.float32
    assert u.min() >= -1.0 and u.max() < 1.0
    # value = (2m - 2^24) / 2^24 with m < 2^24: integer numerator
    num = u.astype(np.float64) * 2.0**23
    assert np.all(num == np.round(num))
    # first value from the counter 0
    x0 = int(synth.splitmix64(np.array([0], dtype=np.uint64))[0])
    assert u.ravel()[0] == np.float32(2.0 * (x0 >> 40) * 2.0**-24 - 1.0)


def test_normal_moments_and_fields_independent():
    z = synth.normal(0, 0, (64, 64, 64))
    assert abs(z.mean()) < 0.01
    assert abs(z.std() - 1.0) < 0.01
    z1 = synth.normal(0, 1, (64, 64, 64))
    assert abs(np.corrcoef(z.ravel(), z1.ravel())[0, 1]) < 0.01
    # reproducible and seed-dependent
    assert np.array_equal(z, synth.normal(0, 0, (64, 64, 64)))
    assert not np.array_equal(z, synth.normal(1, 0, (64, 64, 64)))


def test_chunking_is_invisible():
    n = synth._CHUNK + 1000
    a = synth.uniform_pm1(3, 2, (n,))
    x = synth.splitmix64(np.uint64(synth.counter_base(3, 2)) + np.arange(n - 5, n, dtype=np.uint64))
    tail = (2.0 * ((x >> np.uint64(40)).astype(np.float64) * 2.0**-24) - 1.0).astype(np.float32)
    assert np.array_equal(a[-5:], tail)
