"""Pins for the oracle's Philox4x32-10 and uniform mapping."""
import numpy as np

import oracle
from tests.golden import philox_kat


def test_philox_known_answers():
    for ctr, key, want in philox_kat():
        got = oracle.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == want


def test_uniform_endpoints_open_and_fp32_exact():
    lo = oracle.uniform(0)
    hi = oracle.uniform(0xFFFFFFFF)
    assert lo == 2.0 ** -24
    assert hi == 1.0 - 2.0 ** -24
    for x in [0, 1, 511, 512, 12345678, 0x80000000, 0xFFFFFFFF]:
        u = oracle.uniform(x)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u       # exactly representable in FP32


def test_uniform_moments_from_counter_stream():
    us = []
    for i in range(4000):
        o = oracle.philox4x32_10([i, 7, 3, 0], [0x12964, 0])
        us.extend(oracle.uniform(int(x)) for x in o)
    us = np.array(us)
    n = us.size
    assert abs(us.mean() - 0.5) < 4 * np.sqrt(1 / 12 / n)
    assert abs(us.var() - 1 / 12) < 4 * np.sqrt(1 / 180 / n)
    # neighbouring counters decorrelated
    c = np.corrcoef(us[:-4], us[4:])[0, 1]
    assert abs(c) < 4 / np.sqrt(n)
