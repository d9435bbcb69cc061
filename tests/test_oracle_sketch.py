"""Pins of the oracle's sketch generator (CPU only)."""
import os

import numpy as np
from scipy import stats

from oracle.sketch import gaussian_sketch, splitmix64

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.txt")


def _golden():
    with open(GOLDEN) as fh:
        return [int(t) for t in fh.read().split() if t.isdigit()]


def test_splitmix64_published_outputs():
    assert [splitmix64(1234567, n) for n in range(5)] == _golden()


def test_gaussian_sketch_distribution():
    Om = gaussian_sketch(99, 5, 2000, 40)
    z = np.concatenate([Om.real.ravel(), Om.imag.ravel()])
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 0.5) < 0.01
    assert stats.kstest(z / np.sqrt(0.5), "norm").pvalue > 1e-3
    # real and imaginary parts uncorrelated
    assert abs(np.corrcoef(Om.real.ravel(), Om.imag.ravel())[0, 1]) < 0.02


def test_gaussian_sketch_counter_structure():
    a = gaussian_sketch(7, 3, 50, 10)
    b = gaussian_sketch(7, 3, 80, 12)
    assert np.array_equal(a, b[:50, :10])         # entries depend only on (seed, node, col, row)
    assert not np.allclose(a, gaussian_sketch(7, 4, 50, 10))
    assert not np.allclose(a, gaussian_sketch(8, 3, 50, 10))
