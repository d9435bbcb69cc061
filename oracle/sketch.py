"""Counter-based complex Gaussian sketch (oracle side; test infrastructure only).

The randomised SVD (Sec. 2) applies T_i to "a few random samples".  Both this oracle
and the CUDA path draw them from the same published generator, each side with its
own code, so that their sketches agree to rounding:

* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): the n-th output from seed s is
  mix(s + (n+1) * 0x9E3779B97F4A7C15) mod 2^64 with the finaliser
  z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
  z ^= z >> 31.
* Counter of entry (node c, column j, interface index x): n = 2 * idx and
  2 * idx + 1 with idx = (c * 4096 + j) * 2^20 + x.
* Uniforms: u1 = ((z1 >> 11) + 1) * 2^-53 in (0, 1], u2 = (z2 >> 11) * 2^-53.
* Box-Muller: rho = sqrt(-2 ln u1), re = rho cos(2 pi u2) / sqrt 2,
  im = rho sin(2 pi u2) / sqrt 2, so re and im are each N(0, 1/2).
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> int:
    """The n-th (0-based) SplitMix64 output from ``seed``."""
    z = (seed + (n + 1) * GAMMA) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def _splitmix64_vec(seed: int, n: np.ndarray) -> np.ndarray:
    """Vectorised splitmix64 over an array of counters (uint64 wrap-around)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK) + (n.astype(np.uint64) + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def gaussian_sketch(seed: int, node: int, rows: int, cols: int) -> np.ndarray:
    """Omega for child ``node``: rows x cols complex, re/im ~ N(0, 1/2)."""
    x = np.arange(rows, dtype=np.uint64)[:, None]
    j = np.arange(cols, dtype=np.uint64)[None, :]
    idx = (np.uint64(node) * np.uint64(4096) + j) * np.uint64(1 << 20) + x
    z1 = _splitmix64_vec(seed, np.uint64(2) * idx)
    z2 = _splitmix64_vec(seed, np.uint64(2) * idx + np.uint64(1))
    u1 = ((z1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (z2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    rho = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * np.pi * u2
    return (rho * np.cos(t) + 1j * rho * np.sin(t)) / np.sqrt(2.0)
