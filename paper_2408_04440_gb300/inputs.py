"""Seeded synthetic inputs shared by the tests and the benchmark.

Holds none of the method's arithmetic: only the draws that pick the workload.

Batched workload: independent covariances with bandlimits uniform in
L in {8, ..., 64} and correlation lengths beta uniform in [2, 8).  The draws
come from SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) started at the seed, taken in the order L_0, beta_0,
L_1, beta_1, ...:
    L    = 8 + (x mod 57)
    beta = 2 + 6 * (x >> 11) * 2^-53
"""
from __future__ import annotations

MASK64 = (1 << 64) - 1


def splitmix64(state: int):
    """Generator of SplitMix64 outputs from the 64-bit seed `state`."""
    while True:
        state = (state + 0x9E3779B97F4A7C15) & MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        yield z ^ (z >> 31)


def batch_draws(count: int, seed: int = 3, lmin: int = 8, lmax: int = 64, bmin: float = 2.0, bmax: float = 8.0):
    """(L_b, beta_b) for b < count."""
    g = splitmix64(seed)
    out = []
    span = lmax - lmin + 1
    for _ in range(count):
        L = lmin + next(g) % span
        beta = bmin + (bmax - bmin) * (next(g) >> 11) * 2.0**-53
        out.append((int(L), float(beta)))
    return out
