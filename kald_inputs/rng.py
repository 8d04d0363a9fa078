"""Seeded, counter-free random numbers for the synthetic test systems.

splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) written out from its published definition, so that
every run, on either machine, draws the same masses and the same random force
constants.  Pure integer arithmetic modulo 2**64; no numpy RNG is involved.
"""

from __future__ import annotations

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15
_MIX1 = 0xBF58476D1CE4E5B9
_MIX2 = 0x94D049BB133111EB


class SplitMix64:
    """64-bit generator; `next_u64` advances the state by the golden gamma."""

    def __init__(self, seed: int):
        self.state = int(seed) & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GOLDEN) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * _MIX1) & _MASK
        z = ((z ^ (z >> 27)) * _MIX2) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, n: int) -> int:
        """Integer in [0, n) (multiply-shift on the top 53 bits)."""
        return ((self.next_u64() >> 11) * n) >> 53

    def normal(self) -> float:
        """Standard normal by Box-Muller on two uniforms."""
        import math
        u1 = self.uniform()
        u2 = self.uniform()
        u1 = max(u1, 1e-300)
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def shuffled_labels(n: int, n_heavy: int, seed: int) -> list[int]:
    """Exact-count binary labels: `n_heavy` ones among `n`, placed by a
    Fisher-Yates shuffle driven by splitmix64(seed)."""
    labels = [1] * n_heavy + [0] * (n - n_heavy)
    g = SplitMix64(seed)
    for i in range(n - 1, 0, -1):
        j = g.below(i + 1)
        labels[i], labels[j] = labels[j], labels[i]
    return labels
