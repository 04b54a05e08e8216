"""SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used to make every synthetic model reproducible from
its seed.  Pure Python; draws only structure, never the method's arithmetic."""

MASK64 = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = int(seed) & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) by the multiply-high reduction."""
        if n <= 0:
            raise ValueError("n must be positive")
        return (self.next() * n) >> 64

    def uniform_int(self, lo: int, hi: int) -> int:
        """Uniform integer in the closed range [lo, hi]."""
        return lo + self.below(hi - lo + 1)

    def chance(self, p: float) -> bool:
        return self.next() < int(p * (1 << 64))

    def random(self) -> float:
        return (self.next() >> 11) * (1.0 / (1 << 53))
