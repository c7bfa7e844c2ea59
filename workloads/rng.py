"""Counter-based SplitMix64 stream (Steele, Lea and Flood, OOPSLA 2014).

Used so that every synthetic workload is bit-identical on every machine and
Python/numpy version: the stream is defined by integer arithmetic only.
"""
import numpy as np

_M64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def _mix(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


class SplitMix64:
    """Scalar SplitMix64 stream with a few convenience draws."""

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + _GAMMA) & _M64
        return _mix(self.state)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive); rejection-free modulo is
        fine here because spans are tiny compared with 2^64."""
        span = hi - lo + 1
        return lo + self.next_u64() % span

    def uniform(self) -> float:
        """Uniform float in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def bernoulli(self, p: float) -> bool:
        return self.uniform() < p

    def u64_block(self, n: int) -> np.ndarray:
        """n consecutive outputs as a numpy uint64 array (vectorised)."""
        idx = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + idx * np.uint64(_GAMMA)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * _GAMMA) & _M64
        return z
