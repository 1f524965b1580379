"""Counter-based splitmix64 generator (Steele, Lea & Flood, OOPSLA 2014).

Every random number of a workload is a pure function of (seed, counter), so any
sample can be regenerated independently of draw order and of numpy's own
generators.  Seeds follow the convention ``config_id * 10**6 + instance``.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters) -> np.ndarray:
    """Return the splitmix64 outputs for state = seed + (counter + 1) * golden."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of splitmix64."""
    z = splitmix64(seed, np.arange(offset, offset + n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n standard normals by Box-Muller on consecutive uniform pairs."""
    u = uniform(seed, 2 * n, 2 * offset)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def randint(seed: int, n: int, lo: int, hi: int, offset: int = 0) -> np.ndarray:
    """n integers uniform in [lo, hi] (inclusive)."""
    u = uniform(seed, n, offset)
    return lo + np.minimum((u * (hi - lo + 1)).astype(np.int64), hi - lo)
