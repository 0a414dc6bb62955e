"""Counter-based random numbers: SplitMix64 (Steele, Lea & Flood 2014).

Every random draw of a workload is a pure function of (seed, counter), so a
value can be regenerated anywhere from its index alone.  The 64-bit mixer is
the published SplitMix64 finaliser: add the golden-ratio increment, then two
xor-shift-multiply rounds and a final xor-shift.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter) -> np.ndarray:
    """Hash (seed, counter) -> uint64, elementwise over ``counter``."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (np.uint64(seed) ^ c) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counter) -> np.ndarray:
    """Uniform double in [0, 1) from the top 53 bits of the hash."""
    z = splitmix64(seed, counter)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def stream(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n consecutive uniforms of one stream (counters offset .. offset+n-1)."""
    return uniform01(seed, np.arange(offset, offset + n, dtype=np.uint64))
