"""Counter-based random numbers (SplitMix64 finaliser, Steele, Lea & Flood 2014).

Every variate is a pure function of (seed, stream, index), so a field comes
out the same whatever the chunking or thread count that produced it.
Uniforms come from the top 53 bits of the 64-bit hash; normals from the
Box-Muller transform of consecutive uniform pairs.
"""

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z):
    """SplitMix64 output function applied to an array of uint64 states."""
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed, stream):
    """64-bit key for one (seed, stream) pair."""
    with np.errstate(over="ignore"):
        k = _mix64(np.array([np.uint64(seed) * _GOLDEN + np.uint64(stream)], dtype=np.uint64))
        return _mix64(k ^ np.uint64(0xD1B54A32D192ED03))[0]


def counter_uniforms(seed, stream, start, count):
    """``count`` uniforms in (0, 1] for counters start .. start+count-1."""
    key = _key(seed, stream)
    with np.errstate(over="ignore"):
        ctr = np.arange(start, start + count, dtype=np.uint64)
        z = _mix64(key + (ctr + np.uint64(1)) * _GOLDEN)
    # 53 random bits, shifted into (0, 1] so that log() below is finite.
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def counter_normals(seed, stream, count, chunk=1 << 24):
    """``count`` standard normals; normal i uses uniforms 2*(i//2), 2*(i//2)+1."""
    npairs = (count + 1) // 2
    out = np.empty(2 * npairs, dtype=np.float64)
    for p0 in range(0, npairs, chunk):
        n = min(chunk, npairs - p0)
        u = counter_uniforms(seed, stream, 2 * p0, 2 * n)
        rad = np.sqrt(-2.0 * np.log(u[0::2]))
        ang = (2.0 * np.pi) * u[1::2]
        out[2 * p0 : 2 * (p0 + n) : 2] = rad * np.cos(ang)
        out[2 * p0 + 1 : 2 * (p0 + n) : 2] = rad * np.sin(ang)
    return out[:count]
