"""Counter-based random numbers for input generation.

The generator is the SplitMix64 output function (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) evaluated at
``state = key + (counter + 1) * 0x9E3779B97F4A7C15``. Each input family uses its
own key (seed mixed with a stream tag), so the numbers drawn for a problem never
coincide with the hash that the solver derives from its own seed.
"""
import numpy as np

from . import detmath

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed, stream):
    # stream tags keep input families independent of each other
    with np.errstate(over="ignore"):
        return _mix(np.uint64(seed) * np.uint64(0xD1B54A32D192ED03) + np.uint64(stream) + _GOLDEN)


def splitmix_bits(seed, stream, count, offset=0):
    ctr = np.arange(offset, offset + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = _key(seed, stream) + (ctr + np.uint64(1)) * _GOLDEN
    return _mix(state)


def splitmix_uniform(seed, stream, count, offset=0):
    """Uniform doubles in [0, 1) with 53 random bits each."""
    bits = splitmix_bits(seed, stream, count, offset)
    return (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def splitmix_normal(seed, stream, count, offset=0):
    """Standard normals by the Box-Muller transform on pairs of uniforms."""
    u = splitmix_uniform(seed, stream, 2 * count, 2 * offset)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * detmath.log(u1)) * detmath.cos(2.0 * np.pi * u2)
