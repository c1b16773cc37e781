"""SplitMix64 in counter form (Steele, Lea & Flood 2014), vectorised with numpy.

``splitmix64(seed, idx)`` returns the idx-th 64-bit output of the SplitMix64
stream whose initial state is ``seed``:  state_i = seed + (idx+1)*G (mod 2^64),
then the published finaliser
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z =  z ^ (z >> 31)
Uniform doubles take the top 53 bits: u = (z >> 11) * 2^-53 in [0, 1).
"""
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, idx):
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (idx + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed, idx):
    """Doubles in [0, 1) from the top 53 bits of each SplitMix64 output."""
    z = splitmix64(seed, idx)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_pm_half(seed, idx):
    """Doubles in [-1/2, 1/2): uniform01 - 0.5 (the start-block distribution)."""
    return uniform01(seed, idx) - 0.5


def normals(seed, n, offset=0):
    """n standard normals by Box-Muller on consecutive uniform pairs.

    Pair p uses outputs offset+2p and offset+2p+1: r = sqrt(-2 ln(1-u1)),
    n_{2p} = r cos(2 pi u2), n_{2p+1} = r sin(2 pi u2).
    """
    npair = (n + 1) // 2
    idx = offset + np.arange(2 * npair, dtype=np.uint64)
    u = uniform01(seed, idx)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))
    out = np.empty(2 * npair)
    out[0::2] = r * np.cos(2.0 * np.pi * u2)
    out[1::2] = r * np.sin(2.0 * np.pi * u2)
    return out[:n]
