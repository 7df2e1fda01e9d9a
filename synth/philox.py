"""Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw 2011,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), vectorised in numpy.

Each call maps a batch of 128-bit counters and one 64-bit key to 128 random
bits per counter.  The generator is keyed by the Fourier mode of the initial
density field, so a mode draws the same numbers at every grid resolution.
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)
_SH = np.uint64(32)


def philox4x32(c0, c1, c2, c3, key0, key1, rounds=10):
    """Apply `rounds` Philox-4x32 rounds to counters (c0..c3) under (key0, key1).

    Counter words are numpy arrays of 32-bit values (any unsigned dtype);
    the key is two Python ints.  Returns four uint32 arrays.
    """
    x0 = np.asarray(c0, dtype=np.uint64) & _MASK
    x1 = np.asarray(c1, dtype=np.uint64) & _MASK
    x2 = np.asarray(c2, dtype=np.uint64) & _MASK
    x3 = np.asarray(c3, dtype=np.uint64) & _MASK
    k0 = int(key0) & 0xFFFFFFFF
    k1 = int(key1) & 0xFFFFFFFF
    for _ in range(rounds):
        p0 = _M0 * x0                      # 32x32 -> 64-bit products
        p1 = _M1 * x2
        hi0, lo0 = p0 >> _SH, p0 & _MASK
        hi1, lo1 = p1 >> _SH, p1 & _MASK
        x0, x1, x2, x3 = (hi1 ^ x1 ^ np.uint64(k0), lo1,
                          hi0 ^ x3 ^ np.uint64(k1), lo0)
        k0 = (k0 + _W0) & 0xFFFFFFFF
        k1 = (k1 + _W1) & 0xFFFFFFFF
    return (x0.astype(np.uint32), x1.astype(np.uint32),
            x2.astype(np.uint32), x3.astype(np.uint32))


def uniform01(u32):
    """Map uint32 words to doubles in (0, 1): (u + 1/2) / 2^32."""
    return (np.asarray(u32, dtype=np.float64) + 0.5) * (1.0 / 4294967296.0)


def mode_gaussians(nx, ny, nz, seed):
    """Two independent standard normals per integer wave-vector (nx, ny, nz).

    The counter is the wave-vector (two's-complement 32-bit words) and the key
    is the 64-bit seed, so the draw for a mode does not depend on the grid
    size.  Box-Muller on the first two words gives the pair.
    """
    c0 = np.asarray(nx, dtype=np.int64).astype(np.uint64) & _MASK
    c1 = np.asarray(ny, dtype=np.int64).astype(np.uint64) & _MASK
    c2 = np.asarray(nz, dtype=np.int64).astype(np.uint64) & _MASK
    c3 = np.zeros_like(c0)
    r0, r1, _, _ = philox4x32(c0, c1, c2, c3, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u1 = uniform01(r0)
    u2 = uniform01(r1)
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return rad * np.cos(ang), rad * np.sin(ang)
