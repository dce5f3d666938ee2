"""Philox4x32-10 counter-based generator and the sampler's draw layout (oracle side).

TEST INFRASTRUCTURE ONLY: part of the FP64 CPU oracle; never imported by the
product library (which implements the same published generator in its own code).

Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC 2011): ten rounds of
  (x0, x1, x2, x3) -> (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0))
with M0 = 0xD2511F53, M1 = 0xCD9E8D57 and a Weyl key schedule
k0 += 0x9E3779B9, k1 += 0xBB67AE85 between rounds.

The paper draws random numbers for the prior sample, the Markov kernel and the
resampling step but fixes no generator; this layout is the library's convention:
counter = (c0 block, c1 particle, c2 event, c3 purpose), key = the 64-bit seed.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = np.uint64(0xFFFFFFFF)

PURPOSE_PRIOR = 1
PURPOSE_PCN_XI = 2
PURPOSE_PCN_U = 3
PURPOSE_RESAMPLE = 4
PURPOSE_DA_U = 5


def philox4x32_10(c0, c1, c2, c3, seed):
    """Vectorised Philox4x32-10. Counters are uint32-valued arrays (broadcast), seed a uint64."""
    x0, x1, x2, x3 = (np.asarray(c, dtype=np.uint64) & MASK for c in (c0, c1, c2, c3))
    x0, x1, x2, x3 = np.broadcast_arrays(x0, x1, x2, x3)
    k0 = int(seed) & 0xFFFFFFFF
    k1 = (int(seed) >> 32) & 0xFFFFFFFF
    for r in range(10):
        p0 = M0 * x0                      # exact: 32x32 -> 64 bits fits in uint64
        p1 = M1 * x2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        x0, x1, x2, x3 = (hi1 ^ x1 ^ np.uint64(k0), lo1, hi0 ^ x3 ^ np.uint64(k1), lo0)
        if r < 9:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
    return x0, x1, x2, x3


def u53(hi, lo):
    """Uniform double in [0, 1) from two 32-bit words (27 high bits of hi, 26 of lo)."""
    hi = np.asarray(hi, dtype=np.uint64) >> np.uint64(5)
    lo = np.asarray(lo, dtype=np.uint64) >> np.uint64(6)
    return (hi.astype(np.float64) * 67108864.0 + lo.astype(np.float64)) * (1.0 / 9007199254740992.0)


def normals(J, K, event, purpose, seed):
    """(J, K) standard normals by Box-Muller: block b of particle j gives entries 2b, 2b+1."""
    nb = (K + 1) // 2
    b = np.arange(nb, dtype=np.uint64)[None, :]
    j = np.arange(J, dtype=np.uint64)[:, None]
    x0, x1, x2, x3 = philox4x32_10(b, j, event, purpose, seed)
    u1 = u53(x0, x1)
    u2 = u53(x2, x3)
    r = np.sqrt(-2.0 * np.log(1.0 - u1))          # 1 - u1 in (0, 1]
    z = np.empty((J, 2 * nb))
    z[:, 0::2] = r * np.cos(2.0 * np.pi * u2)
    z[:, 1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:, :K]


def uniforms_open(J, event, purpose, seed):
    """(J,) uniforms in (0, 1]: 1 - u53 of block 0 of each particle."""
    j = np.arange(J, dtype=np.uint64)
    x0, x1, _, _ = philox4x32_10(0, j, event, purpose, seed)
    return 1.0 - u53(x0, x1)


def uniform_scalar(event, purpose, seed):
    """One uniform in [0, 1) (resampling offset): block 0, particle 0."""
    x0, x1, _, _ = philox4x32_10(0, 0, event, purpose, seed)
    return float(u53(x0, x1))
