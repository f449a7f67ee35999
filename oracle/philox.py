"""Philox4xW-10 counter-based generator and the Gaussian noise drawn from it.

TEST INFRASTRUCTURE ONLY: see oracle/__init__.py.

The generator is Philox from Salmon, Moraes, Dror & Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC'11), written from that paper's description:
a 4-word counter is encrypted by R = 10 rounds, each round multiplying words 0
and 2 by fixed odd constants, taking the high and low halves of both products
and mixing the high halves with the other two words and the round key; the key
is advanced by a Weyl increment between rounds.  W = 32 is the variant the noise
uses; W = 64 is kept because numpy's Philox bit generator is the 4x64-10
variant, which lets tests pin the round structure against a library routine.

The paper (Sec. II.A, Eq. EM) only requires W and W~ to be independent vectors of
i.i.d. standard normals; this counter layout is the library's choice:
    key     = (seed & 0xffffffff, seed >> 32)
    counter = (pair index k//2 of the particle-major noise index k = 3 i + c,
               step, stream, instance)      stream 0: W (Lanczos), 1: W~ (RFD)
The four 32-bit outputs (x0, x1, x2, x3) give two 53-bit uniforms in (0, 1]:
    u1 = ((x0 >> 5) * 2^26 + (x1 >> 6) + 1) * 2^-53,  u2 likewise from (x2, x3),
and the Box-Muller transform gives the normals of indices 2p and 2p + 1:
    n_{2p} = sqrt(-2 ln u1) cos(2 pi u2),   n_{2p+1} = sqrt(-2 ln u1) sin(2 pi u2).
"""
import numpy as np

# Multipliers and Weyl key increments of the published generator, per word width.
_CONST = {
    32: dict(M=(0xD2511F53, 0xCD9E8D57), K=(0x9E3779B9, 0xBB67AE85)),
    64: dict(M=(0xD2E7470EE14C6C93, 0xCA5A826395121157), K=(0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)),
}


def philox4(counter, key, width=32, rounds=10):
    """Encrypt one 4-word counter under a 2-word key; plain Python integers in and out."""
    mask = (1 << width) - 1
    M0, M1 = _CONST[width]["M"]
    K0, K1 = _CONST[width]["K"]
    c = [int(v) & mask for v in counter]
    k0, k1 = int(key[0]) & mask, int(key[1]) & mask
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + K0) & mask
            k1 = (k1 + K1) & mask
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> width, p0 & mask
        hi1, lo1 = p1 >> width, p1 & mask
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c


def philox4x32_vec(c0, c1, c2, c3, k0, k1, rounds=10):
    """Vectorised Philox4x32 over numpy arrays of counters (uint64 arrays holding 32-bit words)."""
    mask = np.uint64(0xFFFFFFFF)
    M0, M1 = (np.uint64(v) for v in _CONST[32]["M"])
    K0, K1 = (np.uint64(v) for v in _CONST[32]["K"])
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & mask for v in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + K0) & mask
            k1 = (k1 + K1) & mask
        p0 = M0 * c0  # < 2^64: exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def raw_words(n_pairs, seed, step, stream, instance=0):
    """The four 32-bit outputs for pair counters 0 .. n_pairs-1 (arrays of shape (n_pairs,))."""
    p = np.arange(n_pairs, dtype=np.uint64)
    z = np.zeros_like(p)
    return philox4x32_vec(p, z + np.uint64(step & 0xFFFFFFFF), z + np.uint64(stream & 0xFFFFFFFF),
                          z + np.uint64(instance & 0xFFFFFFFF), seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def normals(n, seed, step, stream, instance=0):
    """n standard normals, element k is the noise of particle-major index k (k = 3 i + c)."""
    npairs = (n + 1) // 2
    x0, x1, x2, x3 = raw_words(npairs, seed, step, stream, instance)
    two26 = 67108864.0
    u1 = ((x0 >> np.uint64(5)).astype(np.float64) * two26 + (x1 >> np.uint64(6)).astype(np.float64) + 1.0) * 2.0**-53
    u2 = ((x2 >> np.uint64(5)).astype(np.float64) * two26 + (x3 >> np.uint64(6)).astype(np.float64) + 1.0) * 2.0**-53
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * npairs)
    out[0::2] = rad * np.cos(2.0 * np.pi * u2)
    out[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return out[:n]
