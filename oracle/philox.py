"""Philox4x32-10 counter-based generator and the normal transform.

Test infrastructure (see ``oracle/__init__``).

Philox4x32-10 is written from its published definition (J. K. Salmon,
M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11): ten rounds of the S-box
  (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
with multipliers M0 = 0xD2511F53, M1 = 0xCD9E8D57, the key bumped by the Weyl
constants (0x9E3779B9, 0xBB67AE85) between rounds.

Normal transform (a format shared with the CUDA library):
  u1 = ((x0 >> 5) * 2^26 + (x1 >> 6) + 1) * 2^-53   in (0, 1]
  u2 = ((x2 >> 5) * 2^26 + (x3 >> 6) + 1) * 2^-53
  z0 = sqrt(-2 ln u1) cos(2 pi u2),  z1 = sqrt(-2 ln u1) sin(2 pi u2)  (Box–Muller)
Stream layout: key = (seed mod 2^32, seed div 2^32); the normal with index q of
sample s in stream t is half (q mod 2) of the pair drawn with counter
(floor(q/2) mod 2^32, s, t, floor(q/2) div 2^32).
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)

STREAM_NOISE = 0
STREAM_TARGET = 1


def philox4x32_10(ctr, key):
    """Philox4x32-10.  ctr: [4, n] uint32-valued, key: [2] or [2, n].  Returns [4, n] uint32."""
    c = [np.asarray(ctr[i], dtype=np.uint64) & _MASK for i in range(4)]
    k0 = np.asarray(key[0], dtype=np.uint64) & _MASK
    k1 = np.asarray(key[1], dtype=np.uint64) & _MASK
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c).astype(np.uint32)


def uniform53(x_hi, x_lo):
    """53-bit uniform in (0, 1] from two 32-bit words."""
    a = np.asarray(x_hi, dtype=np.uint64) >> np.uint64(5)
    b = np.asarray(x_lo, dtype=np.uint64) >> np.uint64(6)
    return ((a * np.uint64(1 << 26) + b + np.uint64(1)).astype(np.float64)) * 2.0**-53


def normals(seed, sample, q, stream=STREAM_NOISE):
    """Standard normals with global indices ``q`` (int array) of one sample."""
    q = np.asarray(q, dtype=np.int64)
    pair = q // 2
    n = len(pair)
    ctr = np.stack([pair & 0xFFFFFFFF, np.full(n, sample), np.full(n, stream), pair >> 32])
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    x = philox4x32_10(ctr, key)
    u1 = uniform53(x[0], x[1])
    u2 = uniform53(x[2], x[3])
    rad = np.sqrt(-2.0 * np.log(u1))
    z0 = rad * np.cos(2.0 * np.pi * u2)
    z1 = rad * np.sin(2.0 * np.pi * u2)
    return np.where(q % 2 == 0, z0, z1)
