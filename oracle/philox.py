"""Philox4x32-10 and the Gaussian draws of the method (oracle side).

Philox4x32-10 follows its published definition (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11): a 128-bit counter of four
32-bit words and a 64-bit key of two words; each of the 10 rounds multiplies
words 0 and 2 by the constants 0xD2511F53 and 0xCD9E8D57, splits the 64-bit
products into high and low halves and recombines them with words 1, 3 and the
key; the key is bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85) between
rounds.

The map to normals is this library's own convention (the paper only asks for
standard Gaussian matrices, Sec. 3.1):
  element e (column-major linear index) of the stream (seed, stream) uses the
  Philox block with counter (p_lo, p_hi, stream_lo, stream_hi), p = e // 2, key
  (seed_lo, seed_hi). Its words give two 53-bit uniforms in (0, 1)
      u = ((w_a >> 5) * 2^26 + (w_b >> 6) + 0.5) / 2^53
  from (w0, w1) and (w2, w3), and Box-Muller gives
      r = sqrt(-2 ln u1), z_even = r cos(2 pi u2), z_odd = r sin(2 pi u2).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(counter, key):
    """Apply Philox4x32-10 to arrays of counters.

    counter: uint64 array (..., 4) holding 32-bit words; key: (k0, k1) ints.
    Returns uint64 array (..., 4) of 32-bit output words.
    """
    c = np.asarray(counter, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
        p0 = M0 * c0                      # exact: both factors < 2^32
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0)), lo1, (hi0 ^ c3 ^ np.uint64(k1)), lo0
    return np.stack([c0, c1, c2, c3], axis=-1)


def _uniform53(wa, wb):
    a = (wa >> np.uint64(5)).astype(np.float64)
    b = (wb >> np.uint64(6)).astype(np.float64)
    return (a * 67108864.0 + b + 0.5) / 9007199254740992.0


def gaussian(seed: int, stream: int, rows: int, cols: int, col0: int = 0) -> np.ndarray:
    """Columns col0 .. col0+cols-1 of the (rows x infinity) standard-normal matrix
    of stream ``stream``; element (i, j) has linear index e = i + rows * j."""
    i = np.arange(rows, dtype=np.uint64)[:, None]
    j = np.arange(col0, col0 + cols, dtype=np.uint64)[None, :]
    e = i + np.uint64(rows) * j
    p = e >> np.uint64(1)
    ctr = np.stack([p & MASK32, p >> np.uint64(32),
                    np.full_like(p, stream & 0xFFFFFFFF),
                    np.full_like(p, (stream >> 32) & 0xFFFFFFFF)], axis=-1)
    w = philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))
    u1 = _uniform53(w[..., 0], w[..., 1])
    u2 = _uniform53(w[..., 2], w[..., 3])
    r = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    odd = (e & np.uint64(1)).astype(bool)
    return np.where(odd, r * np.sin(ang), r * np.cos(ang))
