"""Philox4x32-10 counter-based generator and Box-Muller normals (oracle side).

The ASE noise of the channel (Sec. IV-A: white Gaussian noise added by every
EDFA) is drawn from a counter-based generator so that the CUDA path and this
oracle produce the same realisation without passing the noise as an input.
Both sides implement, independently, the published definition of Philox4x32
with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11):

  round:  (c0, c1, c2, c3), key (k0, k1)
          hi0:lo0 = M0 * c0,  hi1:lo1 = M1 * c2   (32x32 -> 64-bit products)
          c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
  key schedule between rounds: k0 += W0, k1 += W1 (mod 2^32)
  M0 = 0xD2511F53, M1 = 0xCD9E8D57, W0 = 0x9E3779B9, W1 = 0xBB67AE85.

Pinned by the known-answer vectors published with the Random123 library
(tests/golden/philox4x32_10_kat.txt).

Counter layout used for ASE (a reading; the paper does not fix one):
  key = (seed & 0xffffffff, seed >> 32)
  ctr = (k >> 1, waveform b, span s, counter & 0xffffffff)
Frequency bin k uses words (0, 1) if k is even and (2, 3) if k is odd:
  u1 = (w_a + 0.5) 2^-32,  u2 = (w_b + 0.5) 2^-32,
  g  = sqrt(-2 ln u1) (cos 2 pi u2 + j sin 2 pi u2)     (E|g|^2 = 2).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32-10 on arrays.

    ctr: uint32-valued array [..., 4]; key: uint32-valued array [..., 2]
    (broadcastable).  Returns uint32 array [..., 4].
    """
    c = [np.asarray(ctr[..., i], dtype=np.uint64) for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64)
    k1 = np.asarray(key[..., 1], dtype=np.uint64)
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c[0]          # < 2^64, exact in uint64
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=-1).astype(np.uint32)


def ase_normals(n: int, batch: int, span: int, seed: int, counter: int) -> np.ndarray:
    """Unit-variance-per-component complex normals g[b, k] (E|g|^2 = 2)."""
    k = np.arange(n, dtype=np.uint64)
    b = np.arange(batch, dtype=np.uint64)
    ctr = np.zeros((batch, n, 4), dtype=np.uint64)
    ctr[..., 0] = (k >> np.uint64(1))[None, :]
    ctr[..., 1] = b[:, None]
    ctr[..., 2] = np.uint64(span)
    ctr[..., 3] = np.uint64(counter & 0xFFFFFFFF)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    w = philox4x32_10(ctr, key).astype(np.float64)
    odd = (np.arange(n) % 2 == 1)[None, :]
    wa = np.where(odd, w[..., 2], w[..., 0])
    wb = np.where(odd, w[..., 3], w[..., 1])
    u1 = (wa + 0.5) * 2.0 ** -32
    u2 = (wb + 0.5) * 2.0 ** -32
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2 * np.pi * u2) + 1j * r * np.sin(2 * np.pi * u2)
